"""The allocation-free rescoring entry point, mad_rescore_noalloc.

Some callers cannot allocate device memory -- their GPU memory is reserved
up front by another allocator, or they cannot afford cudaMalloc's
device-wide synchronisation -- so the library offers one entry point that
works out of a fixed static device array instead.  These tests call it
through the C ABI and check that it returns the same pairs and the same
bits as mad_rescore, twice in a row (the shared array keeps the previous
call's contents, which must not leak into the next result), and that it
refuses candidate lists beyond its fixed capacity.

This file is collected last on purpose; it also runs alone in a fresh
process (it builds the library and its inputs itself).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from gpu_cases import Case  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _candidates(case, s, seed, tprime):
    import paper_1506_03872_gb300 as mad
    mad.mad_sample(case.ctx.ctx, s, seed)
    return mad.mad_topk(case.ctx.ctx, tprime)


@pytest.mark.parametrize("name,t", [("plain_small", 10), ("dense_ragged_f32", 97),
                                    ("chung_lu_small", 50)])
def test_noalloc_matches_rescore_twice(name, t):
    import paper_1506_03872_gb300 as mad
    s = 200_000
    c = Case(name, s_max=s)
    try:
        cand, nc = _candidates(c, s, 21, 4000)
        assert nc > t
        ref, nr = mad.mad_rescore(c.ctx.ctx, cand, nc, t)
        ri, rj, rx, rc = mad.decode_pairs(ref, nr)
        for _ in range(2):
            got, ng = mad.mad_rescore_noalloc(c.Am, c.Bm, cand, nc, t)
            gi, gj, gx, gc = mad.decode_pairs(got, ng)
            assert ng == nr
            assert np.array_equal(gi, ri) and np.array_equal(gj, rj)
            assert np.array_equal(gx, rx)
            # bit-identical dot products (same fixed summation order)
            assert np.array_equal(gc.view(np.int64), rc.view(np.int64))
    finally:
        c.close()


def test_noalloc_small_then_large_request():
    """A short call after a longer one must not see the longer call's data."""
    import paper_1506_03872_gb300 as mad
    s = 200_000
    c = Case("plain_small", s_max=s)
    try:
        cand, nc = _candidates(c, s, 22, 3000)
        big, nb = mad.mad_rescore_noalloc(c.Am, c.Bm, cand, nc, 200)
        small, ns = mad.mad_rescore_noalloc(c.Am, c.Bm, cand[:7], 7, 5)
        ref, nr = mad.mad_rescore(c.ctx.ctx, cand[:7], 7, 5)
        assert ns == nr == 5
        assert np.array_equal(small[:ns].cpu().numpy(), ref[:nr].cpu().numpy())
    finally:
        c.close()


def test_noalloc_rejects_more_candidates_than_its_array_holds():
    import paper_1506_03872_gb300 as mad
    c = Case("plain_small", s_max=1 << 16)
    try:
        n = mad.MAD_NOALLOC_MAX_CANDIDATES + 1
        i = np.arange(n) % c.m
        j = np.arange(n) // c.m
        cand = mad.encode_pairs(i, j)
        with pytest.raises(mad.MadError) as e:
            mad.mad_rescore_noalloc(c.Am, c.Bm, cand, n, 10)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
    finally:
        c.close()


def test_noalloc_bad_candidate_then_valid_call():
    """A candidate outside A (i >= m) is refused with MAD_ERR_ARG; the error
    word lives in the shared array, and the next valid call must start from
    a cleared status and match mad_rescore."""
    import paper_1506_03872_gb300 as mad
    s = 200_000
    c = Case("plain_small", s_max=s)
    try:
        cand, nc = _candidates(c, s, 23, 500)
        bad = mad.encode_pairs(np.array([3, c.m + 5]), np.array([4, 1]))
        with pytest.raises(mad.MadError) as e:
            mad.mad_rescore_noalloc(c.Am, c.Bm, bad, 2, 2)
        assert e.value.status == mad.MAD_ERR_ARG
        got, ng = mad.mad_rescore_noalloc(c.Am, c.Bm, cand, nc, 20)
        ref, nr = mad.mad_rescore(c.ctx.ctx, cand, nc, 20)
        assert ng == nr == 20
        assert np.array_equal(got[:ng].cpu().numpy(), ref[:nr].cpu().numpy())
    finally:
        c.close()


def test_noalloc_allocates_no_device_memory():
    """After a warm-up call, a call leaves the device's free memory and the
    caching allocator's reserved bytes unchanged (the output buffer is
    allocated by the caller beforehand)."""
    import paper_1506_03872_gb300 as mad
    s = 200_000
    c = Case("dense_ragged_f32", s_max=s)
    try:
        cand, nc = _candidates(c, s, 24, 3000)
        out = mad.new_pairs(50)
        mad.mad_rescore_noalloc(c.Am, c.Bm, cand, nc, 50, out=out)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        _, ng = mad.mad_rescore_noalloc(c.Am, c.Bm, cand, nc, 50, out=out)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert ng == 50
        assert free1 == free0
        assert torch.cuda.memory_reserved() == reserved0
    finally:
        c.close()
