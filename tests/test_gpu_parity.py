"""GPU parity: every step of the library against the CPU oracle on the same
seeded inputs, through the C ABI.

Integer and index results are compared bit for bit (tables, draws, x_ij,
Omega_t', Omega_t); FP64 dot products are compared bit for bit as well,
since both sides use the same fixed summation order (the benchmark spec's bound
of 1e-12 relative is checked on top).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from gpu_cases import Case  # noqa: E402

CASES = ["plain_small", "dense_ragged_f32", "dense_wide_rows", "dense_deep", "dense_factors_small",
         "dense_mixed_signs_zeros",
         "dense_nonneg", "gram_dense", "dense_square_sym", "chung_lu_small", "bipartite_binary", "chung_lu_square_sym"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mad():
    import paper_1506_03872_gb300 as mad
    return mad


@pytest.mark.parametrize("name", CASES)
def test_tables_bit_exact(name):
    _tables_match(name)


@pytest.mark.parametrize("d", [1, 7, 33, 97, 130, 200, 229, 256])
def test_tables_short_rows(d):
    """Every chunk count of the register-row kernel of A (d <= 256), with
    rows whose length is and is not a multiple of four."""
    _tables_match(f"dense_short_d{d}")


def _tables_match(name):
    mad = _mad()
    c = Case(name, s_max=1 << 20)
    try:
        g = {k: mad.mad_export_table(c.ctx.ctx, k).cpu().numpy() for k in mad.TABLES}
        o = c.oracle
        assert np.array_equal(g["T1"].view(np.uint64), o.table("T1"))
        T2 = g["T2"].view(np.uint32)
        integer = c.oracle.scalars()["F"] == 0 and hasattr(c, "csr")
        mask = np.uint32(0xFFFFFFFF) if integer else np.uint32(0x7FFFFFFF)
        assert np.array_equal(T2 & mask, o.table("T2"))
        if not integer:
            TA = g["TA"].view(np.uint32)
            TB = g["TB"].view(np.uint32)
            assert np.array_equal(TA & mask, o.table("TA"))
            assert np.array_equal(TB & mask, o.table("TB"))
            sa = (c.A.astype(np.float32) < 0).ravel()
            sb = (c.B.astype(np.float32) < 0).ravel()
            assert np.array_equal((T2 >> np.uint32(31)).astype(bool), sa)
            assert np.array_equal((TA >> np.uint32(31)).astype(bool), sa)
            assert np.array_equal((TB >> np.uint32(31)).astype(bool), sb)
            for k in ("na", "nb", "r"):
                assert np.array_equal(g[k].view(np.uint32), o.table(k).view(np.uint32)), k
        st = mad.mad_stats(c.ctx.ctx)
        sc = o.scalars()
        assert st["t1_total"] == sc["T1_total"]
        assert st["f"] == sc["F"]
        if not integer:
            assert st["e1"] == sc["E1"]
    finally:
        c.close()


@pytest.mark.parametrize("name", CASES)
def test_draws_bit_exact(name):
    mad = _mad()
    c = Case(name, s_max=1 << 20)
    try:
        seed, first, count = 0x9E3779B97F4A7C15, (1 << 33) + 12345, 40_000
        gi, gk, gj, gkp, gv = [x.cpu().numpy() for x in mad.mad_debug_draws(c.ctx.ctx, seed, first, count)]
        oi, ok, oj, okp, ov = c.oracle.draw(seed, first, count)
        for a, b, nm in ((gi, oi, "i"), (gk, ok, "k"), (gj, oj, "j"), (gkp, okp, "k'")):
            assert np.array_equal(a.view(np.uint32), b), nm
        assert np.array_equal(gv, ov), "increment"
    finally:
        c.close()


@pytest.mark.parametrize("name", CASES)
def test_x_bit_exact(name):
    mad = _mad()
    s, seed = 300_000, 77
    c = Case(name, s_max=s)
    try:
        mad.mad_sample(c.ctx.ctx, s, seed)
        keys, vals, n = mad.mad_export_x(c.ctx.ctx, cap=s + 1)
        keys = keys.cpu().numpy().view(np.uint64)
        vals = vals.cpu().numpy()
        order = np.argsort(keys)
        assert c.oracle.sample(s, seed) == 0
        ok, ov = c.oracle.x()
        assert n == len(ok)
        assert np.array_equal(keys[order], ok)
        assert np.array_equal(vals[order], ov)
        st = mad.mad_stats(c.ctx.ctx)
        sc = c.oracle.scalars()
        assert st["inserted"] == sc["inserted"]
        assert st["diag_skipped"] == sc["diag_skipped"]
        assert st["distinct"] == len(ok)
    finally:
        c.close()


@pytest.mark.parametrize("name", CASES)
def test_pipeline_bit_exact(name):
    """Alg. 2 then Alg. 3: Omega_t' and Omega_t with their values."""
    mad = _mad()
    s, seed, tprime, t = 200_000, 5, 1000, 37
    c = Case(name, s_max=s)
    try:
        mad.mad_sample(c.ctx.ctx, s, seed)
        cand, nc = mad.mad_topk(c.ctx.ctx, tprime)
        ci, cj, cx, _ = mad.decode_pairs(cand, nc)
        c.oracle.sample(s, seed)
        okeys, ox = c.oracle.topk(tprime)
        assert nc == len(okeys)
        assert np.array_equal(mad.keys_of(ci, cj), okeys)
        assert np.array_equal(cx, ox)
        res, nr = mad.mad_rescore(c.ctx.ctx, cand, nc, t)
        ri, rj, rx, rc = mad.decode_pairs(res, nr)
        oc = c.oracle.rescore(okeys)
        tk, tc = __import__("oracle").topt(okeys, oc, t)
        assert nr == len(tk)
        assert np.array_equal(mad.keys_of(ri, rj), tk)
        assert np.array_equal(rc.view(np.int64), tc.view(np.int64))
        # x carried through rescoring
        xmap = dict(zip(okeys.tolist(), ox.tolist()))
        assert [xmap[k] for k in tk.tolist()] == rx.tolist()
    finally:
        c.close()


@pytest.mark.parametrize("name", ["plain_small", "chung_lu_small"])
def test_split_ranges_equal_one_call(name):
    mad = _mad()
    s, seed = 100_000, 3
    a = Case(name, s_max=s)
    b = Case(name, s_max=s)
    try:
        mad.mad_sample(a.ctx.ctx, s, seed, 0)
        for lo, hi in ((0, 1), (1, 40_000), (40_000, 40_017), (40_017, s)):
            mad.mad_sample(b.ctx.ctx, hi - lo, seed, lo)
        ka, va, _ = mad.mad_export_x(a.ctx.ctx, s + 1)
        kb, vb, _ = mad.mad_export_x(b.ctx.ctx, s + 1)
        ka, va, kb, vb = [x.cpu().numpy() for x in (ka, va, kb, vb)]
        oa, ob = np.argsort(ka), np.argsort(kb)
        assert np.array_equal(ka[oa], kb[ob]) and np.array_equal(va[oa], vb[ob])
    finally:
        a.close()
        b.close()


def test_rescore_within_1e12_of_long_double():
    mad = _mad()
    c = Case("plain_small", s_max=1 << 16)
    try:
        rng = np.random.Generator(np.random.PCG64(5))
        i = rng.integers(0, c.m, 5000)
        j = rng.integers(0, c.n, 5000)
        keys = np.unique(mad.keys_of(i, j))
        i, j = (keys >> np.uint64(32)).astype(np.uint32), (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)
        cand = mad.encode_pairs(i, j)
        res, nr = mad.mad_rescore(c.ctx.ctx, cand, len(keys), len(keys))
        ri, rj, _, rc = mad.decode_pairs(res, nr)
        Al = c.A.astype(np.longdouble)
        Bl = c.B.astype(np.longdouble)
        ref = (Al[ri] * Bl[:, rj].T).sum(axis=1)
        scale = (np.abs(Al[ri]) * np.abs(Bl[:, rj].T)).sum(axis=1)
        assert np.all(np.abs(rc - ref) <= 1e-12 * np.maximum(np.abs(ref), 1e-3 * scale))
    finally:
        c.close()


def test_empty_and_degenerate_requests():
    mad = _mad()
    c = Case("plain_small", s_max=1000)
    try:
        cand, nc = mad.mad_topk(c.ctx.ctx, 10)          # nothing sampled yet
        assert nc == 0
        mad.mad_sample(c.ctx.ctx, 0, 1)                 # empty range
        mad.mad_sample(c.ctx.ctx, 1, 1)                 # a single diamond
        cand, nc = mad.mad_topk(c.ctx.ctx, 0)
        assert nc == 0
        cand, nc = mad.mad_topk(c.ctx.ctx, 5)
        assert nc <= 1
        res, nr = mad.mad_rescore(c.ctx.ctx, cand, nc, 0)
        assert nr == 0
    finally:
        c.close()


def test_reset_over_earlier_keys():
    """A 4096-row instance with a hash of a few million slots: after a
    reset over the keys of an earlier run, X equals the oracle's for the new
    seed."""
    import oracle
    mad = _mad()
    rng = np.random.Generator(np.random.PCG64(49))
    A = (rng.standard_normal((4096, 16)) * np.exp(0.5 * rng.standard_normal((4096, 1))))
    B = rng.standard_normal((16, 2000))
    A, B = A.astype(np.float32), B.astype(np.float32)
    s = 1_000_000
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context() as c:
        mad.mad_build_tables(c.ctx, mad.dense(tA), mad.dense(tB), s)
        assert mad.mad_stats(c.ctx)["hash_capacity"] * 16 > (24 << 20)
        mad.mad_sample(c.ctx, s, 5)
        mad.mad_reset_hash(c.ctx)
        mad.mad_sample(c.ctx, s, 6)
        keys, vals, n = mad.mad_export_x(c.ctx, cap=s + 1)
        st = mad.mad_stats(c.ctx)
    keys = keys.cpu().numpy().view(np.uint64)
    vals = vals.cpu().numpy()
    order = np.argsort(keys)
    o = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), 0, s)
    assert o.sample(s, 6) == 0
    ok, ov = o.x()
    assert st["device_error"] == 0
    assert n == len(ok)
    assert np.array_equal(keys[order], ok)
    assert np.array_equal(vals[order], ov)
