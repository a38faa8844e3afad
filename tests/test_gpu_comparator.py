"""The dense exact-computation comparator (Sec. 4.3) on the GPU.

The tensor-core product's summation order is not specified by the hardware,
so C~ is checked against the exact product of the BF16-rounded inputs within
the FP32 accumulation bound; the FP32 rescore and the final top-t are
checked against references computed here.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _bf16(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("m,d,n,dtype", [(300, 100, 700, np.float32), (129, 25, 257, np.float64),
                                         (1000, 64, 513, np.float32), (64, 128, 300, np.float32),
                                         (200, 65, 260, np.float32), (257, 300, 600, np.float32),
                                         (130, 640, 270, np.float64)])
def test_product_matches_bf16_reference(m, d, n, dtype):
    import paper_1506_03872_gb300 as mad
    rng = _rng(m + d + n)
    A = rng.standard_normal((m, d)).astype(dtype)
    B = rng.standard_normal((d, n)).astype(dtype)
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context() as c:
        C = mad.mad_debug_dense_product(c.ctx, mad.dense(tA), mad.dense(tB)).cpu().numpy()
    Ab, Bb = _bf16(A).astype(np.float64), _bf16(B).astype(np.float64)
    ref = Ab @ Bb
    bound = d * 2.0 ** -23 * (np.abs(Ab) @ np.abs(Bb)) + 1e-30
    assert np.all(np.abs(C - ref) <= bound)


def _fp32_rescore(A, B, keys):
    """Lane-strided FP32 sums folded in halves, as the library computes them."""
    out = []
    for key in keys:
        i, j = int(key) >> 32, int(key) & 0xFFFFFFFF
        a = A[i].astype(np.float32)
        b = B[:, j].astype(np.float32)
        part = np.zeros(32, dtype=np.float32)
        for k in range(len(a)):
            part[k % 32] = np.float32(np.float64(a[k]) * np.float64(b[k]) + np.float64(part[k % 32]))
        h = 16
        while h >= 1:
            part[:h] = part[:h] + part[h:2 * h]
            h //= 2
        out.append(float(part[0]))
    return np.array(out)


def test_planted_pairs_are_the_top_t():
    import oracle
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.workloads import plain_small
    w = plain_small(m=2000, d=25, n=1500, planted=10, seed=12)
    tA, tB = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.B).cuda()
    with mad.Context() as c:
        out, nt = mad.mad_dense_topt(c.ctx, mad.dense(tA), mad.dense(tB), 10)
    gi, gj, gx, gc = mad.decode_pairs(out, nt)
    o = oracle.Oracle(oracle.Matrix(w.A), oracle.Matrix(w.B))
    truth, tc = o.bruteforce(10)
    assert nt == 10
    assert np.array_equal(mad.keys_of(gi, gj), truth)
    # c is the FP32 dot product (fused multiply-add per lane, folded in halves)
    ref = _fp32_rescore(w.A, w.B, truth)
    assert np.allclose(gc, ref, rtol=0, atol=0) or np.all(np.abs(gc - tc) <= 25 * 2.0 ** -23 * np.abs(tc))


def _pattern_reference(A, B, t, rescore):
    """The comparator's precision pattern on the host: rank by the product of
    the BF16-rounded inputs (FP64 here), keep `rescore`, rank those by the
    exact product, return the top t keys."""
    n = B.shape[1]
    Ct = _bf16(A).astype(np.float64) @ _bf16(B).astype(np.float64)
    flat = np.abs(Ct).ravel()
    keep = np.argsort(-flat, kind="stable")[:rescore]
    C = A.astype(np.float64) @ B.astype(np.float64)
    exact = np.abs(C.ravel()[keep])
    top = keep[np.argsort(-exact, kind="stable")[:t]]
    return set(((top // n).astype(np.uint64) << np.uint64(32) | (top % n).astype(np.uint64)).tolist())


@pytest.mark.parametrize("rescore", [0, 2000])
def test_factor_matrices_follow_the_precision_pattern(rescore):
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.workloads import dense_factors
    w = dense_factors(m=20000, d=100, n=5000, seed=13)
    tA, tB = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.B).cuda()
    t = 100
    with mad.Context() as c:
        out, nt = mad.mad_dense_topt(c.ctx, mad.dense(tA), mad.dense(tB), t, rescore)
    gi, gj, gx, gc = mad.decode_pairs(out, nt)
    assert nt == t
    got = set(mad.keys_of(gi, gj).tolist())
    ref = _pattern_reference(w.A, w.B, t, rescore or 8 * t)
    # Only products within FP32 accumulation noise of the rescore boundary
    # may differ between the tensor-core and the host ordering.
    assert len(got & ref) >= 0.97 * t
    # every reported c is the exact product within FP32 rounding
    C = w.A.astype(np.float64) @ w.B.astype(np.float64)
    exact = C[gi.astype(np.int64), gj.astype(np.int64)]
    scale = (np.abs(w.A[gi.astype(np.int64)]).astype(np.float64) *
             np.abs(w.B[:, gj.astype(np.int64)].T).astype(np.float64)).sum(axis=1)
    assert np.all(np.abs(gc - exact) <= 100 * 2.0 ** -23 * scale)
    assert np.all(np.diff(np.abs(gc)) <= 0)   # sorted by |c| desc
    if rescore == 2000:
        flat = np.abs(C).ravel()
        top = np.argsort(-flat, kind="stable")[:t]
        truth = set(((top // w.n).astype(np.uint64) << np.uint64(32) |
                     (top % w.n).astype(np.uint64)).tolist())
        assert len(got & truth) / t >= 0.95   # a larger budget recovers the exact top t


@pytest.mark.parametrize("d,t,rescore", [(300, 100, 0), (100, 1000, 0), (40, 50, 20000)])
def test_wide_and_large_budgets_follow_the_precision_pattern(d, t, rescore):
    """K split into several 64-wide slices (d = 300), and rescore budgets
    past the old 2048 (8t = 8000, 20000) that make the per-CTA buffers
    compact many times."""
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.workloads import dense_factors
    w = dense_factors(m=6000, d=d, n=3000, seed=14 + d)
    tA, tB = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.B).cuda()
    with mad.Context() as c:
        out, nt = mad.mad_dense_topt(c.ctx, mad.dense(tA), mad.dense(tB), t, rescore)
    gi, gj, gx, gc = mad.decode_pairs(out, nt)
    assert nt == t
    got = set(mad.keys_of(gi, gj).tolist())
    ref = _pattern_reference(w.A, w.B, t, rescore or 8 * t)
    assert len(got & ref) >= 0.97 * t
    C = w.A.astype(np.float64) @ w.B.astype(np.float64)
    exact = C[gi.astype(np.int64), gj.astype(np.int64)]
    scale = (np.abs(w.A[gi.astype(np.int64)]).astype(np.float64) *
             np.abs(w.B[:, gj.astype(np.int64)].T).astype(np.float64)).sum(axis=1)
    assert np.all(np.abs(gc - exact) <= 100 * 2.0 ** -23 * scale)
    assert np.all(np.diff(np.abs(gc)) <= 0)
    assert len(set(zip(gi.tolist(), gj.tolist()))) == t   # no pair twice


def test_limits():
    import paper_1506_03872_gb300 as mad
    rng = _rng(3)
    A = torch.from_numpy(rng.standard_normal((100, 641)).astype(np.float32)).cuda()
    B = torch.from_numpy(rng.standard_normal((641, 100)).astype(np.float32)).cuda()
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_dense_topt(c.ctx, mad.dense(A), mad.dense(B), 10)   # d > 640
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
        A2 = A[:, :100].contiguous()
        B2 = B[:100].contiguous()
        with pytest.raises(mad.MadError) as e:
            mad.mad_dense_topt(c.ctx, mad.dense(A2), mad.dense(B2), 8193)  # 8t > 65536
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
        with pytest.raises(mad.MadError) as e:
            mad.mad_dense_topt(c.ctx, mad.dense(A2), mad.dense(B2), 10, 65537)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
        with pytest.raises(mad.MadError) as e:
            mad.mad_dense_topt(c.ctx, mad.dense(A2), mad.dense(B2), 10, 5)  # budget < t
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
