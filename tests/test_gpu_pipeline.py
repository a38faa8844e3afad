"""The fused dense pass (mad_pipeline_*) against the CPU oracle: Omega_t'
(keys and x, as a set) and Omega_t (keys, x and the FP64 c, in order) bit
for bit; a CUDA-graph
replay on new contents of the same input buffers matches the oracle on the
new inputs; device-side lengths cover short and multi-tile candidate
lists."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _inputs(seed, m=2051, d=100, n=3001):
    """Log-normal row and column scales times Gaussian directions (several
    tiles and ragged tails in every table)."""
    rng = _rng(seed)
    A = rng.standard_normal((m, d)) * np.exp(0.5 * rng.standard_normal((m, 1)))
    B = rng.standard_normal((d, n)) * np.exp(0.5 * rng.standard_normal((1, n)))
    return A.astype(np.float32), B.astype(np.float32)


def _oracle_pass(A, B, flags, s, seed, tprime, t):
    o = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), flags, s)
    assert o.sample(s, seed) == 0
    keys, x = o.topk(tprime)
    c = o.rescore(keys)
    tk, tc = oracle.topt(keys, c, t)
    return keys, x, tk, tc


def _check(mad, out, counts, cand, ref):
    keys, x, tk, tc = ref
    nc, nr = [int(v) for v in counts.cpu().numpy()]
    assert nc == len(keys)
    ci, cj, cx, _ = mad.decode_pairs(cand, nc)
    # Omega_t' as a set (the fused pass need not order it)
    gk = mad.keys_of(ci, cj)
    go, oo = np.argsort(gk), np.argsort(keys)
    assert np.array_equal(gk[go], keys[oo])
    assert np.array_equal(cx[go], x[oo])
    assert nr == len(tk)
    ri, rj, rx, rc = mad.decode_pairs(out, nr)
    assert np.array_equal(mad.keys_of(ri, rj), tk)
    assert np.array_equal(rc.view(np.int64), tc.view(np.int64))
    xmap = dict(zip(keys.tolist(), x.tolist()))
    assert [xmap[k] for k in tk.tolist()] == rx.tolist()


@pytest.mark.parametrize("flags,tprime,t", [(0, 1000, 37), (0, 5000, 100), (1, 300, 10)])
def test_pass_matches_oracle(flags, tprime, t):
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(60 + flags)
    if flags & 1:
        A, B = np.abs(A), np.abs(B)
    s, seed = 300_000, 11
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context(flags) as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out = mad.new_pairs(t)
        cand = mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        st = mad.mad_stats(c.ctx)
        _check(mad, out, counts, cand, _oracle_pass(A, B, flags, s, seed, tprime, t))
        o = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), flags, s)
        sc = o.scalars()
        assert st["t1_total"] == sc["T1_total"] and st["f"] == sc["F"] and st["e1"] == sc["E1"]
        assert st["sampled"] == s


def test_ties_and_long_lists():
    """Inputs with few distinct values (many equal x and equal c: the key
    breaks the ties in both selections), a candidate list longer than one
    block selects (t' = 20000), and a final top t longer than one block
    sorts (t = 3000)."""
    import paper_1506_03872_gb300 as mad
    rng = _rng(66)
    A = rng.integers(-2, 3, (1500, 12)).astype(np.float32)
    B = rng.integers(-2, 3, (12, 2500)).astype(np.float32)
    for s, tprime, t in ((200_000, 3000, 200), (60_000, 20_000, 3000)):
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        with mad.Context() as c:
            mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
            out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
            counts = torch.zeros(2, dtype=torch.int32, device="cuda")
            mad.mad_pipeline_run(c.ctx, 17, out, counts, cand)
            mad.mad_pipeline_status(c.ctx)
            _check(mad, out, counts, cand, _oracle_pass(A, B, 0, s, 17, tprime, t))


def test_gram_pass_matches_oracle():
    import paper_1506_03872_gb300 as mad
    rng = _rng(65)
    A = rng.standard_normal((700, 30)).astype(np.float32)
    B = np.ascontiguousarray(A.T)
    flags, s, seed, tprime, t = 2 | 4, 200_000, 3, 800, 25
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context(flags) as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        _check(mad, out, counts, cand, _oracle_pass(A, B, flags, s, seed, tprime, t))


def test_square_sym_pass_matches_oracle():
    """The fused pass with the squared symmetric update (Sec. 3.2.3) on a
    dense symmetric matrix: two records per diamond reach X."""
    import paper_1506_03872_gb300 as mad
    rng = _rng(66)
    S = rng.standard_normal((500, 500))
    S = (S + S.T).astype(np.float32)
    S[np.abs(S) < 0.4] = 0.0
    flags, s, seed, tprime, t = 2 | 4 | 8, 150_000, 4, 900, 30
    tA, tB = torch.from_numpy(S).cuda(), torch.from_numpy(S.copy()).cuda()
    with mad.Context(flags) as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        _check(mad, out, counts, cand, _oracle_pass(S, S.copy(), flags, s, seed, tprime, t))


def test_graph_replay_on_new_inputs():
    """Captured once, replayed after the inputs' contents change: nothing of
    the first inputs may survive in host-side state."""
    import paper_1506_03872_gb300 as mad
    A0, B0 = _inputs(70)
    A1, B1 = _inputs(71)
    s, seed, tprime, t = 250_000, 21, 2000, 50
    tA, tB = torch.from_numpy(A0).cuda(), torch.from_numpy(B0).cuda()
    with mad.Context() as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):   # one eager run on the capture stream first
            mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        for A, B in ((A1, B1), (A0, B0)):
            tA.copy_(torch.from_numpy(A))
            tB.copy_(torch.from_numpy(B))
            out.zero_()
            cand.zero_()
            counts.zero_()
            g.replay()
            torch.cuda.synchronize()
            mad.mad_pipeline_status(c.ctx)
            _check(mad, out, counts, cand, _oracle_pass(A, B, 0, s, seed, tprime, t))


def test_short_lists_and_limits():
    """Fewer positive x than t' (a tiny budget), and argument checks."""
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(72, m=300, d=20, n=400)
    s, seed, tprime, t = 50, 9, 1000, 30
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_run(c.ctx, seed, mad.new_pairs(t),
                                 torch.zeros(2, dtype=torch.int32, device="cuda"))
        assert e.value.status == mad.MAD_ERR_STATE
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, 10, 11)   # t > t'
        assert e.value.status == mad.MAD_ERR_ARG
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, 1 << 18, 10)
        assert e.value.status == mad.MAD_ERR_ARG
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        ref = _oracle_pass(A, B, 0, s, seed, tprime, t)
        assert len(ref[0]) < tprime
        _check(mad, out, counts, cand, ref)
    # Mixed formats and wedge contexts are refused (0/1 CSR on both sides is
    # planned: see the CSR tests below).
    rp = torch.tensor([0, 1, 2], dtype=torch.int64, device="cuda")
    ci = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    M = mad.csr(rp, ci, (2, 2))
    Dm = torch.ones(2, 2, device="cuda")
    with mad.Context(2) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, M, mad.dense(Dm), 100, 10, 5)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
    with mad.Context(2 | 16) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, M, M, 100, 10, 5)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED


def _oracle_x(A, B, flags, s, seed):
    o = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), flags, s)
    assert o.sample(s, seed) == 0
    return o.x(), o.scalars()


def _export_sorted(mad, ctx, cap):
    keys, vals, n = mad.mad_export_x(ctx, cap=cap)
    keys = keys.cpu().numpy().view(np.uint64)
    vals = vals.cpu().numpy()
    order = np.argsort(keys)
    return keys[order], vals[order], n


@pytest.mark.parametrize("variant", ["plain", "heavy_rows", "zero_rows", "nonneg", "wide_columns"])
def test_pass_x_matches_oracle(variant):
    """X after the fused pass, every key and sum, against the oracle: the
    pass builds the home regions whole (and an overflow table), so this
    covers rows owned by one group of buckets, rows whose diamonds run into
    later groups, groups too large for the shared-memory image (rows with
    thousands of expected diamonds), rows that are never drawn, and keys
    that spill past their group's regions."""
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(80)
    flags = 0
    if variant == "wide_columns":
        # More than 2^24 columns: the builder keeps 64-bit keys in its image.
        A, B = _inputs(81, m=600, d=3, n=(1 << 24) + 4099)
    if variant == "heavy_rows":
        A[[5, 900, 901, 2050]] *= 8.0
    elif variant == "zero_rows":
        A[[0, 1, 2, 700, 701, 2049, 2050]] = 0.0
    elif variant == "nonneg":
        A, B, flags = np.abs(A), np.abs(B), 1
    s, seed, tprime, t = 300_000, 23, 2000, 40
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    (ok, ov), sc = _oracle_x(A, B, flags, s, seed)
    with mad.Context(flags) as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        keys, vals, n = _export_sorted(mad, c.ctx, s + 1)
        assert n == len(ok)
        assert np.array_equal(keys, ok)
        assert np.array_equal(vals, ov)
        st = mad.mad_stats(c.ctx)
        assert st["inserted"] == sc["inserted"]
        assert st["distinct"] == len(ok)
        _check(mad, out, counts, cand, _oracle_pass(A, B, flags, s, seed, tprime, t))


def test_stepwise_after_pass_starts_empty():
    """mad_reset_hash after a fused pass empties the regions and the
    overflow table; the step-wise sampler then builds the oracle's X."""
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(81)
    A[[3, 4]] *= 8.0
    s, tprime, t = 200_000, 1000, 20
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context() as c:
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, 31, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        mad.mad_reset_hash(c.ctx)
        mad.mad_sample(c.ctx, s, 32)
        keys, vals, n = _export_sorted(mad, c.ctx, s + 1)
        (ok, ov), _ = _oracle_x(A, B, 0, s, 32)
        assert n == len(ok)
        assert np.array_equal(keys, ok)
        assert np.array_equal(vals, ov)


def test_pass_overflow_table():
    """Home regions sized for half the expected diamonds: most groups of
    regions fill up and their further keys go to the overflow table, whose
    contents must complete X exactly."""
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(82)
    s, seed, tprime, t = 200_000, 41, 1500, 30
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    (ok, ov), sc = _oracle_x(A, B, 0, s, seed)
    with mad.Context() as c:
        mad.mad_debug_set_hash_layout(c.ctx, 0.5, 1 << 19)
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        mad.mad_pipeline_status(c.ctx)
        st = mad.mad_stats(c.ctx)
        assert st["hash_capacity"] < len(ok)   # the regions alone cannot hold X
        keys, vals, n = _export_sorted(mad, c.ctx, s + 1)
        assert n == len(ok)
        assert np.array_equal(keys, ok)
        assert np.array_equal(vals, ov)
        assert st["inserted"] == sc["inserted"]
        _check(mad, out, counts, cand, _oracle_pass(A, B, 0, s, seed, tprime, t))


def test_pass_overflow_full_is_reported():
    """Regions and overflow table both too small: the pass reports
    MAD_ERR_HASH_FULL instead of returning a partial X silently."""
    import paper_1506_03872_gb300 as mad
    A, B = _inputs(83)
    s, tprime, t = 200_000, 1000, 20
    tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_debug_set_hash_layout(c.ctx, 2.0, 0)
        assert e.value.status == mad.MAD_ERR_ARG
        mad.mad_debug_set_hash_layout(c.ctx, 0.5, 1024)
        mad.mad_pipeline_plan(c.ctx, mad.dense(tA), mad.dense(tB), s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        mad.mad_pipeline_run(c.ctx, 43, out, counts, cand)
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_status(c.ctx)
        assert e.value.status == mad.MAD_ERR_HASH_FULL


# ---------------------------------------------------------------------------
# 0/1 CSR inputs: the fused pass planned once (the step-wise build sizes the
# guides, the closure filter and the hash), run eagerly and from a graph.
# ---------------------------------------------------------------------------
def _csr_case(name):
    """(rowptr_a, col_a, shape_a, rowptr_b, col_b, shape_b, flags, oracle matrices)."""
    if name in ("chung_lu", "chung_lu_square_sym", "chung_lu_ties"):
        from paper_1506_03872_gb300.workloads import chung_lu
        w = (chung_lu(nodes=20_000, edges=200_000, seed=16) if name == "chung_lu_ties"
             else chung_lu(nodes=6000, edges=60_000, seed=14))
        M = oracle.Matrix(rowptr=w.rowptr, colidx=w.colidx, shape=(w.m, w.m))
        flags = w.flags | (8 if name == "chung_lu_square_sym" else 0)
        return (w.rowptr, w.colidx, (w.m, w.m), w.rowptr, w.colidx, (w.m, w.m), flags, M, M)
    rng = _rng(15)
    A = rng.random((900, 300)) < np.linspace(0.002, 0.08, 300)[None, :]
    B = rng.random((300, 1100)) < 0.03
    A[:, 0] = B[0, :] = True

    def csr(D):
        rp = np.concatenate([[0], np.cumsum(D.sum(1))]).astype(np.int64)
        return rp, np.nonzero(D)[1].astype(np.int32)
    ra, ca = csr(A)
    rb, cb = csr(B)
    MA = oracle.Matrix(rowptr=ra, colidx=ca, shape=A.shape)
    MB = oracle.Matrix(rowptr=rb, colidx=cb, shape=B.shape)
    return (ra, ca, A.shape, rb, cb, B.shape, 0, MA, MB)


@pytest.mark.parametrize("name", ["chung_lu", "bipartite", "chung_lu_square_sym", "chung_lu_ties"])
def test_csr_pass_matches_oracle_eager_and_from_a_graph(name):
    """Omega_t' of a 0/1 pass comes from a radix selection over every key at
    or above the t'-th count (counts tie in large numbers there); the last
    case has t' = 20000 with more candidates than the dense pass's list."""
    import paper_1506_03872_gb300 as mad
    ra, ca, sa, rb, cb, sb, flags, MA, MB = _csr_case(name)
    s, seed, tprime, t = 400_000, 7, 2000, 50
    if name == "chung_lu_ties":
        s, tprime, t = 3_000_000, 20_000, 100
    keep = [torch.from_numpy(x).cuda() for x in (ra, ca, rb, cb)]
    Am = mad.csr(keep[0], keep[1], sa)
    Bm = mad.csr(keep[2], keep[3], sb)
    o = oracle.Oracle(MA, MB, flags, s)
    assert o.sample(s, seed) == 0
    keys, x = o.topk(tprime)
    tk, tc = oracle.topt(keys, o.rescore(keys), t)
    ref = (keys, x, tk, tc)
    with mad.Context(flags) as c:
        mad.mad_pipeline_plan(c.ctx, Am, Bm, s, tprime, t)
        out, cand = mad.new_pairs(t), mad.new_pairs(tprime)
        counts = torch.zeros(2, dtype=torch.int32, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):   # eager on the capture stream
            mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        mad.mad_pipeline_status(c.ctx)
        _check(mad, out, counts, cand, ref)
        # The same pass captured once and replayed (with another seed first,
        # so nothing of the eager run survives into the replay's result).
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            mad.mad_pipeline_run(c.ctx, seed, out, counts, cand)
        out.zero_()
        cand.zero_()
        counts.zero_()
        g.replay()
        torch.cuda.synchronize()
        mad.mad_pipeline_status(c.ctx)
        _check(mad, out, counts, cand, ref)
        # Step-wise X after the pass: the pass's X is the step-wise one.
        st = mad.mad_stats(c.ctx)
        sc = o.scalars()
        assert st["inserted"] == sc["inserted"] and st["diag_skipped"] == sc["diag_skipped"]
