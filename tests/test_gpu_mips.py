"""Batched queries on the GPU against the oracle run on each query alone
(A = the query as a 1 x d matrix, the same items, s_max, budget and seed +
q): the top-t' candidates (keys and x) and the final top t (keys and the
FP64 c) are bit-identical; a CUDA-graph replay reproduces the eager run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.workloads import batched_queries
    w = batched_queries(n=3000, d=40, nq=24, s_lo=1000, s_hi=20000, tprime=50, t=5, seed=14)
    s_q = w.meta["s_per_query"]
    s_max = 1 << 15
    tQ, tB = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.B).cuda()
    ctx = mad.Context()
    mad.mad_mips_items(ctx.ctx, mad.dense(tB), s_max)
    mad.mad_mips_plan(ctx.ctx, s_q, w.tprime, w.t)
    out = mad.new_pairs(w.m * w.t)
    nout = torch.zeros(w.m, dtype=torch.int32, device="cuda")
    cand = mad.new_pairs(w.m * w.tprime)
    mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout, cand)
    torch.cuda.synchronize()
    st = mad.mad_stats(ctx.ctx)
    yield w, s_q, s_max, ctx, (tQ, tB), out.cpu().numpy(), nout.cpu().numpy(), cand.cpu().numpy(), st
    ctx.close()


def _oracle_query(w, s_q, s_max, q):
    import oracle
    o = oracle.Oracle(oracle.Matrix(np.ascontiguousarray(w.A[q:q + 1])), oracle.Matrix(w.B), 0,
                      s_max)
    assert o.sample(int(s_q[q]), w.sampler_seed + q) == 0
    keys, x = o.topk(w.tprime)
    c = o.rescore(keys)
    tk, tc = oracle.topt(keys, c, w.t)
    return keys, x, tk, tc


def test_batch_matches_single_query_runs(batch):
    w, s_q, s_max, ctx, _, out, nout, cand, st = batch
    assert st["device_error"] == 0
    for q in range(w.m):
        keys, x, tk, tc = _oracle_query(w, s_q, s_max, q)
        K = len(keys)
        cj = (cand[q * w.tprime:q * w.tprime + K, 0] >> 32) & 0xFFFFFFFF
        ci = cand[q * w.tprime:q * w.tprime + K, 0] & 0xFFFFFFFF
        assert np.all(ci == q)
        assert np.array_equal(cj.astype(np.uint64), keys & np.uint64(0xFFFFFFFF)), q
        assert np.array_equal(cand[q * w.tprime:q * w.tprime + K, 1], x), q
        T = int(nout[q])
        assert T == len(tk)
        rows = out[q * w.t:q * w.t + T]
        assert np.array_equal(((rows[:, 0] >> 32) & 0xFFFFFFFF).astype(np.uint64),
                              tk & np.uint64(0xFFFFFFFF)), q
        assert np.array_equal(rows[:, 2].view(np.int64), tc.view(np.int64)), q


def test_graph_replay_reproduces_the_batch(batch):
    import paper_1506_03872_gb300 as mad
    w, s_q, s_max, ctx, (tQ, tB), out0, nout0, cand0, _ = batch
    out = mad.new_pairs(w.m * w.t)
    nout = torch.zeros(w.m, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):   # one eager run on the capture stream first
        mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout)
    out.zero_()
    nout.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), out0)
    assert np.array_equal(nout.cpu().numpy(), nout0)


def test_batch_limits(batch):
    import paper_1506_03872_gb300 as mad
    w, s_q, s_max, ctx, (tQ, tB), *_ = batch
    with mad.Context() as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_mips_plan(c.ctx, s_q, 10, 5)   # no items yet
        assert e.value.status == mad.MAD_ERR_STATE
        mad.mad_mips_items(c.ctx, mad.dense(tB), s_max)
        with pytest.raises(mad.MadError) as e:
            mad.mad_mips_plan(c.ctx, s_q, 2000, 5)   # t' above 1024
        assert e.value.status == mad.MAD_ERR_ARG
        with pytest.raises(mad.MadError) as e:
            mad.mad_mips_plan(c.ctx, np.array([s_max + 1], dtype=np.uint64), 10, 5)
        assert e.value.status == mad.MAD_ERR_ARG


@pytest.mark.parametrize("cfg", [dict(region_lg=2, chunk_mult=4, blocks_per_sm=2,
                                      select_threads=128),
                                 dict(region_lg=1, chunk_mult=2, blocks_per_sm=3,
                                      select_threads=512),
                                 dict(chunk_mult=8, select_threads=256)])
def test_launch_shapes_give_the_same_results(batch, cfg):
    """mad_mips_config changes the time only: every launch shape returns the
    default shape's candidates and results bit for bit."""
    import paper_1506_03872_gb300 as mad
    w, s_q, s_max, ctx, (tQ, tB), out0, nout0, cand0, _ = batch
    try:
        mad.mad_mips_config(ctx.ctx, **cfg)
        mad.mad_mips_plan(ctx.ctx, s_q, w.tprime, w.t)
        out = mad.new_pairs(w.m * w.t)
        nout = torch.zeros(w.m, dtype=torch.int32, device="cuda")
        cand = mad.new_pairs(w.m * w.tprime)
        mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout, cand)
        torch.cuda.synchronize()
        assert np.array_equal(nout.cpu().numpy(), nout0)
        assert np.array_equal(out.cpu().numpy(), out0)
        assert np.array_equal(cand.cpu().numpy(), cand0)
        assert mad.mad_stats(ctx.ctx)["device_error"] == 0
    finally:
        mad.mad_mips_config(ctx.ctx)
        mad.mad_mips_plan(ctx.ctx, s_q, w.tprime, w.t)


def test_autotuner_picks_a_shape_and_caches_it(batch, tmp_path, monkeypatch):
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300 import autotune
    w, s_q, s_max, ctx, (tQ, tB), out0, nout0, cand0, _ = batch
    monkeypatch.setenv("MAD_TUNE_CACHE", str(tmp_path / "tuned.json"))
    try:
        res = autotune.tune_mips(ctx.ctx, tQ, w.d, w.n, s_q, w.tprime, w.t, w.sampler_seed,
                                 reps=1)
        assert res["cached"] is False and res["ms"] <= res["default_ms"]
        assert set(res["best"]) == set(autotune.DEFAULT) and len(res["trials"]) >= 5
        out = mad.new_pairs(w.m * w.t)
        nout = torch.zeros(w.m, dtype=torch.int32, device="cuda")
        mad.mad_mips_run(ctx.ctx, mad.dense(tQ), w.sampler_seed, out, nout)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), out0)
        again = autotune.tune_mips(ctx.ctx, tQ, w.d, w.n, s_q, w.tprime, w.t, w.sampler_seed)
        assert again["cached"] is True and again["best"] == res["best"]
        with pytest.raises(mad.MadError):
            mad.mad_mips_config(ctx.ctx, chunk_mult=3)
    finally:
        mad.mad_mips_config(ctx.ctx)
        mad.mad_mips_plan(ctx.ctx, s_q, w.tprime, w.t)
