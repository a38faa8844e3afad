"""Alias-table draws (MAD_ALIAS; Sec. 4.1) on the GPU, through the C ABI,
against the oracle's alias sampler: every alias table (entries, segment and
row totals), every draw (i, k, j, k', v), X after s diamonds, and Omega_t'
and Omega_t, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402

ALIAS = 32


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _case(name):
    """(A, B, flags) of an alias case."""
    rng = _rng({"two_level": 81, "factors_f32": 82, "f64_nonneg": 83, "gram_excl": 84}[name])
    if name == "two_level":
        # T1 over 1500 rows and TB rows of 2500 entries: two levels; exact
        # zeros in A and a zero column of B.
        A = rng.standard_normal((1500, 7)) * np.exp(0.7 * rng.standard_normal((1500, 1)))
        B = rng.standard_normal((7, 2500)) * np.exp(0.7 * rng.standard_normal((1, 2500)))
        A[rng.random(A.shape) < 0.03] = 0.0
        B[:, 5] = 0.0
        return A.astype(np.float32), B.astype(np.float32), 0
    if name == "factors_f32":
        from paper_1506_03872_gb300.workloads import dense_factors
        w = dense_factors(m=4000, d=100, n=1500, seed=85)
        return w.A, w.B, 0
    if name == "f64_nonneg":
        A = np.abs(rng.standard_normal((300, 20)))
        B = np.abs(rng.standard_normal((20, 1100)))
        return A, B, 1
    if name == "gram_excl":
        A = rng.standard_normal((1200, 30)).astype(np.float32)
        return A, np.ascontiguousarray(A.T), 2 | 4
    raise KeyError(name)


class AliasCase:
    def __init__(self, name, s_max):
        import paper_1506_03872_gb300 as mad
        A, B, flags = _case(name)
        self.A, self.B = A, B
        self.flags = flags | ALIAS
        self.ctx = mad.Context(self.flags)
        self.t = [torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()]
        self.ctx.build(mad.dense(self.t[0]), mad.dense(self.t[1]), s_max, keep=tuple(self.t))
        self.oracle = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), self.flags, s_max)

    def close(self):
        self.ctx.close()


CASES = ["two_level", "factors_f32", "f64_nonneg", "gram_excl"]


@pytest.mark.parametrize("name", CASES)
def test_alias_tables_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    c = AliasCase(name, 1 << 20)
    try:
        for fam in ("T1", "T2", "TA", "TB"):
            ent, segX, rowX = c.oracle.alias_table(fam)
            g = mad.mad_export_table(c.ctx.ctx, fam + "al").cpu().numpy().view(np.uint64)
            g = g.reshape(-1, 2)
            assert len(g) == len(ent), fam
            assert np.array_equal(g[:, 0], ent["t"]), fam
            assert np.array_equal((g[:, 1] & np.uint64(0xFFFFFFFF)).astype(np.uint32), ent["a"]), fam
            gs = mad.mad_export_table(c.ctx.ctx, fam + "as").cpu().numpy().view(np.uint64)
            gr = mad.mad_export_table(c.ctx.ctx, fam + "ar").cpu().numpy().view(np.uint64)
            assert np.array_equal(gs, segX) and np.array_equal(gr, rowX), fam
    finally:
        c.close()


@pytest.mark.parametrize("name", CASES)
def test_alias_draws_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    c = AliasCase(name, 1 << 20)
    try:
        first, count = (1 << 33) + 5, 40_000
        gi, gk, gj, gkp, gv = [x.cpu().numpy() for x in
                               mad.mad_debug_draws(c.ctx.ctx, 91, first, count)]
        oi, ok, oj, okp, ov = c.oracle.draw(seed=91, first=first, count=count)
        assert np.array_equal(gi, oi) and np.array_equal(gk, ok)
        assert np.array_equal(gj, oj) and np.array_equal(gkp, okp)
        assert np.array_equal(gv, ov)
        assert mad.mad_stats(c.ctx.ctx)["device_error"] == 0
    finally:
        c.close()


@pytest.mark.parametrize("name", ["two_level", "factors_f32", "gram_excl"])
def test_alias_x_and_top_t_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    s, seed, tprime, t = 300_000, 23, 1500, 30
    c = AliasCase(name, s)
    try:
        mad.mad_sample(c.ctx.ctx, s, seed)
        keys, vals, n = mad.mad_export_x(c.ctx.ctx, cap=s + 1)
        k = keys[:n].cpu().numpy().view(np.uint64)
        v = vals[:n].cpu().numpy()
        order = np.argsort(k)
        assert c.oracle.sample(s, seed) == 0
        ok_, ov_ = c.oracle.x()
        oo = np.argsort(ok_)
        assert np.array_equal(k[order], ok_[oo]) and np.array_equal(v[order], ov_[oo])
        st = mad.mad_stats(c.ctx.ctx)
        sc = c.oracle.scalars()
        assert st["inserted"] == sc["inserted"] and st["diag_skipped"] == sc["diag_skipped"]
        cand, nc = mad.mad_topk(c.ctx.ctx, tprime)
        res, nr = mad.mad_rescore(c.ctx.ctx, cand, nc, t)
        c.oracle.reset()
        rk, rc = c.oracle.run(s, seed, tprime, t)
        gi, gj, _, gc = mad.decode_pairs(res, nr)
        assert np.array_equal(mad.keys_of(gi, gj), rk)
        assert np.array_equal(gc.view(np.int64), rc.view(np.int64))
    finally:
        c.close()


def test_alias_refusals():
    """MAD_ALIAS with wedges, 0/1 inputs and the fused pass is refused."""
    import paper_1506_03872_gb300 as mad
    with pytest.raises(mad.MadError) as e:
        mad.mad_create(ALIAS | 16)
    assert e.value.status == mad.MAD_ERR_ARG
    rng = _rng(86)
    Ab = (rng.random((50, 30)) < 0.2)
    Ab[:, 0] = True
    rp = np.concatenate([[0], np.cumsum(Ab.sum(1))]).astype(np.int64)
    ta = [torch.from_numpy(rp).cuda(), torch.from_numpy(np.nonzero(Ab)[1].astype(np.int32)).cuda()]
    At = np.ascontiguousarray(Ab.T)
    rpt = np.concatenate([[0], np.cumsum(At.sum(1))]).astype(np.int64)
    tb = [torch.from_numpy(rpt).cuda(), torch.from_numpy(np.nonzero(At)[1].astype(np.int32)).cuda()]
    with mad.Context(ALIAS) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.csr(ta[0], ta[1], Ab.shape),
                                 mad.csr(tb[0], tb[1], At.shape), 1000)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
    Ad = torch.randn(100, 8, device="cuda")
    Bd = torch.randn(8, 90, device="cuda")
    with mad.Context(ALIAS) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, mad.dense(Ad), mad.dense(Bd), 10_000, 100, 10)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
