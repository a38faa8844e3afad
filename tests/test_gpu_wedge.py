"""Wedge sampling (MAD_WEDGE contexts; the paper's comparison method) on the
GPU, through the C ABI, against the oracle's wedge sampler: the centre and
column tables, every draw (i, k, j, v), the whole X after s wedges and
Omega_t' / Omega_t, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import oracle  # noqa: E402

WEDGE = 16


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _case(name):
    """(kind, payload, flags) of a wedge case."""
    rng = _rng({"dense_ragged_f32": 61, "dense_f64_nonneg": 62, "dense_gram": 63,
                "chung_lu_gram": 64}[name])
    if name == "dense_ragged_f32":
        A = rng.standard_normal((1031, 37)) * np.exp(0.5 * rng.standard_normal((1031, 1)))
        B = rng.standard_normal((37, 2049)) * np.exp(0.5 * rng.standard_normal((1, 2049)))
        A[rng.random(A.shape) < 0.05] = 0.0
        A[:, 5] = 0.0
        return "dense", (A.astype(np.float32), B.astype(np.float32)), 0
    if name == "dense_f64_nonneg":
        A = np.abs(rng.standard_normal((300, 20)))
        B = np.abs(rng.standard_normal((20, 500)))
        return "dense", (A, B), 1
    if name == "dense_gram":
        A = rng.standard_normal((400, 30)).astype(np.float32)
        return "dense", (A, np.ascontiguousarray(A.T)), 2 | 4
    if name == "chung_lu_gram":
        from paper_1506_03872_gb300.workloads import chung_lu
        w = chung_lu(nodes=6000, edges=50_000, seed=12)
        return "csr", (w.rowptr, w.colidx, w.m), w.flags
    raise KeyError(name)


class WedgeCase:
    def __init__(self, name, s_max):
        import paper_1506_03872_gb300 as mad
        kind, payload, flags = _case(name)
        self.flags = flags | WEDGE
        self.ctx = mad.Context(self.flags)
        if kind == "dense":
            A, B = payload
            self.A, self.B = A, B
            self.t = [torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()]
            self.Am, self.Bm = mad.dense(self.t[0]), mad.dense(self.t[1])
            MA, MB = oracle.Matrix(A), oracle.Matrix(B)
        else:
            rp, ci, nodes = payload
            self.t = [torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()]
            self.Am = self.Bm = mad.csr(self.t[0], self.t[1], (nodes, nodes))
            MA = MB = oracle.Matrix(rowptr=rp, colidx=ci, shape=(nodes, nodes))
        self.ctx.build(self.Am, self.Bm, s_max, keep=tuple(self.t))
        self.oracle = oracle.Oracle(MA, MB, self.flags, s_max)
        self.dense = kind == "dense"

    def close(self):
        self.ctx.close()


@pytest.mark.parametrize("name", ["dense_ragged_f32", "dense_f64_nonneg", "dense_gram",
                                  "chung_lu_gram"])
def test_wedge_tables_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    c = WedgeCase(name, 1 << 20)
    try:
        tk = mad.mad_export_table(c.ctx.ctx, "TK").cpu().numpy().view(np.uint64)
        assert np.array_equal(tk, c.oracle.table("TK"))
        st = mad.mad_stats(c.ctx.ctx)
        assert st["t1_total"] == int(tk[-1])
        if c.dense:
            nac = mad.mad_export_table(c.ctx.ctx, "nac").cpu().numpy()
            assert np.array_equal(nac.view(np.uint32), c.oracle.table("nac").view(np.uint32))
            tac = mad.mad_export_table(c.ctx.ctx, "TAc").cpu().numpy().view(np.uint32)
            if c.flags & 2:
                assert len(tac) == 0   # Gram: column k of A is row k of B (TB)
            else:
                ref = c.oracle.table("TAc")
                assert np.array_equal(tac & np.uint32(0x7FFFFFFF), ref)
                signs = (tac >> np.uint32(31)).astype(bool)
                Af = c.A.astype(np.float32)
                assert np.array_equal(signs, (Af.T.reshape(-1) < 0))
    finally:
        c.close()


@pytest.mark.parametrize("name", ["dense_ragged_f32", "dense_f64_nonneg", "dense_gram",
                                  "chung_lu_gram"])
def test_wedge_draws_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    c = WedgeCase(name, 1 << 20)
    try:
        first, count = (1 << 33) + 17, 40_000
        gi, gk, gj, gkp, gv = [x.cpu().numpy() for x in
                               mad.mad_debug_draws(c.ctx.ctx, 77, first, count)]
        oi, ok, oj, okp, ov = c.oracle.draw(seed=77, first=first, count=count)
        assert np.array_equal(gk, ok)
        assert np.array_equal(gi, oi) and np.array_equal(gj, oj)
        assert np.all(gkp == 0)
        assert np.array_equal(gv, ov)
        assert mad.mad_stats(c.ctx.ctx)["device_error"] == 0
    finally:
        c.close()


@pytest.mark.parametrize("name", ["dense_ragged_f32", "dense_gram", "chung_lu_gram"])
def test_wedge_x_and_top_t_bit_exact(name):
    import paper_1506_03872_gb300 as mad
    s, seed, tprime, t = 300_000, 19, 1500, 30
    c = WedgeCase(name, s)
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


def test_wedge_refusals():
    """MAD_WEDGE with the squared symmetric update, 0/1 inputs that are not
    Gram, and the fused pass are refused."""
    import paper_1506_03872_gb300 as mad
    with pytest.raises(mad.MadError) as e:
        mad.mad_create(WEDGE | 8 | 2)
    assert e.value.status == mad.MAD_ERR_ARG
    rng = _rng(5)
    A = (rng.random((50, 30)) < 0.2)
    B = (rng.random((30, 40)) < 0.2)
    A[:, 0] = B[0, :] = True
    rpa = np.concatenate([[0], np.cumsum(A.sum(1))]).astype(np.int64)
    rpb = np.concatenate([[0], np.cumsum(B.sum(1))]).astype(np.int64)
    ta = [torch.from_numpy(rpa).cuda(), torch.from_numpy(np.nonzero(A)[1].astype(np.int32)).cuda()]
    tb = [torch.from_numpy(rpb).cuda(), torch.from_numpy(np.nonzero(B)[1].astype(np.int32)).cuda()]
    with mad.Context(WEDGE) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_build_tables(c.ctx, mad.csr(ta[0], ta[1], A.shape),
                                 mad.csr(tb[0], tb[1], B.shape), 1000)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
    Ad = torch.randn(100, 8, device="cuda")
    Bd = torch.randn(8, 90, device="cuda")
    with mad.Context(WEDGE) as c:
        with pytest.raises(mad.MadError) as e:
            mad.mad_pipeline_plan(c.ctx, mad.dense(Ad), mad.dense(Bd), 10_000, 100, 10)
        assert e.value.status == mad.MAD_ERR_UNSUPPORTED
