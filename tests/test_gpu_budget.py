"""The learned budget predictor's kernels on the GPU: the instance features
against NumPy, inference and training of the perceptron against the NumPy
statement in tests/mlp_reference.py."""
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


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_features_dense_and_binary():
    import paper_1506_03872_gb300 as mad
    from paper_1506_03872_gb300.workloads import chung_lu, dense_factors
    w = dense_factors(m=3000, d=40, n=2000, seed=17)
    tA, tB = torch.from_numpy(w.A).cuda(), torch.from_numpy(w.B).cuda()
    with mad.Context() as c:
        mad.mad_build_tables(c.ctx, mad.dense(tA), mad.dense(tB), 10 ** 6)
        f = mad.mad_budget_features(c.ctx)
        st = mad.mad_stats(c.ctx)
        T1 = mad.mad_export_table(c.ctx, "T1").cpu().numpy().view(np.uint64).astype(np.float64)
    q = np.diff(np.concatenate([[0.0], T1]))
    ref = [np.log10(3000), np.log10(2000), np.log10(40), np.log10(3000 * 40), np.log10(40 * 2000), 0,
           np.log10(st["w1"]), np.log10(np.linalg.norm(w.A, axis=1).max()),
           np.log10(np.linalg.norm(w.B, axis=0).max()), np.log10((q ** 2).sum() / q.sum() ** 2),
           np.log10(q.max() / q.sum())]
    ref.append(ref[6] - 2 * (ref[7] + ref[8]))
    assert np.allclose(f, np.array(ref, np.float32), rtol=0, atol=2e-5)
    g = chung_lu(nodes=3000, edges=30000, seed=18)
    rp, ci = torch.from_numpy(g.rowptr).cuda(), torch.from_numpy(g.colidx).cuda()
    M = mad.csr(rp, ci, (g.m, g.d))
    with mad.Context(g.flags) as c:
        mad.mad_build_tables(c.ctx, M, M, 10 ** 6)
        f = mad.mad_budget_features(c.ctx)
    deg = np.diff(g.rowptr)
    assert f[5] == 1.0
    assert np.isclose(f[7], np.log10(np.sqrt(deg.max())), atol=1e-6)
    assert np.isclose(f[8], np.log10(np.sqrt(np.bincount(g.colidx).max())), atol=1e-6)


def _params(f, seed):
    import mlp_reference as R
    rng = _rng(seed)
    return (rng.standard_normal(R.H * f + 3 * R.H + R.H * R.H + 1) * 0.15).astype(np.float32)


def test_inference_matches_reference():
    import mlp_reference as R
    import paper_1506_03872_gb300 as mad
    f, n = 12, 777
    p = _params(f, 1)
    X = _rng(2).standard_normal((n, f)).astype(np.float32)
    y = mad.mad_mlp_predict(torch.from_numpy(p).cuda(), torch.from_numpy(X).cuda()).cpu().numpy()
    ref, _ = R.forward(p, X, np.float64)
    assert np.allclose(y, ref, rtol=1e-5, atol=1e-5)


def test_training_follows_reference_and_learns():
    import mlp_reference as R
    import paper_1506_03872_gb300 as mad
    f, n = 12, 300
    rng = _rng(3)
    X = rng.standard_normal((n, f)).astype(np.float32)
    y = (X[:, 0] * 1.5 - X[:, 3] + 0.5 * np.abs(X[:, 5]) + 4.0).astype(np.float32)
    p0 = _params(f, 4)
    epochs, lr, q = 40, 3e-3, 0.8
    P = torch.from_numpy(p0).cuda()
    loss = torch.zeros(epochs, device="cuda")
    with mad.Context() as c:
        mad.mad_mlp_train(c.ctx, P, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), epochs,
                          lr, q, loss)
        torch.cuda.synchronize()
    p_ref, loss_ref = R.train(p0, X, y, epochs, lr, q)
    assert np.allclose(loss.cpu().numpy(), loss_ref, rtol=2e-3, atol=1e-5)
    assert np.allclose(P.cpu().numpy(), p_ref, rtol=1e-2, atol=2e-4)
    # a longer run fits the target
    P = torch.from_numpy(p0).cuda()
    loss = torch.zeros(1500, device="cuda")
    with mad.Context() as c:
        mad.mad_mlp_train(c.ctx, P, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), 1500,
                          1e-2, 0.5, loss)
        torch.cuda.synchronize()
    ls = loss.cpu().numpy()
    assert ls[-1] < 0.1 * ls[0]


def test_budget_experiment_runs_small():
    from paper_1506_03872_gb300 import budget
    res = budget.experiment(count=8, train_fraction=0.5, log=None)
    assert res["test"] == 4
    assert 0.0 <= res["recall_predicted_mean"] <= 1.0
    assert res["train_loss_first_last"][1] <= res["train_loss_first_last"][0]
