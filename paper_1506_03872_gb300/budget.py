"""Learned diamond budget: a small perceptron, trained on recall curves the
sampler itself produced, proposes the number of diamonds s that reaches a
target recall of the top t on an instance, from cheap statistics of the
instance (`mad_budget_features`).  Training and inference run in the
library's kernels (`mad_mlp_train`, `mad_mlp_predict`); this module only
generates the seeded instances, measures their recall curves against exact
ground truth, normalises the features and applies the fallback rule.

Theorem 2 of the paper says s of order ||W||_1 / tau^2 diamonds separate the
entries above tau; tau is unknown before the run, so the features carry
||W||_1, sizes, and Cauchy-Schwarz and concentration stand-ins for it.  A
run with the proposed budget falls back to the fixed budget when its own
exact rescoring contradicts the proposal: with tau_hat the t-th largest
exact |c| it found, s * tau_hat^2 / ||W||_1 must reach the smallest value
seen on training instances that met the target.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

# Budgets tried per instance: 1e4 .. 1e8 in steps of sqrt(10).
LADDER = [int(round(10 ** (4 + q / 2))) for q in range(9)]
TARGET = 0.95
BEYOND = 8.75        # label of an instance that misses the target at every budget


def instance(index: int, seed: int = 5):
    """Instance `index` of the mixed training recipe: even indices are
    dense factor matrices (m, n log-uniform in [1e4, 2e5], d uniform in
    [20, 300]), odd ones Chung-Lu 0/1 graphs (nodes log-uniform in
    [1e4, 2e5], mean degree 20, Gram pairs without the diagonal); t = 10,
    t' = 1000."""
    from . import workloads as W
    rng = np.random.Generator(np.random.PCG64([seed, index]))
    if index % 2 == 0:
        m = int(np.exp(rng.uniform(np.log(1e4), np.log(2e5))))
        n = int(np.exp(rng.uniform(np.log(1e4), np.log(2e5))))
        d = int(rng.integers(20, 301))
        w = W.dense_factors(m=m, d=d, n=n, seed=10_000 + index, s=LADDER[-1], t=10, tprime=1000)
    else:
        nodes = int(np.exp(rng.uniform(np.log(1e4), np.log(2e5))))
        w = W.chung_lu(nodes=nodes, edges=10 * nodes, seed=10_000 + index, s=LADDER[-1], t=10,
                       tprime=1000)
    w.sampler_seed = 20_000 + index
    return w


@dataclass
class Curve:
    features: np.ndarray
    w1: float
    s: list          # budgets run
    recall: list     # recall of the top t at each budget
    ms: list         # device time of build + sample + top-t' + rescore
    tau_hat: list    # t-th largest exact |c| found at each budget

    def label(self) -> float:
        """log10 of the first budget reaching the target (BEYOND if none)."""
        for s, r in zip(self.s, self.recall):
            if r >= TARGET:
                return float(np.log10(s))
        return BEYOND


def recall_curve(w, full: bool = False) -> Curve:
    """Features and the recall curve over LADDER (stopping at the first
    budget that reaches the target unless `full`)."""
    import torch

    from . import (Context, csr, decode_pairs, dense, mad_budget_features, mad_build_tables,
                   mad_rescore, mad_sample, mad_stats, mad_topk)
    from .truth import ground_truth_dense, ground_truth_gram_binary, recall_of
    dev = torch.device("cuda")
    if w.csr:
        rp, ci = torch.from_numpy(w.rowptr).to(dev), torch.from_numpy(w.colidx).to(dev)
        A = B = csr(rp, ci, (w.m, w.d))
        keep = (rp, ci)
        tau, counts = ground_truth_gram_binary(w.rowptr, w.colidx, w.t, dev)
        truth = set()
    else:
        tA, tB = torch.from_numpy(w.A).to(dev), torch.from_numpy(w.B).to(dev)
        A, B = dense(tA), dense(tB)
        keep = (tA, tB)
        truth, tau = ground_truth_dense(tA, tB, w.t)
        counts = None
    ctx = Context(w.flags)
    try:
        mad_build_tables(ctx.ctx, A, B, LADDER[-1])
        feats = mad_budget_features(ctx.ctx)
        w1 = mad_stats(ctx.ctx)["w1"]
        cur = Curve(feats, w1, [], [], [], [])
        for s in LADDER:
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            mad_build_tables(ctx.ctx, A, B, s)
            mad_sample(ctx.ctx, s, w.sampler_seed)
            cand, nc = mad_topk(ctx.ctx, w.tprime)
            res, nr = mad_rescore(ctx.ctx, cand, nc, w.t)
            e1.record()
            torch.cuda.synchronize()
            gi, gj, gx, gc = decode_pairs(res, nr)
            r, _ = recall_of(w, gi, gj, gc, truth, tau, counts)
            cur.s.append(s)
            cur.recall.append(float(r))
            cur.ms.append(e0.elapsed_time(e1))
            cur.tau_hat.append(float(np.abs(gc).min()) if nr >= w.t else 0.0)
            if r >= TARGET and not full:
                break
        del keep
        return cur
    finally:
        ctx.close()


class BudgetPredictor:
    """log10 of the budget from the features; trained with the library's
    kernels on the pinball loss of level `quantile` (so it errs towards
    larger budgets)."""

    def __init__(self, f: int, seed: int = 0):
        import torch

        from . import MAD_MLP_HIDDEN, mlp_params
        rng = np.random.Generator(np.random.PCG64(seed))
        h = MAD_MLP_HIDDEN
        parts = [rng.uniform(-1, 1, h * f) * np.sqrt(6.0 / f), np.zeros(h),
                 rng.uniform(-1, 1, h * h) * np.sqrt(6.0 / h), np.zeros(h),
                 rng.uniform(-1, 1, h) * np.sqrt(3.0 / h), np.zeros(1)]
        p = np.concatenate(parts).astype(np.float32)
        assert p.size == mlp_params(f)
        self.params = torch.from_numpy(p).cuda()
        self.f = f
        self.mu = np.zeros(f, np.float32)
        self.sd = np.ones(f, np.float32)
        self.y_mu = 0.0

    def _x(self, X):
        import torch
        return torch.from_numpy(((np.asarray(X, np.float32) - self.mu) / self.sd).astype(np.float32)).cuda()

    def fit(self, X, y, epochs: int = 3000, lr: float = 3e-3, quantile: float = 0.8):
        import torch

        from . import mad_mlp_train
        from . import Context
        X = np.asarray(X, np.float32)
        self.mu = X.mean(axis=0)
        self.sd = np.maximum(X.std(axis=0), 1e-3).astype(np.float32)
        self.y_mu = float(np.mean(y))
        yt = torch.from_numpy((np.asarray(y, np.float32) - self.y_mu).astype(np.float32)).cuda()
        loss = torch.zeros(epochs, dtype=torch.float32, device="cuda")
        with Context() as c:
            mad_mlp_train(c.ctx, self.params, self._x(X), yt, epochs, lr, quantile, loss)
            torch.cuda.synchronize()
        return loss.cpu().numpy()

    def predict(self, X) -> np.ndarray:
        from . import mad_mlp_predict
        return mad_mlp_predict(self.params, self._x(X)).cpu().numpy() + self.y_mu


def experiment(count: int = 512, train_fraction: float = 0.75, seed: int = 5,
               log=print) -> dict:
    """The learned-budget experiment: `count` instances of the mixed recipe,
    a predictor trained on the first part, evaluated on the rest against
    the fixed budget LADDER[-1] (with the fallback rule)."""
    t0 = time.perf_counter()
    curves = []
    n_train = int(round(count * train_fraction))
    for q in range(count):
        w = instance(q, seed)
        curves.append(recall_curve(w, full=q >= n_train))
        if log and (q + 1) % 32 == 0:
            log(f"instances {q + 1}/{count} ({time.perf_counter() - t0:.0f} s)")
    X = np.stack([c.features for c in curves])
    y = np.array([c.label() for c in curves], np.float32)
    model = BudgetPredictor(X.shape[1], seed)
    loss = model.fit(X[:n_train], y[:n_train])
    # fallback constant: the smallest s tau_hat^2 / ||W||_1 among training
    # instances that reached the target
    rho = [s * th * th / c.w1 for c in curves[:n_train] for s, r, th in zip(c.s, c.recall, c.tau_hat)
           if r >= TARGET]
    rho_min = float(np.min(rho)) if rho else 0.0
    pred = model.predict(X[n_train:])
    rec_p, rec_f, ms_p, ms_f, fell_back, hit = [], [], [], [], 0, 0
    kind = []
    for c, yh in zip(curves[n_train:], pred):
        kind.append(int(c.features[5]))
        fixed = len(c.s) - 1
        if yh >= np.log10(LADDER[-1]) + 0.25:
            q = fixed
        else:
            q = next((i for i, s in enumerate(c.s) if np.log10(s) >= yh - 1e-6), fixed)
        ms = c.ms[q]
        r = c.recall[q]
        if q != fixed and c.s[q] * c.tau_hat[q] ** 2 / c.w1 < rho_min:
            fell_back += 1
            ms += c.ms[fixed]
            r = c.recall[fixed]
        rec_p.append(r)
        rec_f.append(c.recall[fixed])
        ms_p.append(ms)
        ms_f.append(c.ms[fixed])
        hit += r >= TARGET
    per_kind = {}
    for kname, kv in (("dense", 0), ("binary", 1)):
        sel = [q for q, k in enumerate(kind) if k == kv]
        if sel:
            per_kind[kname] = {
                "test": len(sel),
                "meeting_target_predicted": int(sum(rec_p[q] >= TARGET for q in sel)),
                "meeting_target_fixed": int(sum(rec_f[q] >= TARGET for q in sel)),
                "time_saved_fraction": float(1.0 - sum(ms_p[q] for q in sel) / sum(ms_f[q] for q in sel)),
            }
    return {
        "instances": count, "train": n_train, "test": count - n_train, "per_kind": per_kind,
        "label_reached": int(np.sum(y < BEYOND)),
        "train_loss_first_last": [float(loss[0]), float(loss[-1])],
        "recall_predicted_mean": float(np.mean(rec_p)),
        "recall_fixed_mean": float(np.mean(rec_f)),
        "test_meeting_target_predicted": int(hit),
        "test_meeting_target_fixed": int(np.sum(np.array(rec_f) >= TARGET)),
        "fallbacks": fell_back,
        "ms_predicted_mean": float(np.mean(ms_p)),
        "ms_fixed_mean": float(np.mean(ms_f)),
        "time_saved_fraction": float(1.0 - np.sum(ms_p) / np.sum(ms_f)),
        "seconds": round(time.perf_counter() - t0, 1),
    }
