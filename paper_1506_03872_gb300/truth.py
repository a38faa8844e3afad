"""Exact ground truth for recall measurements (test, bench and training
harness; not on the sampling path): the exact top t of a dense product by
FP32 cuBLAS with a rounding margin and FP64 rescoring, and of a 0/1 Gram
product by degree pruning; recall of a returned top t against it."""
from __future__ import annotations

import numpy as np


def ground_truth_dense(A, B, t):
    """Exact top-t of |A B| (harness only): FP32 cuBLAS GEMM in row blocks
    with a margin covering its rounding error, then FP64 rescoring."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    m, d = A.shape
    n = B.shape[1]
    na = A.double().norm(dim=1).max().item()
    nb = B.double().norm(dim=0).max().item()
    err = 2.0 * d * 2.0 ** -24 * na * nb
    block = 8192
    vals = []
    for r0 in range(0, m, block):
        c = (A[r0:r0 + block] @ B).abs_()
        v, _ = torch.topk(c.flatten(), min(8 * t, c.numel()))
        vals.append(v)
    theta = torch.topk(torch.cat(vals), t).values[-1].item()
    cand = []
    for r0 in range(0, m, block):
        c = (A[r0:r0 + block] @ B).abs_()
        idx = torch.nonzero(c >= theta - 2 * err)
        idx[:, 0] += r0
        cand.append(idx)
    cand = torch.cat(cand)
    exact = (A[cand[:, 0]].double() * B[:, cand[:, 1]].T.double()).sum(dim=1).abs()
    order = torch.argsort(-exact, stable=True)[:t]
    keys = (cand[order, 0].to(torch.int64) << 32) | cand[order, 1].to(torch.int64)
    tau = exact[order[-1]].item()
    ground_truth_dense.top1 = exact[order[0]].item()
    return set(keys.cpu().tolist()), tau


def ground_truth_gram_binary(rowptr, colidx, t, device, h0=2048):
    """Exact top-t common-neighbour counts over unordered off-diagonal pairs
    of a symmetric 0/1 adjacency (harness only; recall ground truth).

    A pair's count is at most the smaller of its two degrees.  So with H the
    h highest-degree nodes, once the t-th largest count among pairs inside H
    exceeds the largest degree outside H, no pair with an end outside H can
    reach or tie it, and the top t inside H is the top t overall.  Counts
    inside H are dense products of 0/1 column blocks (FP16 on a GPU, partial
    sums of at most 2048 ones exact; FP32 elsewhere) accumulated in FP32; h
    doubles until the condition holds.

    Returns (tau, counts) with tau the t-th largest count and `counts` a
    function giving the exact count of given (i, j) pairs inside H (None
    outside H)."""
    import torch
    rp = torch.as_tensor(np.asarray(rowptr, dtype=np.int64), device=device)
    ci = torch.as_tensor(np.asarray(colidx).astype(np.int64), device=device)
    n = rp.numel() - 1
    deg = rp[1:] - rp[:-1]
    order = torch.argsort(-deg, stable=True)
    fdt = torch.float16 if rp.is_cuda else torch.float32
    chunk = 2048
    h = min(n, max(h0, 2 * t))
    while True:
        H = order[:h]
        outside = int(deg[order[h]].item()) if h < n else -1
        lens = deg[H]
        total = int(lens.sum().item())
        local = torch.repeat_interleave(torch.arange(h, device=device), lens)
        first = torch.repeat_interleave(rp[H] - (torch.cumsum(lens, 0) - lens), lens)
        cols = ci[torch.arange(total, device=device) + first]
        cs, perm = torch.sort(cols)
        ls = local[perm]
        _, inv = torch.unique_consecutive(cs, return_inverse=True)
        u = int(inv[-1].item()) + 1 if total else 0
        C = torch.zeros(h, h, dtype=torch.float32, device=device)
        bounds = torch.searchsorted(inv, torch.arange(0, u + chunk, chunk, device=device))
        for q in range((u + chunk - 1) // chunk):
            lo, hi = int(bounds[q].item()), int(bounds[q + 1].item())
            blk = torch.zeros(h, chunk, dtype=fdt, device=device)
            blk[ls[lo:hi], inv[lo:hi] - q * chunk] = 1
            C += (blk @ blk.T).float()
        iu = torch.triu_indices(h, h, 1, device=device)
        vals = C[iu[0], iu[1]]
        kk = min(t, vals.numel())
        tau = float(torch.topk(vals, kk).values[-1].item()) if kk else 0.0
        if tau > outside or h >= n:
            break
        h = min(n, 2 * h)
    pos = torch.full((n,), -1, dtype=torch.int64, device=device)
    pos[H] = torch.arange(h, device=device)
    Cc = C

    def counts(i, j):
        pi = pos[torch.as_tensor(np.asarray(i, dtype=np.int64), device=device)]
        pj = pos[torch.as_tensor(np.asarray(j, dtype=np.int64), device=device)]
        inside = (pi >= 0) & (pj >= 0)
        v = torch.full(pi.shape, float("nan"), dtype=torch.float64, device=device)
        v[inside] = Cc[pi[inside], pj[inside]].double()
        return v.cpu().numpy()

    counts.top1 = float(vals.max().item()) if vals.numel() else 0.0
    return tau, counts


def recall_of(w, gi, gj, gc, truth, tau, counts=None):
    """|Omega_t ∩ T_t| / t.  Dense: key intersection with the exact top t.
    Integer (C3): results with an exact count >= the t-th largest count are
    hits, since pairs tied with the t-th value are all top-t pairs; the
    reported counts are also checked against the exact ones."""
    if counts is None:
        got = set(mad_keys(gi, gj))
        return len(got & truth) / w.t, None
    exact = counts(gi, gj)
    known = ~np.isnan(exact)
    mismatch = int(np.sum(exact[known] != gc[known]))
    hits = int(np.sum(gc >= tau))
    return min(hits, w.t) / w.t, mismatch


def mad_keys(gi, gj):
    return ((gi.astype(np.int64) << 32) | gj.astype(np.int64)).tolist()
