"""Seeded synthetic inputs for t-MAD search (numpy PCG64).

This module builds inputs only; it holds none of diamond sampling's
arithmetic and both the CUDA library's tests and the CPU oracle read from it.
Each workload stands in for a family of the paper's experiments (Sec. 6.1),
whose datasets are not available here:

* ``plain_small``      -- A 1000x25, B 25x1000, FP64 N(0,1), 10 planted pairs
                          at ~3x the background maximum |c_ij|.
* ``dense_factors``    -- recommender factor matrices (stands in for the
                          MovieLens SVD factors of Sec. 6.1): every vector
                          (row of A, column of B) is a log-normal norm
                          (sigma 0.5) times a uniform random direction, FP32.
* ``chung_lu``         -- 0/1 symmetric adjacency of a Chung-Lu graph with
                          power-law expected degrees (exponent 2.1), CSR with
                          sorted int32 columns (stands in for the SNAP graphs
                          of Sec. 6.1 used as A^T A).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np


@dataclass
class Workload:
    name: str
    A: Optional[np.ndarray] = None          # dense m x d (row-major)
    B: Optional[np.ndarray] = None          # dense d x n (row-major)
    rowptr: Optional[np.ndarray] = None     # CSR of A (and of B = A^T) for graphs
    colidx: Optional[np.ndarray] = None
    m: int = 0
    d: int = 0
    n: int = 0
    s: int = 0
    t: int = 0
    tprime: int = 0
    flags: int = 0
    sampler_seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def csr(self) -> bool:
        return self.rowptr is not None


def _unit_rows(rng: np.random.Generator, count: int, d: int, sigma: float) -> np.ndarray:
    g = rng.standard_normal((count, d))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    norms = np.exp(sigma * rng.standard_normal(count))
    return g * norms[:, None]


def plain_small(m: int = 1000, d: int = 25, n: int = 1000, planted: int = 10, seed: int = 1,
                s: int = 100_000, t: int = 10, tprime: int = 100) -> Workload:
    """A (m x d), B (d x n) i.i.d. N(0,1) in FP64 with ``planted`` pairs.

    Planted pair p (distinct rows i_p, distinct columns j_p) sets column
    b_{j_p} to a_{i_p} scaled so that a_{i_p} . b_{j_p} = 3 (1 + 0.02 p) M,
    with M the largest |a_i . b_j| before planting.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.standard_normal((m, d))
    B = rng.standard_normal((d, n))
    background = float(np.abs(A @ B).max())
    rows = rng.choice(m, size=planted, replace=False)
    cols = rng.choice(n, size=planted, replace=False)
    for p, (i, j) in enumerate(zip(rows, cols)):
        a = A[i]
        B[:, j] = a * (3.0 * background * (1.0 + 0.02 * p) / float(a @ a))
    return Workload("plain_small", A=A, B=np.ascontiguousarray(B), m=m, d=d, n=n, s=s, t=t,
                    tprime=tprime, sampler_seed=101,
                    meta={"planted_rows": rows, "planted_cols": cols, "background": background})


def dense_factors(m: int = 200_000, d: int = 100, n: int = 50_000, seed: int = 2,
                  s: int = 10_000_000, t: int = 100, tprime: int = 10_000,
                  sigma: float = 0.5) -> Workload:
    """Factor matrices: A rows and B columns are exp(sigma z) * unit Gaussian."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = _unit_rows(rng, m, d, sigma).astype(np.float32)
    Bt = _unit_rows(rng, n, d, sigma).astype(np.float32)
    B = np.ascontiguousarray(Bt.T)
    return Workload("dense_factors", A=A, B=B, m=m, d=d, n=n, s=s, t=t, tprime=tprime,
                    sampler_seed=102)


def batched_queries(n: int = 1_000_000, d: int = 300, nq: int = 10_000, seed: int = 4,
                    s_lo: int = 1_000, s_hi: int = 100_000, t: int = 5, tprime: int = 100,
                    sigma: float = 0.5) -> Workload:
    """Batched maximum-|inner-product| queries: n item vectors and nq query
    vectors, each exp(sigma z) * a unit Gaussian direction, and a budget per
    query drawn uniformly from [s_lo, s_hi].  A = the queries (nq x d), B =
    the items as columns (d x n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    B = np.empty((d, n), dtype=np.float32)
    step = 65536
    for j0 in range(0, n, step):
        j1 = min(n, j0 + step)
        B[:, j0:j1] = _unit_rows(rng, j1 - j0, d, sigma).astype(np.float32).T
    Q = _unit_rows(rng, nq, d, sigma).astype(np.float32)
    s_q = rng.integers(s_lo, s_hi + 1, size=nq, dtype=np.int64).astype(np.uint64)
    return Workload("batched_queries", A=Q, B=B, m=nq, d=d, n=n, s=int(s_q.sum()), t=t,
                    tprime=tprime, sampler_seed=104,
                    meta={"s_per_query": s_q, "s_max": int(s_hi)})


def _chung_lu_offset(nodes: int, exponent: float, max_share: float) -> float:
    """Offset v0 in w_v = (v + v0)^(-1/(exponent-1)) so that the heaviest
    node holds ``max_share`` of the total weight (caps the largest degree)."""
    alpha = 1.0 / (exponent - 1.0)
    v = np.arange(nodes, dtype=np.float64)
    lo, hi = 0.0, float(nodes)
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        w = (v + mid) ** (-alpha)
        share = w[0] / w.sum()
        if share > max_share:
            lo = mid
        else:
            hi = mid
    return hi


def _draw_nodes(rng: np.random.Generator, cdf: np.ndarray, count: int) -> np.ndarray:
    """``count`` i.i.d. node draws from the cumulative weights ``cdf``."""
    u = rng.random(count)
    order = np.argsort(u, kind="stable")
    out = np.empty(count, dtype=np.int64)
    out[order] = np.searchsorted(cdf, u[order], side="right")
    return np.minimum(out, len(cdf) - 1)


def chung_lu(nodes: int = 1_000_000, edges: int = 10_000_000, exponent: float = 2.1,
             seed: int = 3, s: int = 100_000_000, t: int = 1000, tprime: int = 100_000,
             max_degree_share: Optional[float] = None) -> Workload:
    """Undirected Chung-Lu graph: ``edges`` endpoint pairs drawn i.i.d. with
    probability proportional to w_u w_v, self-loops and duplicates dropped,
    then symmetrised.  The heaviest node's expected share of endpoints is
    capped (default 1/sqrt(2 edges)), the usual structural cutoff."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if max_degree_share is None:
        max_degree_share = 1.0 / np.sqrt(2.0 * edges)
    v0 = _chung_lu_offset(nodes, exponent, max_degree_share)
    w = (np.arange(nodes, dtype=np.float64) + v0) ** (-1.0 / (exponent - 1.0))
    p = w / w.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    src = _draw_nodes(rng, cdf, edges)
    dst = _draw_nodes(rng, cdf, edges)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = np.sort(np.minimum(src, dst) * nodes + np.maximum(src, dst))
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    lo, hi = key // nodes, key % nodes
    both = np.sort(np.concatenate([lo * nodes + hi, hi * nodes + lo]))
    rows, cols = both // nodes, both % nodes
    counts = np.bincount(rows, minlength=nodes)
    rowptr = np.zeros(nodes + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colidx = cols.astype(np.int32)
    # A = B = adjacency (symmetric), Gram pairs, diagonal excluded.
    flags = 2 | 4
    return Workload("chung_lu", rowptr=rowptr, colidx=colidx, m=nodes, d=nodes, n=nodes, s=s,
                    t=t, tprime=tprime, flags=flags, sampler_seed=103,
                    meta={"v0": v0, "undirected_edges": int(len(key))})


def by_name(name: str, **kw) -> Workload:
    return {"plain_small": plain_small, "dense_factors": dense_factors,
            "chung_lu": chung_lu, "batched_queries": batched_queries}[name](**kw)
