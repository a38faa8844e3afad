"""Shared set-up for the GPU parity tests: one seeded input, the library
context built on it, and the CPU oracle built on the same arrays."""
from __future__ import annotations

import numpy as np

import oracle
from paper_1506_03872_gb300 import workloads as W


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def case_inputs(name: str):
    """(kind, payload, flags) for a named parity case."""
    if name == "plain_small":            # the small FP64 workload, full size
        w = W.plain_small()
        return "dense", (w.A, w.B), 0
    if name == "dense_ragged_f32":        # several tiles and ragged tails
        rng = _rng(41)
        A = (rng.standard_normal((2051, 100)) * np.exp(0.5 * rng.standard_normal((2051, 1))))
        B = (rng.standard_normal((100, 3001)) * np.exp(0.5 * rng.standard_normal((1, 3001))))
        return "dense", (A.astype(np.float32), B.astype(np.float32)), 0
    if name == "dense_wide_rows":          # rows of B longer than the wide-row threshold
        rng = _rng(47)
        A = (rng.standard_normal((500, 60)) * np.exp(0.5 * rng.standard_normal((500, 1))))
        B = (rng.standard_normal((60, 20011)) * np.exp(0.5 * rng.standard_normal((1, 20011))))
        B[3, :] = 0.0
        return "dense", (A.astype(np.float32), B.astype(np.float32)), 0
    if name == "dense_deep":               # d above 256: the general row kernel of A
        rng = _rng(48)
        A = rng.standard_normal((300, 300)) * np.exp(0.5 * rng.standard_normal((300, 1)))
        B = rng.standard_normal((300, 450))
        return "dense", (A.astype(np.float32), B.astype(np.float32)), 0
    if name.startswith("dense_short_d"):   # d <= 256: the register-row kernel of A
        d = int(name[len("dense_short_d"):])
        rng = _rng(50 + d)
        A = rng.standard_normal((257, d)) * np.exp(0.5 * rng.standard_normal((257, 1)))
        A[rng.random(A.shape) < 0.1] = 0.0
        B = rng.standard_normal((d, 301)) * np.exp(0.5 * rng.standard_normal((1, 301)))
        return "dense", (A.astype(np.float32), B.astype(np.float32)), 0
    if name == "dense_factors_small":
        w = W.dense_factors(m=4000, d=100, n=1500, seed=8)
        return "dense", (w.A, w.B), 0
    if name == "dense_mixed_signs_zeros":  # exact zeros, tiny and huge values
        rng = _rng(43)
        A = rng.standard_normal((300, 37)).astype(np.float32)
        A[rng.random(A.shape) < 0.3] = 0.0
        A[5, :] = 0.0
        A[7, 3] = 1e-30
        B = rng.standard_normal((37, 513)).astype(np.float32) * 1e3
        B[rng.random(B.shape) < 0.2] = 0.0
        return "dense", (A, B), 0
    if name == "dense_nonneg":
        rng = _rng(44)
        A = np.abs(rng.standard_normal((500, 50))).astype(np.float32)
        B = np.abs(rng.standard_normal((50, 700))).astype(np.float32)
        return "dense", (A, B), 1
    if name == "gram_dense":
        rng = _rng(45)
        A = rng.standard_normal((400, 30))
        return "dense", (A, np.ascontiguousarray(A.T)), 2 | 4
    if name == "dense_square_sym":          # Sec. 3.2.3 on dense A = A^T = B
        rng = _rng(47)
        S = rng.standard_normal((350, 350))
        S = (S + S.T).astype(np.float32)
        S[np.abs(S) < 0.3] = 0.0
        return "dense", (S, S.copy()), 2 | 4 | 8
    if name == "chung_lu_small":
        w = W.chung_lu(nodes=5000, edges=40000, seed=9)
        return "csr", (w.rowptr, w.colidx, w.m), w.flags
    if name == "chung_lu_square_sym":      # Sec. 3.2.3 update on A = A^T
        w = W.chung_lu(nodes=5000, edges=40000, seed=9)
        return "csr", (w.rowptr, w.colidx, w.m), w.flags | 8
    if name == "bipartite_binary":         # 0/1 CSR, A != B^T, no Gram
        rng = _rng(46)
        A = (rng.random((600, 80)) < 0.05)
        B = (rng.random((80, 900)) < 0.04)
        A[:, 0] = True
        B[0, :5] = True
        return "csr2", (A, B), 0
    raise KeyError(name)


def _csr_of(M):
    rowptr = np.concatenate([[0], np.cumsum(M.sum(axis=1))]).astype(np.int64)
    colidx = np.nonzero(M)[1].astype(np.int32)
    return rowptr, colidx


class Case:
    """Library context and oracle on the same inputs."""

    def __init__(self, name: str, s_max: int, hash_capacity: int = 0):
        import torch

        import paper_1506_03872_gb300 as mad
        self.name = name
        kind, payload, flags = case_inputs(name)
        self.flags = flags
        self.ctx = mad.Context(flags)
        if hash_capacity:
            mad.mad_set_hash_capacity(self.ctx.ctx, hash_capacity)
        if kind == "dense":
            A, B = payload
            self.A, self.B = A, B
            tA = torch.from_numpy(A).cuda()
            tB = torch.from_numpy(B).cuda()
            self.Am, self.Bm = mad.dense(tA), mad.dense(tB)
            self.ctx.build(self.Am, self.Bm, s_max, keep=(tA, tB))
            self.oracle = oracle.Oracle(oracle.Matrix(A), oracle.Matrix(B), flags, s_max)
            self.m, self.d, self.n = A.shape[0], A.shape[1], B.shape[1]
        else:
            if kind == "csr":
                rowptr, colidx, nodes = payload
                ra, ca, rb, cb = rowptr, colidx, rowptr, colidx
                shapeA = shapeB = (nodes, nodes)
            else:
                Ad, Bd = payload
                ra, ca = _csr_of(Ad)
                rb, cb = _csr_of(Bd)
                shapeA, shapeB = Ad.shape, Bd.shape
            self.csr = (ra, ca, rb, cb)
            t = [torch.from_numpy(x).cuda() for x in (ra, ca, rb, cb)]
            self.Am, self.Bm = mad.csr(t[0], t[1], shapeA), mad.csr(t[2], t[3], shapeB)
            self.ctx.build(self.Am, self.Bm, s_max, keep=tuple(t))
            self.oracle = oracle.Oracle(oracle.Matrix(rowptr=ra, colidx=ca, shape=shapeA),
                                        oracle.Matrix(rowptr=rb, colidx=cb, shape=shapeB),
                                        flags, s_max)
            self.m, self.d, self.n = shapeA[0], shapeA[1], shapeB[1]

    def close(self):
        self.ctx.close()
