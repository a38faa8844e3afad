"""CPU oracle for diamond sampling (arXiv:1506.03872, Alg. 2 and Alg. 3).

Test infrastructure only.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` load it; the library under
``paper_1506_03872_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``mad_oracle.cpp`` (plain C++17, single thread); this
module compiles it with g++ and wraps it with ctypes.  Inputs are numpy
arrays; every function mirrors one step of the paper:

* ``Oracle(A, B, flags, s_max)``  -- weights and sampling tables (Alg. 2,
  weight line; Sec. 4.2 cumulative tables).
* ``draw`` / ``draw_list``          -- the per-diamond draws (Alg. 2 loop).
* ``sample``                        -- accumulate x_ij (Alg. 2 loop body).
* ``topk``                          -- Omega_t' (Alg. 3, first step).
* ``rescore``                       -- exact dot products (Alg. 3).
* ``topt``                          -- Omega_t (Alg. 3, last step).
* ``bruteforce``                    -- exact t-MAD ground truth (Defn. 1).
* ``sparse_exact``                  -- exact top t by the row-wise sparse
  product (the paper's exact computation, Sec. 4.3).
* ``enumerate``                     -- exact three-path law (Lemma 1).
* ``enumerate_wedges``              -- exact wedge law (the appendix's wedge
  sampling; Oracle(..., flags | WEDGE) draws wedges instead of diamonds).
* ``alias_table``                   -- the alias tables of Oracle(..., flags |
  ALIAS), whose draws take the same laws from alias tables (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mad_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

FMT_DENSE, FMT_CSR = 0, 1
DT_F32, DT_F64, DT_BINARY = 0, 1, 2
NONNEG, GRAM, EXCLUDE_DIAG, SQUARE_SYM, WEDGE, ALIAS = 1, 2, 4, 8, 16, 32
ALIAS_SEG = 1024
ALIAS_ENTRY = np.dtype([("t", np.uint64), ("a", np.uint32), ("pad", np.uint32)])
STATUS = {0: "ok", 1: "bad argument", 4: "overflow", 5: "empty", 8: "unsupported"}


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, IEEE FP32/FP64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
            "-fno-fast-math", "-o", tmp, _SRC,
        ])
        os.replace(tmp, _LIB)
    return _LIB


_lib: Optional[ctypes.CDLL] = None


def _L() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        u64, i64, u32, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
        lib.or_create.restype = P
        lib.or_create.argtypes = [i32, i32, i64, i64, i64, P, P, P,
                                  i32, i32, i64, i64, i64, P, P, P,
                                  u32, u64, ctypes.POINTER(ctypes.c_int)]
        lib.or_destroy.argtypes = [P]
        lib.or_table.restype = i64
        lib.or_table.argtypes = [P, i32, P]
        lib.or_scalars.argtypes = [P, P]
        lib.or_draw.argtypes = [P, u64, u64, u64, P, P, P, P, P]
        lib.or_draw_list.argtypes = [P, u64, u64, P, P, P, P, P, P]
        lib.or_sample.restype = i32
        lib.or_sample.argtypes = [P, u64, u64, u64]
        lib.or_reset.argtypes = [P]
        lib.or_x_export.restype = i64
        lib.or_x_export.argtypes = [P, P, P]
        lib.or_topk.restype = i64
        lib.or_topk.argtypes = [P, u64, P, P]
        lib.or_rescore.argtypes = [P, i64, P, P]
        lib.or_topt.restype = i64
        lib.or_topt.argtypes = [i64, P, P, u64, P, P]
        lib.or_bruteforce.restype = i64
        lib.or_bruteforce.argtypes = [P, u64, P, P]
        lib.or_sparse_exact.restype = i64
        lib.or_sparse_exact.argtypes = [P, u64, P, P]
        lib.or_alias.restype = i64
        lib.or_alias.argtypes = [P, i32, i32, P]
        lib.or_enumerate_wedges.restype = i64
        lib.or_enumerate_wedges.argtypes = [P, i64, P, P, P, P, P]
        lib.or_enumerate.restype = i64
        lib.or_enumerate.argtypes = [P, i64, P, P, P, P, P, P]
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_diamond_uniforms.argtypes = [u64, u64, u32, P]
        _lib = lib
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _L().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def diamond_uniforms(seed: int, ell: int, instance: int = 0) -> np.ndarray:
    """The four 64-bit uniforms (i, k, j, k') of diamond ``ell``."""
    out = np.zeros(4, dtype=np.uint64)
    _L().or_diamond_uniforms(ctypes.c_uint64(seed), ctypes.c_uint64(ell),
                             ctypes.c_uint32(instance), _p(out))
    return out


class Matrix:
    """Host matrix description: dense row-major (f32/f64) or 0/1 CSR."""

    def __init__(self, dense: Optional[np.ndarray] = None, rowptr=None, colidx=None,
                 shape=None):
        if dense is not None:
            self.fmt = FMT_DENSE
            self.values = np.ascontiguousarray(dense)
            if self.values.dtype == np.float64:
                self.dt = DT_F64
            elif self.values.dtype == np.float32:
                self.dt = DT_F32
            else:
                raise TypeError("dense matrices are float32 or float64")
            self.rows, self.cols = self.values.shape
            self.ld = self.cols
            self.rowptr = self.colidx = None
        else:
            self.fmt, self.dt = FMT_CSR, DT_BINARY
            self.rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
            self.colidx = np.ascontiguousarray(colidx, dtype=np.int32)
            self.rows, self.cols = shape
            self.ld = 0
            self.values = None


class Oracle:
    def __init__(self, A: Matrix, B: Matrix, flags: int = 0, s_max: int = 1 << 20):
        lib = _L()
        st = ctypes.c_int(0)
        self._keep = (A, B)
        self.h = lib.or_create(A.fmt, A.dt, A.rows, A.cols, A.ld, _p(A.values), _p(A.rowptr),
                               _p(A.colidx), B.fmt, B.dt, B.rows, B.cols, B.ld, _p(B.values),
                               _p(B.rowptr), _p(B.colidx), flags, s_max, ctypes.byref(st))
        self.status = st.value
        if not self.h:
            raise OracleError(self.status)
        self.m, self.d, self.n = A.rows, A.cols, B.cols
        self.flags = flags

    def __del__(self):
        if getattr(self, "h", None):
            _L().or_destroy(self.h)
            self.h = None

    # --- tables ---------------------------------------------------------
    _TABLES = {"T1": (0, np.uint64), "T2": (1, np.uint32), "TA": (2, np.uint32),
               "TB": (3, np.uint32), "na": (4, np.float32), "nb": (5, np.float32),
               "r": (6, np.float32), "srow": (7, np.float32), "TK": (8, np.uint64),
               "TAc": (9, np.uint32), "nac": (10, np.float32)}

    def table(self, name: str) -> np.ndarray:
        which, dt = self._TABLES[name]
        n = _L().or_table(self.h, which, None)
        out = np.zeros(n, dtype=dt)
        _L().or_table(self.h, which, _p(out))
        return out

    _ALIAS = {"T1": 0, "T2": 1, "TA": 2, "TB": 3}

    def alias_table(self, name: str):
        """(entries, segment totals, row totals) of the alias family `name`
        (T1, T2, TA, TB): entries has fields t, a; row r's segments' entries
        then its top-level entries."""
        fam = self._ALIAS[name]
        out = []
        for part, dt in ((0, ALIAS_ENTRY), (1, np.uint64), (2, np.uint64)):
            n = _L().or_alias(self.h, fam, part, None)
            if n < 0:
                raise ValueError("no alias tables (build with flags | ALIAS)")
            a = np.zeros(n, dtype=dt)
            _L().or_alias(self.h, fam, part, _p(a))
            out.append(a)
        return tuple(out)

    def scalars(self) -> dict:
        out = np.zeros(8, dtype=np.int64)
        _L().or_scalars(self.h, _p(out))
        names = ["E1", "F", "bumps", "T1_total", "sampled", "inserted", "diag_skipped", "x_size"]
        return {k: int(v) for k, v in zip(names, out)}

    # --- sampling -------------------------------------------------------
    def draw(self, seed: int, first: int, count: int):
        arrs = [np.zeros(count, np.uint32) for _ in range(4)] + [np.zeros(count, np.int64)]
        _L().or_draw(self.h, seed, first, count, *[_p(a) for a in arrs])
        return tuple(arrs)

    def draw_list(self, seed: int, ells: np.ndarray):
        ells = np.ascontiguousarray(ells, dtype=np.uint64)
        count = len(ells)
        arrs = [np.zeros(count, np.uint32) for _ in range(4)] + [np.zeros(count, np.int64)]
        _L().or_draw_list(self.h, seed, count, _p(ells), *[_p(a) for a in arrs])
        return tuple(arrs)

    def sample(self, s: int, seed: int, first: int = 0) -> int:
        return _L().or_sample(self.h, s, seed, first)

    def reset(self):
        _L().or_reset(self.h)

    def x(self):
        n = _L().or_x_export(self.h, None, None)
        keys = np.zeros(n, np.uint64)
        vals = np.zeros(n, np.int64)
        _L().or_x_export(self.h, _p(keys), _p(vals))
        return keys, vals

    def topk(self, tprime: int):
        keys = np.zeros(tprime, np.uint64)
        xs = np.zeros(tprime, np.int64)
        cnt = _L().or_topk(self.h, tprime, _p(keys), _p(xs))
        return keys[:cnt], xs[:cnt]

    def rescore(self, keys: np.ndarray) -> np.ndarray:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        c = np.zeros(len(keys), np.float64)
        _L().or_rescore(self.h, len(keys), _p(keys), _p(c))
        return c

    def bruteforce(self, t: int):
        keys = np.zeros(t, np.uint64)
        c = np.zeros(t, np.float64)
        cnt = _L().or_bruteforce(self.h, t, _p(keys), _p(c))
        return keys[:cnt], c[:cnt]

    def sparse_exact(self, t: int):
        """Exact top t by the row-wise sparse product (Sec. 4.3): every
        stored entry of C is a candidate, (|c| desc, key asc)."""
        keys = np.zeros(t, np.uint64)
        c = np.zeros(t, np.float64)
        cnt = _L().or_sparse_exact(self.h, t, _p(keys), _p(c))
        return keys[:cnt], c[:cnt]

    def enumerate(self, cap: int = 1 << 20):
        arrs = [np.zeros(cap, np.uint32) for _ in range(4)]
        prob = np.zeros(cap, np.float64)
        v = np.zeros(cap, np.int64)
        cnt = _L().or_enumerate(self.h, cap, *[_p(a) for a in arrs], _p(prob), _p(v))
        if cnt > cap:
            raise ValueError(f"{cnt} three-paths exceed cap {cap}")
        return tuple(a[:cnt] for a in arrs) + (prob[:cnt], v[:cnt])

    def enumerate_wedges(self, cap: int = 1 << 20):
        """Every wedge (i, k, j) with its probability and increment (wedge
        contexts only)."""
        arrs = [np.zeros(cap, np.uint32) for _ in range(3)]
        prob = np.zeros(cap, np.float64)
        v = np.zeros(cap, np.int64)
        cnt = _L().or_enumerate_wedges(self.h, cap, *[_p(a) for a in arrs], _p(prob), _p(v))
        if cnt < 0:
            raise ValueError("not a wedge oracle")
        if cnt > cap:
            raise ValueError(f"{cnt} wedges exceed cap {cap}")
        return tuple(a[:cnt] for a in arrs) + (prob[:cnt], v[:cnt])

    def run(self, s: int, seed: int, tprime: int, t: int):
        """Alg. 2 followed by Alg. 3: returns (keys, c) of Omega_t."""
        self.reset()
        st = self.sample(s, seed, 0)
        if st:
            raise OracleError(st)
        keys, _ = self.topk(tprime)
        c = self.rescore(keys)
        return topt(keys, c, t)


def topt(keys: np.ndarray, c: np.ndarray, t: int):
    """The t largest by (|c| desc, key asc) (Alg. 3, last step)."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    ok = np.zeros(t, np.uint64)
    oc = np.zeros(t, np.float64)
    cnt = _L().or_topt(len(keys), _p(keys), _p(c), t, _p(ok), _p(oc))
    return ok[:cnt], oc[:cnt]


class OracleError(RuntimeError):
    def __init__(self, status: int):
        super().__init__(f"oracle status {status}: {STATUS.get(status, '?')}")
        self.status = status
