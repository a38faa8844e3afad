"""Diamond sampling for approximate Maximum All-pairs Dot-product search on
GB300 (sm_103a): a thin ctypes binding over the C ABI of ``libmad.so``.

Every function here has the name of the C entry point it calls (see
``include/mad.h``) and only marshals arguments: torch supplies device memory
and streams, the library's CUDA kernels do all the work.  Importing this
package fails loudly when ``libmad.so`` has not been built; there is no CPU
fallback.

Paper: Ballard, Kolda, Pinar, Seshadhri, arXiv:1506.03872 (Alg. 2, Alg. 3).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmad.so")

MAD_OK, MAD_ERR_ARG, MAD_ERR_OOM, MAD_ERR_CUDA, MAD_ERR_OVERFLOW = 0, 1, 2, 3, 4
MAD_ERR_EMPTY, MAD_ERR_HASH_FULL, MAD_ERR_STATE, MAD_ERR_UNSUPPORTED = 5, 6, 7, 8
MAD_DENSE_ROWMAJOR, MAD_CSR = 0, 1
MAD_F32, MAD_F64, MAD_BINARY = 0, 1, 2
MAD_NONNEG, MAD_GRAM, MAD_EXCLUDE_DIAG, MAD_SQUARE_SYM, MAD_WEDGE, MAD_ALIAS = 1, 2, 4, 8, 16, 32
TABLES = {"T1": 0, "T2": 1, "TA": 2, "TB": 3, "na": 4, "nb": 5, "r": 6, "TK": 7, "TAc": 8,
          "nac": 9}
# Alias families (MAD_ALIAS): <family>al entries (two int64 per entry:
# threshold, alias), <family>as segment totals, <family>ar row totals.
for _q, _f in enumerate(("T1", "T2", "TA", "TB")):
    TABLES[_f + "al"], TABLES[_f + "as"], TABLES[_f + "ar"] = 10 + 3 * _q, 11 + 3 * _q, 12 + 3 * _q

# Every symbol include/mad.h declares.
EXPORTS = (
    "mad_create", "mad_destroy", "mad_strerror", "mad_set_hash_capacity", "mad_build_tables",
    "mad_sample", "mad_reset_hash", "mad_topk", "mad_rescore", "mad_stats", "mad_debug_draws",
    "mad_debug_draws_list", "mad_debug_set_hash_layout", "mad_export_x", "mad_export_table", "mad_rescore_noalloc",
    "mad_dense_topt", "mad_debug_dense_product", "mad_set_phase_events", "mad_mips_items",
    "mad_mips_plan", "mad_mips_run", "mad_budget_features", "mad_mlp_train", "mad_mlp_predict",
    "mad_pipeline_plan", "mad_pipeline_run", "mad_pipeline_status", "mad_sparse_topt",
    "mad_probe_gather", "mad_probe_atomics", "mad_export_x_by_owner", "mad_accumulate",
    "mad_select_pairs", "mad_mips_config",
)
MAD_BUDGET_FEATURES = 12
MAD_MLP_HIDDEN = 64


def mlp_params(f: int) -> int:
    """Parameter count of the budget perceptron for f features."""
    return MAD_MLP_HIDDEN * f + 3 * MAD_MLP_HIDDEN + MAD_MLP_HIDDEN * MAD_MLP_HIDDEN + 1
MAD_NOALLOC_MAX_CANDIDATES = 16384


class mad_matrix(ctypes.Structure):
    _fields_ = [("fmt", ctypes.c_int32), ("dt", ctypes.c_int32), ("rows", ctypes.c_int64),
                ("cols", ctypes.c_int64), ("ld", ctypes.c_int64), ("values", ctypes.c_void_p),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p)]


class mad_pair(ctypes.Structure):
    _fields_ = [("i", ctypes.c_uint32), ("j", ctypes.c_uint32), ("x", ctypes.c_int64),
                ("c", ctypes.c_double)]


class mad_stats_t(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_double), ("t1_total", ctypes.c_uint64), ("e1", ctypes.c_int32),
                ("f", ctypes.c_int32), ("sampled", ctypes.c_uint64),
                ("inserted", ctypes.c_uint64), ("diag_skipped", ctypes.c_uint64),
                ("distinct", ctypes.c_uint64), ("positive", ctypes.c_uint64),
                ("hash_capacity", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("integer_mode", ctypes.c_uint32), ("device_error", ctypes.c_uint32)]


class MadError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {mad_strerror(status)} (status {status})")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """The loaded ``libmad.so``; raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, u64, u32, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        L.mad_create.argtypes = [ctypes.POINTER(P), u32]
        L.mad_destroy.argtypes = [P]
        L.mad_destroy.restype = None
        L.mad_strerror.argtypes = [i32]
        L.mad_strerror.restype = ctypes.c_char_p
        L.mad_set_hash_capacity.argtypes = [P, u64]
        L.mad_set_phase_events.argtypes = [P, ctypes.POINTER(P), u32]
        L.mad_mips_items.argtypes = [P, ctypes.POINTER(mad_matrix), u64, P]
        L.mad_mips_plan.argtypes = [P, u32, ctypes.POINTER(u64), u32, u32, P]
        L.mad_mips_config.argtypes = [P, u32, u32, u32, u32]
        L.mad_mips_run.argtypes = [P, ctypes.POINTER(mad_matrix), u64, P, P, P, P]
        L.mad_budget_features.argtypes = [P, P, P]
        L.mad_mlp_train.argtypes = [P, P, P, P, u32, u32, u32, ctypes.c_float, ctypes.c_float, P,
                                    P]
        L.mad_mlp_predict.argtypes = [P, P, u32, u32, P, P]
        L.mad_build_tables.argtypes = [P, ctypes.POINTER(mad_matrix), ctypes.POINTER(mad_matrix),
                                       u64, P]
        L.mad_sample.argtypes = [P, u64, u64, u64, P]
        L.mad_pipeline_plan.argtypes = [P, ctypes.POINTER(mad_matrix), ctypes.POINTER(mad_matrix),
                                        u64, u32, u32, P]
        L.mad_pipeline_run.argtypes = [P, u64, P, P, P, P]
        L.mad_pipeline_status.argtypes = [P, P]
        L.mad_reset_hash.argtypes = [P, P]
        L.mad_topk.argtypes = [P, u32, P, ctypes.POINTER(u32), P]
        L.mad_rescore.argtypes = [P, P, u32, u32, P, ctypes.POINTER(u32), P]
        L.mad_stats.argtypes = [P, ctypes.POINTER(mad_stats_t)]
        L.mad_rescore_noalloc.argtypes = [ctypes.POINTER(mad_matrix), ctypes.POINTER(mad_matrix),
                                          P, u32, u32, P, ctypes.POINTER(u32), P]
        L.mad_dense_topt.argtypes = [P, ctypes.POINTER(mad_matrix), ctypes.POINTER(mad_matrix), u32,
                                     u32, P, ctypes.POINTER(u32), P]
        L.mad_sparse_topt.argtypes = [P, ctypes.POINTER(mad_matrix), ctypes.POINTER(mad_matrix),
                                      u32, u32, P, ctypes.POINTER(u32), P]
        L.mad_export_x_by_owner.argtypes = [P, u32, P, P, u64, P, P]
        L.mad_accumulate.argtypes = [P, P, P, u64, P]
        L.mad_select_pairs.argtypes = [P, P, u64, u32, P, ctypes.POINTER(u32), P]
        L.mad_probe_gather.argtypes = [P, u64, u64, u64, P, P]
        L.mad_probe_atomics.argtypes = [P, u64, u64, u32, u64, P, P]
        L.mad_debug_dense_product.argtypes = [P, ctypes.POINTER(mad_matrix),
                                              ctypes.POINTER(mad_matrix), P, P]
        L.mad_debug_draws.argtypes = [P, u64, u64, u64, P, P, P, P, P, P]
        L.mad_debug_draws_list.argtypes = [P, u64, P, u64, P, P, P, P, P, P]
        L.mad_debug_set_hash_layout.argtypes = [P, ctypes.c_float, u64]
        L.mad_export_x.argtypes = [P, P, P, u64, ctypes.POINTER(u64), P]
        L.mad_export_table.argtypes = [P, i32, P, u64, ctypes.POINTER(u64), P]
        for name in EXPORTS:
            if name not in ("mad_destroy", "mad_strerror"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != MAD_OK:
        raise MadError(status, where)


def _stream(stream) -> ctypes.c_void_p:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


# ---------------------------------------------------------------------------
# Matrix descriptors (torch tensors on the GPU)
# ---------------------------------------------------------------------------
def dense(t) -> mad_matrix:
    """A dense row-major float32/float64 CUDA tensor."""
    import torch
    if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("dense matrices are 2-D CUDA tensors with unit column stride")
    dt = {torch.float32: MAD_F32, torch.float64: MAD_F64}[t.dtype]
    return mad_matrix(MAD_DENSE_ROWMAJOR, dt, t.shape[0], t.shape[1], t.stride(0), t.data_ptr(),
                      None, None)


def csr(rowptr, colidx, shape) -> mad_matrix:
    """A 0/1 CSR matrix: int64 rowptr, int32 colidx (CUDA tensors)."""
    import torch
    if rowptr.dtype != torch.int64 or colidx.dtype != torch.int32:
        raise ValueError("CSR needs int64 rowptr and int32 colidx")
    return mad_matrix(MAD_CSR, MAD_BINARY, shape[0], shape[1], 0, None, rowptr.data_ptr(),
                      colidx.data_ptr())


# ---------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# ---------------------------------------------------------------------------
def mad_strerror(status: int) -> str:
    return lib().mad_strerror(status).decode()


def mad_create(flags: int = 0) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().mad_create(ctypes.byref(ctx), flags), "mad_create")
    return ctx


def mad_destroy(ctx) -> None:
    if ctx:
        lib().mad_destroy(ctx)


def mad_set_hash_capacity(ctx, slots: int) -> None:
    _check(lib().mad_set_hash_capacity(ctx, slots), "mad_set_hash_capacity")


def mad_set_phase_events(ctx, events) -> None:
    """Record the given torch.cuda.Event objects at the sampling phase
    boundaries of later mad_sample calls (see mad.h); [] stops."""
    handles = []
    for ev in events:
        if not ev.cuda_event:
            ev.record()   # torch creates the CUDA event lazily
        handles.append(ev.cuda_event)
    arr = (ctypes.c_void_p * max(1, len(handles)))(*handles)
    _check(lib().mad_set_phase_events(ctx, arr, len(handles)), "mad_set_phase_events")


def mad_build_tables(ctx, A: mad_matrix, B: mad_matrix, s_max: int, stream=None) -> None:
    _check(lib().mad_build_tables(ctx, ctypes.byref(A), ctypes.byref(B), s_max, _stream(stream)),
           "mad_build_tables")


def mad_sample(ctx, s: int, seed: int, first_diamond: int = 0, stream=None) -> None:
    _check(lib().mad_sample(ctx, s, seed, first_diamond, _stream(stream)), "mad_sample")


def mad_reset_hash(ctx, stream=None) -> None:
    _check(lib().mad_reset_hash(ctx, _stream(stream)), "mad_reset_hash")


def new_pairs(count: int):
    """Device buffer for ``count`` mad_pair records (24 bytes each)."""
    import torch
    return torch.empty((max(count, 1), 3), dtype=torch.int64, device="cuda")


def mad_topk(ctx, tprime: int, out=None, stream=None):
    """Omega_t' as a (tprime, 3) int64 CUDA tensor of mad_pair records and its count."""
    if out is None:
        out = new_pairs(tprime)
    n = ctypes.c_uint32(0)
    _check(lib().mad_topk(ctx, tprime, _ptr(out), ctypes.byref(n), _stream(stream)), "mad_topk")
    return out, n.value


def mad_rescore(ctx, cand, ncand: int, t: int, out=None, stream=None):
    """Omega_t from ``ncand`` candidate mad_pair records (CUDA tensor)."""
    if out is None:
        out = new_pairs(t)
    n = ctypes.c_uint32(0)
    _check(lib().mad_rescore(ctx, _ptr(cand), ncand, t, _ptr(out), ctypes.byref(n),
                             _stream(stream)), "mad_rescore")
    return out, n.value


def mad_pipeline_plan(ctx, A: mad_matrix, B: mad_matrix, s: int, tprime: int, t: int,
                      stream=None) -> None:
    """Fix the inputs (both dense, or both 0/1 CSR), the budget s and
    t <= t' of the fused pass and allocate everything it uses
    (synchronises)."""
    _check(lib().mad_pipeline_plan(ctx, ctypes.byref(A), ctypes.byref(B), s, tprime, t,
                                   _stream(stream)), "mad_pipeline_plan")


def mad_pipeline_run(ctx, seed: int, out, counts, cand=None, stream=None) -> None:
    """One fused pass (asynchronous; capturable in a CUDA graph).  out: t
    pairs; counts: two uint32 on the device (an int32 CUDA tensor): the
    candidate and result counts; cand: optional t' pairs receiving
    Omega_t'."""
    _check(lib().mad_pipeline_run(ctx, seed, _ptr(out), _ptr(counts),
                                  _ptr(cand) if cand is not None else None, _stream(stream)),
           "mad_pipeline_run")


def mad_pipeline_status(ctx, stream=None) -> None:
    """Wait for the last fused pass and raise MadError on a device error."""
    _check(lib().mad_pipeline_status(ctx, _stream(stream)), "mad_pipeline_status")


def mad_rescore_noalloc(A: mad_matrix, B: mad_matrix, cand, ncand: int, t: int, out=None,
                        stream=None):
    """mad_rescore without device allocation inside the library (the caller
    owns every buffer).  For callers that cannot allocate GPU memory; at most
    MAD_NOALLOC_MAX_CANDIDATES candidates per call."""
    if out is None:
        out = new_pairs(t)
    n = ctypes.c_uint32(0)
    _check(lib().mad_rescore_noalloc(ctypes.byref(A), ctypes.byref(B), _ptr(cand), ncand, t,
                                     _ptr(out), ctypes.byref(n), _stream(stream)),
           "mad_rescore_noalloc")
    return out, n.value


def mad_dense_topt(ctx, A: mad_matrix, B: mad_matrix, t: int, rescore: int = 0, out=None,
                   stream=None):
    """Top-t of |A B| by the BF16 tensor-core comparator (Sec. 4.3); the
    `rescore` largest BF16 products (0: 8t) are rescored in FP32."""
    if out is None:
        out = new_pairs(t)
    n = ctypes.c_uint32(0)
    _check(lib().mad_dense_topt(ctx, ctypes.byref(A), ctypes.byref(B), t, rescore, _ptr(out),
                                ctypes.byref(n), _stream(stream)), "mad_dense_topt")
    return out, n.value


SPARSE_NO_BOUND = 1


def mad_sparse_topt(ctx, A: mad_matrix, B: mad_matrix, t: int, options: int = 0, out=None,
                    stream=None):
    """Exact top-t counts of a 0/1 product by the sparse comparator
    (Sec. 4.3); options SPARSE_NO_BOUND processes every row and column."""
    if out is None:
        out = new_pairs(t)
    n = ctypes.c_uint32(0)
    _check(lib().mad_sparse_topt(ctx, ctypes.byref(A), ctypes.byref(B), t, options, _ptr(out),
                                 ctypes.byref(n), _stream(stream)), "mad_sparse_topt")
    return out, n.value


def mad_export_x_by_owner(ctx, world: int, cap: int, stream=None):
    """X's keys and values grouped by owner rank: (keys, vals, offsets) with
    owner o's entries at [offsets[o], offsets[o + 1]) (device int64 tensors;
    keys are the uint64 keys bit for bit)."""
    import numpy as np
    import torch
    while True:
        keys = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
        vals = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
        off = np.zeros(world + 1, dtype=np.uint64)
        _check(lib().mad_export_x_by_owner(ctx, world, _ptr(keys), _ptr(vals), cap,
                                           off.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
               "mad_export_x_by_owner")
        if int(off[world]) <= cap:
            return keys[:int(off[world])], vals[:int(off[world])], off.astype(np.int64)
        cap = int(off[world])


def mad_accumulate(ctx, keys, vals, stream=None) -> None:
    """Add (key, value) pairs (device int64 tensors) to X."""
    _check(lib().mad_accumulate(ctx, _ptr(keys), _ptr(vals), keys.numel(), _stream(stream)),
           "mad_accumulate")


def mad_select_pairs(ctx, pairs, n: int, K: int, out=None, stream=None):
    """The K pairs with the largest x > 0 by (x desc, key asc), copied whole."""
    if out is None:
        out = new_pairs(K)
    cnt = ctypes.c_uint32(0)
    _check(lib().mad_select_pairs(ctx, _ptr(pairs), n, K, _ptr(out), ctypes.byref(cnt),
                                  _stream(stream)), "mad_select_pairs")
    return out, cnt.value


def mad_probe_gather(table, count: int, seed: int = 1, sink=None, stream=None) -> None:
    """`count` random 32-byte-sector loads from the device tensor `table`
    (asynchronous; time with events)."""
    sink = table if sink is None else sink
    _check(lib().mad_probe_gather(_ptr(table), table.numel() * table.element_size(), count, seed,
                                  _ptr(sink), _stream(stream)), "mad_probe_gather")


def mad_probe_atomics(table, count: int, mode: int = 0, seed: int = 1, sink=None,
                      stream=None) -> None:
    """`count` random 64-bit atomics on the device tensor `table`: mode 0
    add, mode 1 compare-and-swap (asynchronous; time with events)."""
    sink = table if sink is None else sink
    _check(lib().mad_probe_atomics(_ptr(table), table.numel() * table.element_size(), count, mode,
                                   seed, _ptr(sink), _stream(stream)), "mad_probe_atomics")


def mad_mips_items(ctx, B: mad_matrix, s_max: int, stream=None) -> None:
    """Item-side tables for batched queries (B: d x n dense F32)."""
    _check(lib().mad_mips_items(ctx, ctypes.byref(B), s_max, _stream(stream)), "mad_mips_items")


def mad_mips_config(ctx, region_lg: int = 0, chunk_mult: int = 0, blocks_per_sm: int = 0,
                    select_threads: int = 0) -> None:
    """Launch shape of the next batch plan and run (0: the default)."""
    _check(lib().mad_mips_config(ctx, region_lg, chunk_mult, blocks_per_sm, select_threads),
           "mad_mips_config")


def mad_mips_plan(ctx, s_per_query, tprime: int, t: int, stream=None) -> None:
    """Batch shape: one budget per query (host integers), t' and t."""
    import numpy as np
    s = np.ascontiguousarray(np.asarray(s_per_query, dtype=np.uint64))
    _check(lib().mad_mips_plan(ctx, len(s), s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               tprime, t, _stream(stream)), "mad_mips_plan")


def mad_mips_run(ctx, Q: mad_matrix, seed: int, out, n_out, cand=None, stream=None) -> None:
    """One batch (asynchronous; capturable in a CUDA graph).  out: nq * t
    pairs, n_out: nq uint32 (an int32 CUDA tensor), cand: optional nq * t'
    pairs receiving each query's top-t' candidates."""
    _check(lib().mad_mips_run(ctx, ctypes.byref(Q), seed, _ptr(out), _ptr(n_out),
                              _ptr(cand) if cand is not None else None, _stream(stream)),
           "mad_mips_run")


def mad_budget_features(ctx, stream=None):
    """The MAD_BUDGET_FEATURES statistics of the built instance (numpy)."""
    import numpy as np
    out = np.zeros(MAD_BUDGET_FEATURES, dtype=np.float32)
    _check(lib().mad_budget_features(ctx, out.ctypes.data_as(ctypes.c_void_p), _stream(stream)),
           "mad_budget_features")
    return out


def mad_mlp_train(ctx, params, X, y, epochs: int, lr: float, quantile: float, loss=None,
                  stream=None) -> None:
    """Full-batch Adam on the budget perceptron (CUDA float32 tensors:
    params (mlp_params(f),), X (n, f), y (n,), loss (epochs,) or None)."""
    n, f = X.shape
    _check(lib().mad_mlp_train(ctx, _ptr(params), _ptr(X), _ptr(y), n, f, epochs, lr, quantile,
                               _ptr(loss), _stream(stream)), "mad_mlp_train")


def mad_mlp_predict(params, X, y=None, stream=None):
    """Network outputs for the rows of X (CUDA float32 (n, f))."""
    import torch
    n, f = X.shape
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device=X.device)
    _check(lib().mad_mlp_predict(_ptr(params), _ptr(X), n, f, _ptr(y), _stream(stream)),
           "mad_mlp_predict")
    return y


def mad_debug_dense_product(ctx, A: mad_matrix, B: mad_matrix, stream=None):
    """The comparator's BF16 product A B as an FP32 (m, n) CUDA tensor."""
    import torch
    c = torch.empty((A.rows, B.cols), dtype=torch.float32, device="cuda")
    _check(lib().mad_debug_dense_product(ctx, ctypes.byref(A), ctypes.byref(B), _ptr(c),
                                         _stream(stream)), "mad_debug_dense_product")
    return c


def mad_stats(ctx) -> dict:
    st = mad_stats_t()
    _check(lib().mad_stats(ctx, ctypes.byref(st)), "mad_stats")
    return {name: getattr(st, name) for name, _ in mad_stats_t._fields_}


def mad_debug_draws(ctx, seed: int, first: int, count: int, stream=None):
    import torch
    outs = [torch.empty(max(count, 1), dtype=torch.int32, device="cuda") for _ in range(4)]
    v = torch.empty(max(count, 1), dtype=torch.int64, device="cuda")
    _check(lib().mad_debug_draws(ctx, seed, first, count, *[_ptr(o) for o in outs], _ptr(v),
                                 _stream(stream)), "mad_debug_draws")
    return tuple(o[:count] for o in outs) + (v[:count],)


def mad_debug_set_hash_layout(ctx, region_factor: float, overflow_slots: int = 0) -> None:
    _check(lib().mad_debug_set_hash_layout(ctx, region_factor, overflow_slots),
           "mad_debug_set_hash_layout")


def mad_debug_draws_list(ctx, seed: int, ells, stream=None):
    import torch
    count = ells.numel()
    outs = [torch.empty(max(count, 1), dtype=torch.int32, device="cuda") for _ in range(4)]
    v = torch.empty(max(count, 1), dtype=torch.int64, device="cuda")
    _check(lib().mad_debug_draws_list(ctx, seed, _ptr(ells), count, *[_ptr(o) for o in outs],
                                      _ptr(v), _stream(stream)), "mad_debug_draws_list")
    return tuple(o[:count] for o in outs) + (v[:count],)


def mad_export_x(ctx, cap: int, stream=None):
    import torch
    keys = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    vals = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    n = ctypes.c_uint64(0)
    _check(lib().mad_export_x(ctx, _ptr(keys), _ptr(vals), cap, ctypes.byref(n), _stream(stream)),
           "mad_export_x")
    cnt = min(n.value, cap)
    return keys[:cnt], vals[:cnt], n.value


def mad_export_table(ctx, name: str, stream=None):
    import torch
    which = TABLES[name]
    n = ctypes.c_uint64(0)
    _check(lib().mad_export_table(ctx, which, None, 0, ctypes.byref(n), _stream(stream)),
           "mad_export_table")
    alias = name[-2:] in ("al", "as", "ar")
    dt = torch.int64 if name in ("T1", "TK") or alias else (
        torch.float32 if name in ("na", "nb", "r", "nac") else torch.int32)
    per = 2 if name.endswith("al") else 1   # alias entries: 16 bytes
    out = torch.empty(max(per * n.value, 1), dtype=dt, device="cuda")
    _check(lib().mad_export_table(ctx, which, _ptr(out), n.value, ctypes.byref(n),
                                  _stream(stream)), "mad_export_table")
    return out[:per * n.value]


# ---------------------------------------------------------------------------
# Helpers for reading results on the host
# ---------------------------------------------------------------------------
def decode_pairs(out, n: int) -> Tuple[np.ndarray, np.ndarray, np.ndarray, np.ndarray]:
    """(i, j, x, c) numpy arrays from the first ``n`` mad_pair records."""
    raw = out[:n].cpu().numpy() if hasattr(out, "cpu") else np.asarray(out)[:n]
    raw = np.ascontiguousarray(raw, dtype=np.int64)
    ij = raw[:, 0].view(np.uint64)
    i = (ij & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    j = (ij >> np.uint64(32)).astype(np.uint32)
    return i, j, raw[:, 1].copy(), raw[:, 2].copy().view(np.float64)


def encode_pairs(i, j, x=None):
    """mad_pair records (CUDA int64 tensor) from host index arrays."""
    import torch
    i = np.asarray(i, dtype=np.uint64)
    j = np.asarray(j, dtype=np.uint64)
    raw = np.zeros((len(i), 3), dtype=np.int64)
    raw[:, 0] = (i | (j << np.uint64(32))).view(np.int64)
    if x is not None:
        raw[:, 1] = np.asarray(x, dtype=np.int64)
    return torch.from_numpy(raw).cuda()


def keys_of(i, j) -> np.ndarray:
    return (np.asarray(i, np.uint64) << np.uint64(32)) | np.asarray(j, np.uint64)


class Context:
    """RAII holder of a mad_ctx plus the input tensors it reads."""

    def __init__(self, flags: int = 0):
        self.ctx = mad_create(flags)
        self.flags = flags
        self._inputs = ()

    def build(self, A: mad_matrix, B: mad_matrix, s_max: int, keep=(), stream=None):
        self._inputs = keep
        mad_build_tables(self.ctx, A, B, s_max, stream)

    def close(self):
        if self.ctx:
            mad_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
