// The C ABI declared in include/mad.h: argument checks, memory ownership,
// status codes and the order of the kernel launches.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "mad_internal.cuh"

namespace mad {

mad_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MAD_OK;
  if (e == cudaErrorMemoryAllocation) return MAD_ERR_OOM;
  return MAD_ERR_CUDA;
}

// Every device allocation of a context's pool goes through here.  Host-side
// fault injection for tests of the failure paths (no GPU fault involved):
// with MAD_FAULT=oom[:N] in the environment at mad_create, the context's
// N-th allocation (N = 1 without ":N") and every later one return
// MAD_ERR_OOM instead of allocating.
mad_status pool_malloc(mad_ctx* ctx, void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (ctx->fault_oom_at > 0 && ++ctx->allocs >= ctx->fault_oom_at) return MAD_ERR_OOM;
  const mad_status rs = cuda_status(cudaMallocFromPoolAsync(p, bytes, ctx->pool, st));
  if (rs != MAD_OK) *p = nullptr;
  return rs;
}

mad_status ensure_scratch(mad_ctx* ctx, size_t bytes, cudaStream_t st) {
  if (bytes <= ctx->scratch_bytes) return MAD_OK;
  if (ctx->scratch_fixed) return MAD_ERR_STATE;
  if (ctx->scratch) cudaFreeAsync(ctx->scratch, st);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  const size_t rounded = (bytes + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
  const mad_status rs = pool_malloc(ctx, &ctx->scratch, rounded, st);
  if (rs != MAD_OK) return rs;
  ctx->scratch_bytes = rounded;
  return MAD_OK;
}

}  // namespace mad

using namespace mad;

namespace {

int ceil_log2(uint64_t x) {
  int e = 0;
  while (e < 64 && (1ull << e) < x) ++e;
  return e;
}

template <typename T>
void free_async(T*& p, cudaStream_t st) {
  if (p) cudaFreeAsync((void*)p, st);
  p = nullptr;
}

void free_tables(mad_ctx* ctx, cudaStream_t st) {
  free_async(ctx->T1, st);
  free_async(ctx->T2, st);
  free_async(ctx->TA, st);
  free_async(ctx->TB, st);
  free_async(ctx->na, st);
  free_async(ctx->nb, st);
  free_async(ctx->r, st);
  free_async(ctx->r64, st);
  free_async(ctx->bt, st);
  free_async(ctx->hkeys, st);
  free_async(ctx->hvals, st);
  free_async(ctx->hreg, st);
  free_async(ctx->T2g_ptr, st);
  free_async(ctx->T2g, st);
  free_async(ctx->T2g_sh, st);
  free_async(ctx->bloom, st);
  free_async(ctx->T1g, st);
  free_async(ctx->TBg, st);
  free_async(ctx->TBg_sh, st);
  free_async(ctx->TK, st);
  free_async(ctx->TAc, st);
  free_async(ctx->nac, st);
  for (int f = 0; f < 4; ++f) {
    free_async(ctx->al[f], st);
    free_async(ctx->al_seg[f], st);
    free_async(ctx->al_row[f], st);
    ctx->al_nseg[f] = 0;
  }
  ctx->TK_shift = 0;
  ctx->tk_total = 0;
  free_async(ctx->rg_buf, st);
  ctx->rg_cap = 0;
  free_async(ctx->pipe_buf, st);
  free_async(ctx->pipe_scratch, st);
  ctx->pipe_scratch_bytes = 0;
  ctx->pipe = false;
  free_async(ctx->mips_s, st);
  free_async(ctx->mips_chunk_q, st);
  free_async(ctx->mips_chunk_l0, st);
  ctx->mips_items = false;
  ctx->mips_nq = 0;
  ctx->built = false;
  ctx->regioned = false;
}

template <typename T>
mad_status alloc(mad_ctx* ctx, T*& p, size_t count, cudaStream_t st) {
  if (count == 0) count = 1;
  void* q = nullptr;
  const mad_status rs = pool_malloc(ctx, &q, count * sizeof(T), st);
  p = (T*)q;
  return rs;
}


// Read the device scalars (synchronises the stream).
mad_status read_scalars(mad_ctx* ctx, DevScalars* hs, cudaStream_t st) {
  cudaMemcpyAsync(hs, ctx->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, st);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  ctx->device_error = hs->err;
  return MAD_OK;
}

bool valid_dense(const mad_matrix* M) {
  return M->fmt == MAD_DENSE_ROWMAJOR && (M->dt == MAD_F32 || M->dt == MAD_F64) && M->values &&
         M->ld >= M->cols && M->rows > 0 && M->cols > 0;
}

bool valid_csr(const mad_matrix* M) {
  return M->fmt == MAD_CSR && M->dt == MAD_BINARY && M->rowptr && M->colidx && M->rows > 0 &&
         M->cols > 0 && M->cols < (1ll << 31);
}

// Empty X: every slot up to the hash's extent.
mad_status clear_x_slots(mad_ctx* ctx, cudaStream_t st) {
  return clear_slots(ctx, nullptr, hash_extent(ctx), st);
}

mad_status clear_hash(mad_ctx* ctx, cudaStream_t st) {
  mad_status rs = clear_x_slots(ctx, st);
  if (rs != MAD_OK) return rs;
  cudaMemsetAsync(&ctx->sc->inserted, 0, 5 * sizeof(unsigned long long), st);
  ctx->sampled = 0;
  return cuda_status(cudaGetLastError());
}

}  // namespace

namespace mad {

mad_status read_device_scalars(mad_ctx* ctx, DevScalars* hs, cudaStream_t st) {
  return read_scalars(ctx, hs, st);
}

mad_status clear_x(mad_ctx* ctx, cudaStream_t st) { return clear_x_slots(ctx, st); }

mad_status device_error_status(uint32_t err) {
  if (err & DERR_HASH_FULL) return MAD_ERR_HASH_FULL;
  if (err & DERR_OVERFLOW) return MAD_ERR_OVERFLOW;
  if (err & (DERR_SEARCH | DERR_SELECT)) return MAD_ERR_STATE;
  if (err & DERR_EMPTY) return MAD_ERR_EMPTY;
  return MAD_OK;
}

// Shapes, formats and flags accepted by the table build.
mad_status check_inputs(const mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                        uint64_t s_max, bool* dense_out) {
  if (!A || !B || s_max == 0 || s_max > (1ull << 60)) return MAD_ERR_ARG;
  if (B->rows != A->cols) return MAD_ERR_ARG;
  if (A->rows >= (1ll << 32) - 1 || B->cols >= (1ll << 32) - 1) return MAD_ERR_ARG;
  if ((ctx->flags & MAD_GRAM) && A->rows != B->cols) return MAD_ERR_ARG;  // B = A^T
  const bool dense = A->fmt == MAD_DENSE_ROWMAJOR && B->fmt == MAD_DENSE_ROWMAJOR;
  const bool csr = A->fmt == MAD_CSR && B->fmt == MAD_CSR;
  if (dense) {
    if (!valid_dense(A) || !valid_dense(B)) return MAD_ERR_ARG;
    if (A->cols > 1024) return MAD_ERR_UNSUPPORTED;
  } else if (csr) {
    if (!valid_csr(A) || !valid_csr(B)) return MAD_ERR_ARG;
  } else {
    return MAD_ERR_UNSUPPORTED;
  }
  // The squared symmetric update (Sec. 3.2.3) needs B = A^T = A: Gram
  // inputs, and square ones when dense (the caller guarantees symmetry).
  if ((ctx->flags & MAD_SQUARE_SYM) &&
      (!(ctx->flags & MAD_GRAM) || (!csr && A->rows != A->cols)))
    return MAD_ERR_UNSUPPORTED;
  // Alias tables: dense float inputs, tables of at most 2^20 entries.
  if ((ctx->flags & MAD_ALIAS) &&
      (!dense || A->rows > kAliasSeg * kAliasSeg || B->cols > kAliasSeg * kAliasSeg))
    return MAD_ERR_UNSUPPORTED;
  *dense_out = dense;
  return MAD_OK;
}

// Frees the previous tables and allocates the new ones: every table whose
// size follows from the shapes (for 0/1 inputs, after reading nnz), the
// guides of T1 and of the dense TB rows at their largest size, and the
// hash when its capacity is known before sampling (dense home regions sized
// for s_max, or an explicit capacity).
mad_status alloc_tables(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint64_t s_max,
                        bool dense, cudaStream_t st) {
  free_tables(ctx, st);
  ctx->A = *A;
  ctx->B = *B;
  ctx->dense = dense;
  ctx->integer = !dense;
  ctx->m = A->rows;
  ctx->d = A->cols;
  ctx->n = B->cols;
  ctx->s_max = s_max;
  ctx->sampled = 0;
  mad_status rs = MAD_OK;
  if (!dense) {
    int64_t na = 0, nb = 0;
    cudaMemcpyAsync(&na, A->rowptr + A->rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&nb, B->rowptr + B->rows, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    rs = cuda_status(cudaStreamSynchronize(st));
    if (rs != MAD_OK) return rs;
    if (na <= 0 || nb <= 0) return MAD_ERR_EMPTY;
    ctx->nnz_a = (uint64_t)na;
    ctx->nnz_b = (uint64_t)nb;
    if ((rs = alloc(ctx, ctx->T2, ctx->nnz_a, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->r64, (size_t)ctx->m, st)) != MAD_OK) return rs;
  } else {
    ctx->nnz_a = (uint64_t)(ctx->m * ctx->d);
    ctx->nnz_b = (uint64_t)(ctx->d * ctx->n);
    const size_t eb = B->dt == MAD_F64 ? 8 : 4;
    if ((rs = alloc(ctx, ctx->T2, ctx->nnz_a, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->TA, ctx->nnz_a, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->TB, ctx->nnz_b, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->na, (size_t)ctx->m, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->r, (size_t)ctx->m, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->nb, (size_t)ctx->d, st)) != MAD_OK) return rs;
    char* bt = nullptr;
    if ((rs = alloc(ctx, bt, (size_t)(ctx->n * ctx->d) * eb, st)) != MAD_OK) return rs;
    ctx->bt = bt;
    // Guides of the TB rows: the j search reads two guide entries and a
    // short window of its row.
    ctx->tbg_stride = ((int64_t)1 << tb_guide_width(ctx->n)) + 1;
    if ((rs = alloc(ctx, ctx->TBg_sh, (size_t)ctx->d, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->TBg, (size_t)(ctx->d * ctx->tbg_stride), st)) != MAD_OK) return rs;
  }
  if ((rs = alloc(ctx, ctx->T1, (size_t)ctx->m, st)) != MAD_OK) return rs;
  // Guide of T1: about m power-of-two buckets over [0, total).
  if ((rs = alloc(ctx, ctx->T1g, ((size_t)1 << t1_guide_width(ctx->m)) + 1, st)) != MAD_OK)
    return rs;
  // Dense inputs get a hash with per-row home regions (sized after T1);
  // 0/1 inputs a plain power-of-two table sized from a pilot run of the
  // sampler (their closure rate is unknown until sampled); an explicit
  // capacity is taken as given.
  // Wedge contexts add every wedge (no closure test): a plain table of at
  // least s_max / 0.6 slots.
  const bool wedge = (ctx->flags & MAD_WEDGE) != 0;
  ctx->regioned = dense && ctx->hcap_request == 0 && !wedge;
  uint64_t cap = ctx->hcap_request;
  if (!cap && wedge) cap = wedge_hash_slots(s_max);
  ctx->hov = 0;
  if (ctx->regioned) {
    ctx->hov = ctx->hov_request ? ctx->hov_request : hash_overflow_slots(s_max);
    cap = hash_region_bound((uint64_t)ctx->m, s_max) + ctx->hov;
    if ((rs = alloc(ctx, ctx->hreg, (size_t)ctx->m + 2, st)) != MAD_OK) return rs;
  }
  if (cap) {
    ctx->hcap = ctx->hcap_alloc = cap;
    if ((rs = alloc(ctx, ctx->hkeys, cap, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->hvals, cap, st)) != MAD_OK) return rs;
  }
  return MAD_OK;
}

// The dense table build, enqueued without any wait for the device: tables,
// home regions, guides, and (clear_x) an empty hash.
mad_status enqueue_dense_build(mad_ctx* ctx, cudaStream_t st, bool clear_x) {
  cudaMemsetAsync(ctx->sc, 0, sizeof(DevScalars), st);
  mad_status rs;
  const bool side = ctx->side && ctx->ev_fork && ctx->ev_fork2 && ctx->ev_join;
  if ((rs = build_tables_impl(ctx, st, side)) != MAD_OK) return rs;
  if (ctx->regioned && (rs = build_hash_regions(ctx, st)) != MAD_OK) return rs;
  if (!side && (rs = tb_guide_build(ctx, st)) != MAD_OK) return rs;
  if ((rs = t1_guide_fill(ctx, st)) != MAD_OK) return rs;
  if (clear_x && (rs = clear_x_slots(ctx, st)) != MAD_OK) return rs;
  if (side) cudaStreamWaitEvent(st, ctx->ev_join, 0);   // B^T and the TB guides
  return cuda_status(cudaGetLastError());
}

// Host mirrors of the device scalars after a dense build (synchronises).
mad_status finish_dense_build(mad_ctx* ctx, cudaStream_t st) {
  DevScalars hs;
  unsigned long long used = 0;
  if (ctx->regioned)
    cudaMemcpyAsync(&used, ctx->hreg + ctx->m, sizeof(used), cudaMemcpyDeviceToHost, st);
  mad_status rs = read_scalars(ctx, &hs, st);
  if (rs != MAD_OK) return rs;
  if (hs.err & DERR_OVERFLOW) return MAD_ERR_OVERFLOW;
  if ((hs.err & DERR_EMPTY) || hs.maxr_bits == 0u || hs.maxb_bits == 0u) return MAD_ERR_EMPTY;
  if (ctx->regioned) {
    if (used == 0 || used > ctx->hcap_alloc) return MAD_ERR_STATE;
    ctx->hcap = used;
  }
  ctx->f = hs.f_exp;
  ctx->e1 = hs.e1;
  ctx->t1g_sh = hs.t1g_sh;
  ctx->t1_total = hs.t1_total;
  return MAD_OK;
}


// Scratch of the dense table build: T1 chunk totals, then the home-region
// sizes and their scan.
size_t dense_build_scratch_bytes(const mad_ctx* ctx) {
  const uint64_t m = (uint64_t)ctx->m;
  const size_t chunks = (size_t)((m + 2047) / 2048) * sizeof(unsigned long long);
  const size_t regions = ((m * sizeof(unsigned long long) + 255) & ~(size_t)255) +
                         scan_partial_elems(m) * 8;
  return chunks > regions ? chunks : regions;
}

mad_status plan_dense_tables(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                             uint64_t s_max, cudaStream_t st) {
  bool dense = false;
  mad_status rs = check_inputs(ctx, A, B, s_max, &dense);
  if (rs != MAD_OK) return rs;
  if (!dense) return MAD_ERR_UNSUPPORTED;
  return alloc_tables(ctx, A, B, s_max, true, st);
}

}  // namespace mad

extern "C" {

mad_status mad_create(mad_ctx** out, uint32_t flags) {
  if (!out) return MAD_ERR_ARG;
  *out = nullptr;
  if (flags & ~(uint32_t)(MAD_NONNEG | MAD_GRAM | MAD_EXCLUDE_DIAG | MAD_SQUARE_SYM | MAD_WEDGE |
                          MAD_ALIAS))
    return MAD_ERR_ARG;
  if ((flags & MAD_WEDGE) && (flags & (MAD_SQUARE_SYM | MAD_ALIAS))) return MAD_ERR_ARG;
  mad_ctx* ctx = new (std::nothrow) mad_ctx();
  if (!ctx) return MAD_ERR_OOM;
  ctx->flags = flags;
  if (const char* f = std::getenv("MAD_FAULT")) {
    if (std::strncmp(f, "oom", 3) == 0) {
      ctx->fault_oom_at = 1;
      if (f[3] == ':') ctx->fault_oom_at = std::strtoll(f + 4, nullptr, 10);
      if (ctx->fault_oom_at < 1) ctx->fault_oom_at = 1;
    }
  }
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    e = cudaMemPoolCreate(&ctx->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->sc, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaMemset(ctx->sc, 0, sizeof(DevScalars));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork2, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->sc) cudaFree(ctx->sc);
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return cuda_status(e);
  }
  *out = ctx;
  return MAD_OK;
}

mad_status mad_set_phase_events(mad_ctx* ctx, void* const* events, uint32_t n) {
  if (!ctx || n > 4 || (n && !events)) return MAD_ERR_ARG;
  for (uint32_t q = 0; q < 4; ++q) ctx->phase_ev[q] = q < n ? (cudaEvent_t)events[q] : nullptr;
  ctx->n_phase_ev = n;
  return MAD_OK;
}

void mad_destroy(mad_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  free_tables(ctx, 0);
  if (ctx->scratch) cudaFreeAsync(ctx->scratch, 0);
  cudaStreamSynchronize(0);
  cudaFree(ctx->sc);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_fork2) cudaEventDestroy(ctx->ev_fork2);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  delete ctx;
}

const char* mad_strerror(mad_status s) {
  switch (s) {
    case MAD_OK: return "success";
    case MAD_ERR_ARG: return "invalid argument";
    case MAD_ERR_OOM: return "device out of memory";
    case MAD_ERR_CUDA: return "CUDA runtime error";
    case MAD_ERR_OVERFLOW: return "integer range exceeded (table total or diamonds beyond s_max)";
    case MAD_ERR_EMPTY: return "||W||_1 is zero: no three-path to sample";
    case MAD_ERR_HASH_FULL: return "hash probe limit exceeded (capacity too small)";
    case MAD_ERR_STATE: return "call out of order or inconsistent state";
    case MAD_ERR_UNSUPPORTED: return "unsupported input format";
  }
  return "unknown status";
}

mad_status mad_set_hash_capacity(mad_ctx* ctx, uint64_t slots) {
  if (!ctx) return MAD_ERR_ARG;
  if (slots != 0 && (slots < 1024 || (slots & (slots - 1)) != 0)) return MAD_ERR_ARG;
  ctx->hcap_request = slots;
  return MAD_OK;
}

mad_status mad_debug_set_hash_layout(mad_ctx* ctx, float region_factor, uint64_t overflow_slots) {
  if (!ctx) return MAD_ERR_ARG;
  if (!(region_factor > 0.0f && region_factor <= 1.5f)) return MAD_ERR_ARG;
  if (overflow_slots != 0 && (overflow_slots < 16 || (overflow_slots & (overflow_slots - 1)) != 0))
    return MAD_ERR_ARG;
  ctx->region_factor = region_factor;
  ctx->hov_request = overflow_slots;
  return MAD_OK;
}

// Wedge contexts: the wedge tables after the diamond tables, and the table
// scalars mad_stats reports (||w||_1 = TK's total / 2^EK in place of
// ||W||_1).
mad_status finish_wedge_build(mad_ctx* ctx, cudaStream_t st) {
  mad_status rs = build_wedge_tables(ctx, st);
  if (rs != MAD_OK) return rs;
  ctx->t1_total = ctx->tk_total;
  ctx->e1 = ctx->ek;
  return MAD_OK;
}

mad_status mad_build_tables(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                            uint64_t s_max, mad_stream stream) {
  if (!ctx) return MAD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  bool dense = false;
  mad_status rs = check_inputs(ctx, A, B, s_max, &dense);
  if (rs != MAD_OK) return rs;
  if ((rs = alloc_tables(ctx, A, B, s_max, dense, st)) != MAD_OK) return rs;
  const bool wedge = (ctx->flags & MAD_WEDGE) != 0;
  if (dense) {
    if ((rs = enqueue_dense_build(ctx, st)) != MAD_OK) return rs;
    if ((rs = finish_dense_build(ctx, st)) != MAD_OK) return rs;
    if (wedge && (rs = finish_wedge_build(ctx, st)) != MAD_OK) return rs;
    if ((ctx->flags & MAD_ALIAS) && (rs = build_alias_tables(ctx, st)) != MAD_OK) return rs;
    ctx->built = true;
    return MAD_OK;
  }
  const bool pilot = ctx->hcap_request == 0 && !wedge;
  cudaMemsetAsync(ctx->sc, 0, sizeof(DevScalars), st);
  if ((rs = build_tables_impl(ctx, st)) != MAD_OK) return rs;
  DevScalars hs;
  if ((rs = read_scalars(ctx, &hs, st)) != MAD_OK) return rs;
  if (hs.err & DERR_OVERFLOW) return MAD_ERR_OVERFLOW;
  if (hs.t1_total == 0) return MAD_ERR_EMPTY;
  // Guides of the long T2 rows (the 0/1 sampler's k search).
  if ((rs = alloc(ctx, ctx->T2g_ptr, (size_t)ctx->m + 1, st)) != MAD_OK) return rs;
  if ((rs = alloc(ctx, ctx->T2g_sh, (size_t)ctx->m, st)) != MAD_OK) return rs;
  if ((rs = t2_guide_offsets(ctx, st)) != MAD_OK) return rs;
  unsigned long long gtotal = 0;
  cudaMemcpyAsync(&gtotal, ctx->T2g_ptr + ctx->m, sizeof(gtotal), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  if ((rs = alloc(ctx, ctx->T2g, (size_t)gtotal, st)) != MAD_OK) return rs;
  ctx->t2g_total = gtotal;
  if (gtotal && (rs = t2_guide_fill(ctx, st)) != MAD_OK) return rs;
  // Closure filter: 16 bits per entry, a power of two of 64-bit words.
  const uint64_t nnz_c = (ctx->flags & MAD_GRAM) ? ctx->nnz_a : ctx->nnz_b;
  ctx->bloom_lg = 10;
  while (((1ull << ctx->bloom_lg) * 4ull) < nnz_c && ctx->bloom_lg < 40) ++ctx->bloom_lg;
  if ((rs = alloc(ctx, ctx->bloom, (size_t)1 << ctx->bloom_lg, st)) != MAD_OK) return rs;
  if ((rs = build_bloom(ctx, st)) != MAD_OK) return rs;
  ctx->f = 0;
  ctx->e1 = 0;
  ctx->t1_total = hs.t1_total;
  ctx->t1g_sh = hs.t1g_sh;
  if ((rs = t1_guide_fill(ctx, st)) != MAD_OK) return rs;
  if (pilot) {
    // Fraction of diamonds that add to X, from kPilot diamonds of a fixed
    // seed; the table holds s_max times that fraction plus six standard
    // deviations at load 1/16 (and never more than s_max / 0.6 slots).
    // Measured on GB300: scattered inserts into a table at load 0.46 took
    // 3.3x longer than at load 0.06 with the same number of probes.
    const uint64_t kPilot = 1ull << 20;
    uint64_t hits = 0;
    if ((rs = pilot_inserts(ctx, kPilot, &hits, st)) != MAD_OK) return rs;
    const double f = (double)hits / (double)kPilot;
    const double f_hi = f + 6.0 * std::sqrt(f * (1.0 - f) / (double)kPilot) + 8.0 / (double)kPilot;
    const double per = (ctx->flags & MAD_SQUARE_SYM) ? 2.0 : 1.0;  // inserts per diamond
    const double want = std::min(((double)s_max * std::min(f_hi, per) + 4096.0) * 16.0,
                                 per * (double)s_max / 0.6);
    uint64_t cap = 1024;
    while ((double)cap < want && cap < (1ull << 40)) cap <<= 1;
    ctx->hcap = ctx->hcap_alloc = cap;
    if ((rs = alloc(ctx, ctx->hkeys, cap, st)) != MAD_OK) return rs;
    if ((rs = alloc(ctx, ctx->hvals, cap, st)) != MAD_OK) return rs;
  }
  if ((rs = clear_hash(ctx, st)) != MAD_OK) return rs;
  if (wedge && (rs = finish_wedge_build(ctx, st)) != MAD_OK) return rs;
  ctx->built = true;
  return MAD_OK;
}

mad_status mad_sample(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first_diamond,
                      mad_stream stream) {
  if (!ctx) return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  if (s > ctx->s_max || ctx->sampled > ctx->s_max - s) return MAD_ERR_OVERFLOW;
  const mad_status rs = sample_impl(ctx, s, seed, first_diamond, (cudaStream_t)stream);
  if (rs == MAD_OK) ctx->sampled += s;
  return rs;
}

mad_status mad_reset_hash(mad_ctx* ctx, mad_stream stream) {
  if (!ctx) return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  return clear_hash(ctx, (cudaStream_t)stream);
}

mad_status mad_topk(mad_ctx* ctx, uint32_t tprime, mad_pair* out_dev, uint32_t* n_out_host,
                    mad_stream stream) {
  if (!ctx || !n_out_host || (tprime > 0 && !out_dev)) return MAD_ERR_ARG;
  *n_out_host = 0;
  if (!ctx->built) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  DevScalars hs;
  mad_status rs = read_scalars(ctx, &hs, st);
  if (rs != MAD_OK) return rs;
  if ((rs = device_error_status(hs.err)) != MAD_OK) return rs;
  uint64_t bound = hs.new_keys < ctx->hcap ? hs.new_keys : ctx->hcap;
  if (tprime == 0 || bound == 0) return MAD_OK;
  if ((rs = ensure_scratch(ctx, select_ws_bytes(bound, tprime), st)) != MAD_OK) return rs;
  const SelectWs ws = select_ws_carve(ctx->scratch, bound, tprime);
  uint64_t npos = 0, nsel = 0;
  if ((rs = select_from_hash(ctx, ws, tprime, &nsel, &npos, st)) != MAD_OK) return rs;
  ctx->positive = npos;
  ctx->distinct = hs.new_keys;
  if ((rs = items_to_pairs(ctx, ws.out, nsel, nullptr, nullptr, out_dev, st)) != MAD_OK) return rs;
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  *n_out_host = (uint32_t)nsel;
  return MAD_OK;
}

mad_status mad_rescore(mad_ctx* ctx, const mad_pair* cand_dev, uint32_t ncand, uint32_t t,
                       mad_pair* out_dev, uint32_t* n_out_host, mad_stream stream) {
  if (!ctx || !n_out_host || (ncand > 0 && !cand_dev) || (t > 0 && !out_dev)) return MAD_ERR_ARG;
  *n_out_host = 0;
  if (!ctx->built) return MAD_ERR_STATE;
  if (ncand == 0 || t == 0) return MAD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ws_bytes = select_ws_bytes(ncand, t);
  const size_t cv_off = (ws_bytes + 255) & ~(size_t)255;
  mad_status rs = ensure_scratch(ctx, cv_off + (size_t)ncand * sizeof(double), st);
  if (rs != MAD_OK) return rs;
  if ((rs = rescore_reserve(ctx, ncand, st)) != MAD_OK) return rs;
  const SelectWs ws = select_ws_carve(ctx->scratch, ncand, t);
  double* cvals = (double*)((char*)ctx->scratch + cv_off);
  if ((rs = rescore_items(ctx, cand_dev, ncand, ws.l0, cvals, st)) != MAD_OK) return rs;
  uint64_t nsel = 0;
  if ((rs = select_list(ctx, ws, ncand, t, 8, &nsel, st)) != MAD_OK) return rs;
  if ((rs = items_to_pairs(ctx, ws.out, nsel, cand_dev, cvals, out_dev, st)) != MAD_OK) return rs;
  DevScalars hs;
  if ((rs = read_scalars(ctx, &hs, st)) != MAD_OK) return rs;
  if ((rs = device_error_status(hs.err)) != MAD_OK) return rs;
  *n_out_host = (uint32_t)nsel;
  return MAD_OK;
}

mad_status mad_stats(mad_ctx* ctx, mad_stats_t* out) {
  if (!ctx || !out) return MAD_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  DevScalars hs;
  std::memset(&hs, 0, sizeof(hs));
  mad_status rs = cuda_status(cudaDeviceSynchronize());
  if (rs != MAD_OK) return rs;
  if ((rs = cuda_status(cudaMemcpy(&hs, ctx->sc, sizeof(hs), cudaMemcpyDeviceToHost))) != MAD_OK)
    return rs;
  ctx->device_error = hs.err;
  out->t1_total = ctx->t1_total;
  out->e1 = ctx->e1;
  out->f = ctx->f;
  out->w1 = ctx->integer ? (double)ctx->t1_total : std::ldexp((double)ctx->t1_total, -ctx->e1);
  out->sampled = ctx->sampled;
  out->inserted = hs.inserted;
  out->diag_skipped = hs.diag_skipped;
  out->distinct = hs.new_keys;
  out->positive = ctx->positive;
  out->hash_capacity = ctx->hcap;
  out->launches = ctx->launches;
  out->integer_mode = ctx->integer ? 1u : 0u;
  out->device_error = hs.err;
  return MAD_OK;
}

mad_status mad_dense_topt(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                          uint32_t rescore, mad_pair* out_dev, uint32_t* n_out_host,
                          mad_stream stream) {
  if (!ctx || !A || !B || !n_out_host || !out_dev || t == 0) return MAD_ERR_ARG;
  *n_out_host = 0;
  if (!valid_dense(A) || !valid_dense(B)) return MAD_ERR_UNSUPPORTED;
  if (B->rows != A->cols || A->rows >= (1ll << 31) || B->cols >= (1ll << 31)) return MAD_ERR_ARG;
  const uint64_t keep = rescore ? (uint64_t)rescore : 8ull * t;
  if (A->cols > 640 || keep < t || keep > 65536) return MAD_ERR_UNSUPPORTED;
  rescore = (uint32_t)keep;
  return dense_comparator(ctx, A, B, t, rescore, out_dev, n_out_host, nullptr,
                          (cudaStream_t)stream);
}

mad_status mad_debug_dense_product(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                                   float* c_dev, mad_stream stream) {
  if (!ctx || !A || !B || !c_dev) return MAD_ERR_ARG;
  if (!valid_dense(A) || !valid_dense(B)) return MAD_ERR_UNSUPPORTED;
  if (B->rows != A->cols || A->rows >= (1ll << 31) || B->cols >= (1ll << 31)) return MAD_ERR_ARG;
  if (A->cols > 640) return MAD_ERR_UNSUPPORTED;
  uint32_t dummy = 0;
  return dense_comparator(ctx, A, B, 1, 1, nullptr, &dummy, c_dev, (cudaStream_t)stream);
}

mad_status mad_debug_draws(mad_ctx* ctx, uint64_t seed, uint64_t first, uint64_t count,
                           uint32_t* i_dev, uint32_t* k_dev, uint32_t* j_dev, uint32_t* kp_dev,
                           int64_t* v_dev, mad_stream stream) {
  if (!ctx || (count && (!i_dev || !k_dev || !j_dev || !kp_dev || !v_dev))) return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  return debug_draws_impl(ctx, seed, first, nullptr, count, i_dev, k_dev, j_dev, kp_dev, v_dev,
                          (cudaStream_t)stream);
}

mad_status mad_debug_draws_list(mad_ctx* ctx, uint64_t seed, const uint64_t* ells_dev,
                                uint64_t count, uint32_t* i_dev, uint32_t* k_dev,
                                uint32_t* j_dev, uint32_t* kp_dev, int64_t* v_dev,
                                mad_stream stream) {
  if (!ctx || (count && (!ells_dev || !i_dev || !k_dev || !j_dev || !kp_dev || !v_dev)))
    return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  return debug_draws_impl(ctx, seed, 0, ells_dev, count, i_dev, k_dev, j_dev, kp_dev, v_dev,
                          (cudaStream_t)stream);
}

mad_status mad_export_x(mad_ctx* ctx, uint64_t* keys_dev, int64_t* vals_dev, uint64_t cap,
                        uint64_t* n_host, mad_stream stream) {
  if (!ctx || !n_host || (cap && (!keys_dev || !vals_dev))) return MAD_ERR_ARG;
  *n_host = 0;
  if (!ctx->built) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  mad_status rs = ensure_scratch(ctx, 256, st);
  if (rs != MAD_OK) return rs;
  return export_x(ctx, keys_dev, vals_dev, cap, n_host, (unsigned long long*)ctx->scratch, st);
}

mad_status mad_export_x_by_owner(mad_ctx* ctx, uint32_t world, uint64_t* keys_dev,
                                 int64_t* vals_dev, uint64_t cap, uint64_t* offsets_host,
                                 mad_stream stream) {
  if (!ctx || !offsets_host || world == 0 || world > 65536 || (cap && (!keys_dev || !vals_dev)))
    return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  mad_status rs = ensure_scratch(ctx, sizeof(unsigned long long) * (3 * (size_t)world + 1), st);
  if (rs != MAD_OK) return rs;
  return export_x_by_owner(ctx, world, keys_dev, vals_dev, cap, offsets_host, st);
}

mad_status mad_accumulate(mad_ctx* ctx, const uint64_t* keys_dev, const int64_t* vals_dev,
                          uint64_t n, mad_stream stream) {
  if (!ctx || (n && (!keys_dev || !vals_dev))) return MAD_ERR_ARG;
  if (!ctx->built) return MAD_ERR_STATE;
  return accumulate_pairs(ctx, keys_dev, vals_dev, n, (cudaStream_t)stream);
}

mad_status mad_select_pairs(mad_ctx* ctx, const mad_pair* pairs_dev, uint64_t n, uint32_t K,
                            mad_pair* out_dev, uint32_t* n_out_host, mad_stream stream) {
  if (!ctx || !n_out_host || (n && !pairs_dev) || (K && !out_dev)) return MAD_ERR_ARG;
  *n_out_host = 0;
  uint64_t nsel = 0;
  mad_status rs = select_pairs(ctx, pairs_dev, n, K, out_dev, &nsel, (cudaStream_t)stream);
  if (rs != MAD_OK) return rs;
  *n_out_host = (uint32_t)nsel;
  return MAD_OK;
}

mad_status mad_export_table(mad_ctx* ctx, int which, void* out_dev, uint64_t cap,
                            uint64_t* n_host, mad_stream stream) {
  if (!ctx || !n_host) return MAD_ERR_ARG;
  *n_host = 0;
  if (!ctx->built) return MAD_ERR_STATE;
  const void* src = nullptr;
  size_t elem = 4;
  uint64_t count = 0;
  switch (which) {
    case 0: src = ctx->T1; elem = 8; count = (uint64_t)ctx->m; break;
    case 1: src = ctx->T2; count = ctx->nnz_a; break;
    case 2: src = ctx->TA; count = ctx->TA ? ctx->nnz_a : 0; break;
    case 3: src = ctx->TB; count = ctx->TB ? ctx->nnz_b : 0; break;
    case 4: src = ctx->na; count = ctx->na ? (uint64_t)ctx->m : 0; break;
    case 5: src = ctx->nb; count = ctx->nb ? (uint64_t)ctx->d : 0; break;
    case 6: src = ctx->r; count = ctx->r ? (uint64_t)ctx->m : 0; break;
    case 7: src = ctx->TK ? ctx->TK + ctx->TK_shift : nullptr; elem = 8;
            count = ctx->TK ? (uint64_t)ctx->d : 0; break;
    case 8: src = ctx->TAc; count = ctx->TAc ? (uint64_t)(ctx->m * ctx->d) : 0; break;
    case 9: src = ctx->nac; count = ctx->nac ? (uint64_t)ctx->d : 0; break;
    default: {
      // Alias families (MAD_ALIAS): 10 + 3 f + part, f = T1, T2, TA, TB.
      if (which < 10 || which >= 22) return MAD_ERR_ARG;
      const int f = (which - 10) / 3, part = (which - 10) % 3;
      const int64_t rows = f == kAlT1 ? 1 : f == kAlTB ? ctx->d : ctx->m;
      const int64_t L = f == kAlT1 ? ctx->m : f == kAlTB ? ctx->n : ctx->d;
      const int64_t nseg = ctx->al_nseg[f];
      if (!ctx->al[f]) break;
      if (part == 0) { src = ctx->al[f]; elem = sizeof(AliasEnt); count = (uint64_t)(rows * (L + nseg)); }
      else if (part == 1) { src = ctx->al_seg[f]; elem = 8; count = (uint64_t)(rows * nseg); }
      else { src = ctx->al_row[f]; elem = 8; count = (uint64_t)rows; }
    }
  }
  *n_host = count;
  if (count == 0 || cap == 0) return MAD_OK;
  if (!out_dev) return MAD_ERR_ARG;
  const uint64_t ncopy = count < cap ? count : cap;
  cudaStream_t st = (cudaStream_t)stream;
  cudaMemcpyAsync(out_dev, src, ncopy * elem, cudaMemcpyDeviceToDevice, st);
  return cuda_status(cudaStreamSynchronize(st));
}

}  // extern "C"
