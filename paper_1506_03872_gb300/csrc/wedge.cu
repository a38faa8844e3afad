// Wedge sampling (the paper's comparison method, appendix "Previous
// approach: Wedge sampling", Alg. "MAD wedge sampling"), on the tables of the
// diamond sampler.  With A m x d (rows a_i) and B d x n:
//   w_k = ||a_*k||_1 ||b_k*||_1;  k ~ w_k / ||w||_1;  i ~ |a_ik| / ||a_*k||_1
//   (column k of A);  j ~ |b_kj| / ||b_k*||_1 (row k of B);
//   x_ij += sgn(a_ik b_kj)  (1 for 0/1 and nonnegative inputs),
// so that E[x_ij] = s c_ij / ||w||_1.  The paper prints the increment as
// sgn(a_ki b_ki); its proof uses a_ki b_kj, which is what is added.
//
// Tables, in the numeric conventions of the diamond tables: the column
// sums of |A| in the canonical FP32 order; the column tables TAc
// (column-major, column k at TAc + k m): the prefix over i of |a_ik| 2^e_k
// rounded to nearest-even, e_k = 29 - floor(log2 ||a_*k||_1), the sign of a_ik
// in bit 31; TK: the uint64 prefix over k of w_k 2^EK rounded, EK = 62 -
// ceil(log2 d) - (floor(log2 max w) + 1), a nonzero weight that rounds to 0
// kept as 1.  Gram inputs (B = A^T) need no column tables: column k of A is
// row k of B, so TAc is TB.  0/1 Gram inputs: w_k = deg_k^2 exactly, and i,
// j are uniform among the entries of row k.
#include <cuda_runtime.h>
#include <stdint.h>

#include "draw.cuh"
#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(double v) { return __double2float_rn(v); }

// Column k of dense A: the canonical FP32 sum of |a_ik| (256 strided partial
// sums in ascending i, folded in halves) and the column table.  One block
// of 256 threads per column.
template <typename T>
__global__ void __launch_bounds__(256)
k_col_tables(const T* __restrict__ A, int64_t m, int64_t lda, float* __restrict__ nac,
             uint32_t* __restrict__ TAc) {
  __shared__ float part[256];
  __shared__ uint32_t warp_tot[8];
  __shared__ uint32_t s_carry;
  const int64_t k = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float acc = 0.0f;
  for (int64_t i = tid; i < m; i += 256) acc = __fadd_rn(acc, fabsf(as_f32(A[i * lda + k])));
  part[tid] = acc;
  for (int h = 128; h >= 1; h >>= 1) {
    __syncthreads();
    if (tid < h) part[tid] = __fadd_rn(part[tid], part[tid + h]);
  }
  __syncthreads();
  const float total = part[0];
  if (tid == 0) {
    nac[k] = total;
    s_carry = 0;
  }
  const int e = total > 0.0f ? 29 - ilogb_pos(total) : 0;
  uint32_t* col = TAc + k * m;
  for (int64_t base = 0; base < m; base += 256) {
    const int64_t i = base + tid;
    uint32_t q = 0, sign = 0;
    if (i < m) {
      const float a = as_f32(A[i * lda + k]);
      const float w = fabsf(a);
      if (total > 0.0f) {
        q = (uint32_t)fixed_point(w, e);
        if (w > 0.0f && q == 0u) q = 1u;
      }
      sign = a < 0.0f ? SIGN_BIT : 0u;
    }
    // block inclusive scan of q
    uint32_t x = q;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t before = s_carry;
    for (int w2 = 0; w2 < warp; ++w2) before += warp_tot[w2];
    if (i < m) col[i] = (before + x) | sign;
    __syncthreads();
    if (tid == 255) s_carry = before + x;
  }
}

// Dense centre table: w_k = ||a_*k||_1 (x) ||b_k*||_1, its scale and prefix.
// One block of 1024 threads (d <= 1024).
__global__ void __launch_bounds__(1024)
k_tk_dense(const float* __restrict__ nac, const float* __restrict__ nb, int64_t d, int clog2d,
           unsigned long long* __restrict__ TK, unsigned long long* __restrict__ out_total,
           int* __restrict__ out_ek) {
  __shared__ float s_max[32];
  __shared__ unsigned long long s_sum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float w = tid < d ? __fmul_rn(nac[tid], nb[tid]) : 0.0f;
  float mx = w;
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
  if (lane == 0) s_max[warp] = mx;
  __syncthreads();
  if (warp == 0) {
    float v = s_max[lane];
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) s_max[0] = v;
  }
  __syncthreads();
  const float maxw = s_max[0];
  if (maxw == 0.0f) {
    if (tid == 0) {
      *out_total = 0;
      *out_ek = 0;
    }
    return;
  }
  const int ek = 62 - clog2d - (ilogb_pos(maxw) + 1);
  unsigned long long q = 0;
  if (tid < d) {
    q = (unsigned long long)fixed_point(w, ek);
    if (w > 0.0f && q == 0ull) q = 1ull;
  }
  unsigned long long x = q;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_sum[warp] = x;
  __syncthreads();
  unsigned long long before = 0;
  for (int w2 = 0; w2 < warp; ++w2) before += s_sum[w2];
  if (tid < d) TK[tid] = before + x;
  if (tid == d - 1) {
    *out_total = before + x;
    *out_ek = ek;
  }
}

// 0/1 Gram centre weights: w_k = deg_k^2 (row k of B; column k of A).
__global__ void k_tk_binary(const int64_t* __restrict__ bptr, int64_t d,
                            unsigned long long* __restrict__ w) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < d;
       k += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long deg = (unsigned long long)(bptr[k + 1] - bptr[k]);
    w[k] = deg * deg;
  }
}

struct WedgeTables {
  const unsigned long long* TK;
  unsigned long long tk_total;
  int64_t d;
  const uint32_t* TAc;   // dense non-Gram column tables (null: TB rows, or 0/1)
};

// One wedge: (i, k, j, 0, v).
__device__ __forceinline__ Draw draw_wedge(const SampleParams& p, const WedgeTables& w,
                                           unsigned long long seed, unsigned long long ell,
                                           bool* bad) {
  const Uniforms u = diamond_uniforms(seed, ell);
  const int64_t k = search_u64((const uint64_t*)w.TK, w.d, draw_target(u.u0, w.tk_total), bad);
  Draw dr;
  dr.k = (uint32_t)k;
  dr.kp = 0;
  dr.v = 1;
  if (!p.dense) {
    const int64_t b0 = __ldg(p.b_ptr + k), blen = __ldg(p.b_ptr + k + 1) - b0;
    dr.i = (uint32_t)__ldg(p.b_col + b0 + (int64_t)draw_target(u.u1, (unsigned long long)blen));
    dr.j = (uint32_t)__ldg(p.b_col + b0 + (int64_t)draw_target(u.u2, (unsigned long long)blen));
    return dr;
  }
  // i within column k of A.
  const uint32_t* col;
  int len;
  const uint32_t* colg = nullptr;
  int colg_sh = 0;
  if (w.TAc) {
    col = w.TAc + k * p.m;
    len = (int)p.m;
  } else {
    col = p.TB + k * p.n;   // Gram: column k of A is row k of B
    len = (int)p.n;
    if (p.TBg) {
      colg = p.TBg + k * p.tbg_stride;
      colg_sh = (int)__ldg(p.TBg_sh + k);
    }
  }
  const uint32_t ctot = __ldg(col + len - 1) & PREFIX_MASK;
  const uint32_t ti = (uint32_t)draw_target(u.u1, ctot);
  int pi = colg ? ub_guided_u32(col, colg, colg_sh, ti, PREFIX_MASK)
                : ub_u32(col, len, ti, PREFIX_MASK);
  if (pi >= len) {
    *bad = true;
    pi = len - 1;
  }
  const uint32_t e_i = __ldg(col + pi);
  // j within row k of B.
  const uint32_t* row = p.TB + k * p.n;
  const uint32_t rtot = __ldg(row + p.n - 1) & PREFIX_MASK;
  const uint32_t tj = (uint32_t)draw_target(u.u2, rtot);
  int pj = p.TBg ? ub_guided_u32(row, p.TBg + k * p.tbg_stride, (int)__ldg(p.TBg_sh + k), tj,
                                 PREFIX_MASK)
                 : ub_u32(row, (int)p.n, tj, PREFIX_MASK);
  if (pj >= (int)p.n) {
    *bad = true;
    pj = (int)p.n - 1;
  }
  const uint32_t e_j = __ldg(row + pj);
  dr.i = (uint32_t)pi;
  dr.j = (uint32_t)pj;
  if (!(p.flags & MAD_NONNEG) && ((e_i ^ e_j) & SIGN_BIT)) dr.v = -1;
  return dr;
}

__global__ void __launch_bounds__(256)
k_wedge(const SampleParams p, const WedgeTables w, unsigned long long seed,
        unsigned long long first, unsigned long long s) {
  bool bad = false;
  unsigned long long inserted = 0, diag = 0, created = 0;
  bool full = false;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < s;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const Draw dr = draw_wedge(p, w, seed, first + q, &bad);
    uint32_t a = dr.i, b = dr.j;
    if ((p.flags & MAD_EXCLUDE_DIAG) && a == b) {
      ++diag;
      continue;
    }
    if ((p.flags & MAD_GRAM) && b < a) {
      const uint32_t c = a;
      a = b;
      b = c;
    }
    ++inserted;
    const int r = hash_add(p, ((unsigned long long)a << 32) | b, dr.v);
    if (r == 0) full = true;
    if (r == 2) ++created;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    inserted += __shfl_xor_sync(0xFFFFFFFFu, inserted, o);
    diag += __shfl_xor_sync(0xFFFFFFFFu, diag, o);
    created += __shfl_xor_sync(0xFFFFFFFFu, created, o);
  }
  const unsigned any_bad = __ballot_sync(0xFFFFFFFFu, bad);
  const unsigned any_full = __ballot_sync(0xFFFFFFFFu, full);
  if ((threadIdx.x & 31) == 0) {
    if (inserted) atomicAdd(&p.sc->inserted, inserted);
    if (diag) atomicAdd(&p.sc->diag_skipped, diag);
    if (created) atomicAdd(&p.sc->new_keys, created);
    if (any_bad) atomicOr(&p.sc->err, DERR_SEARCH);
    if (any_full) atomicOr(&p.sc->err, DERR_HASH_FULL);
  }
}

__global__ void __launch_bounds__(256)
k_wedge_draws(const SampleParams p, const WedgeTables w, unsigned long long seed,
              unsigned long long first, const unsigned long long* __restrict__ ells,
              unsigned long long count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
              uint32_t* okp, long long* ov) {
  bool bad = false;
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
       q < count; q += (unsigned long long)gridDim.x * blockDim.x) {
    const Draw dr = draw_wedge(p, w, seed, ells ? ells[q] : first + q, &bad);
    oi[q] = dr.i;
    ok[q] = dr.k;
    oj[q] = dr.j;
    okp[q] = dr.kp;
    ov[q] = dr.v;
  }
  if (bad) atomicOr(&p.sc->err, DERR_SEARCH);
}

int clog2(uint64_t x) {
  int e = 0;
  while (e < 64 && (1ull << e) < x) ++e;
  return e;
}

WedgeTables wedge_tables(const mad_ctx* ctx) {
  WedgeTables w;
  w.TK = ctx->TK;
  w.tk_total = ctx->tk_total;
  w.d = ctx->d;
  w.TAc = ctx->TAc;
  return w;
}

unsigned wedge_grid(unsigned long long work) {
  static int blocks = 0;
  if (!blocks) {
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_wedge, 256, 0);
    blocks = sms * (per_sm > 0 ? per_sm : 1);
  }
  const unsigned long long need = (work + 255) / 256;
  return (unsigned)(need < (unsigned long long)blocks ? (need ? need : 1) : blocks);
}

}  // namespace

uint64_t wedge_hash_slots(uint64_t s_max) {
  uint64_t cap = 1024;
  while ((double)cap < (double)s_max / 0.6 && cap < (1ull << 40)) cap <<= 1;
  return cap;
}

mad_status build_wedge_tables(mad_ctx* ctx, cudaStream_t st) {
  const bool gram = (ctx->flags & MAD_GRAM) != 0;
  if (!ctx->dense && !gram) return MAD_ERR_UNSUPPORTED;   // needs the columns of 0/1 A
  if (ctx->dense && ctx->d > 1024) return MAD_ERR_UNSUPPORTED;
  mad_status rs = MAD_OK;
  void* p = nullptr;
  if ((rs = pool_malloc(ctx, &p, sizeof(unsigned long long) * ((size_t)ctx->d + 1), st)) != MAD_OK)
    return rs;
  ctx->TK = (unsigned long long*)p;
  unsigned long long* total_dev = nullptr;
  int* ek_dev = nullptr;
  if ((rs = ensure_scratch(ctx, 64 + sizeof(unsigned long long) * ((size_t)ctx->d + 2) +
                                    8 * scan_partial_elems((uint64_t)ctx->d + 1),
                           st)) != MAD_OK)
    return rs;
  total_dev = (unsigned long long*)ctx->scratch;
  ek_dev = (int*)(total_dev + 1);
  if (ctx->dense) {
    if ((rs = pool_malloc(ctx, &p, sizeof(float) * (size_t)ctx->d, st)) != MAD_OK) return rs;
    ctx->nac = (float*)p;
    const mad_matrix& A = ctx->A;
    if (!gram) {
      if ((rs = pool_malloc(ctx, &p, sizeof(uint32_t) * (size_t)(ctx->m * ctx->d), st)) != MAD_OK)
        return rs;
      ctx->TAc = (uint32_t*)p;
      if (A.dt == MAD_F64)
        k_col_tables<double><<<(unsigned)ctx->d, 256, 0, st>>>((const double*)A.values, ctx->m,
                                                               A.ld, ctx->nac, ctx->TAc);
      else
        k_col_tables<float><<<(unsigned)ctx->d, 256, 0, st>>>((const float*)A.values, ctx->m,
                                                              A.ld, ctx->nac, ctx->TAc);
      count_launch(ctx);
    } else {
      cudaMemcpyAsync(ctx->nac, ctx->nb, sizeof(float) * (size_t)ctx->d, cudaMemcpyDeviceToDevice,
                      st);
    }
    k_tk_dense<<<1, 1024, 0, st>>>(ctx->nac, ctx->nb, ctx->d, clog2((uint64_t)ctx->d), ctx->TK,
                                    total_dev, ek_dev);
    count_launch(ctx);
  } else {
    unsigned long long* w = total_dev + 2;
    unsigned long long* part = w + ctx->d + 1;   // (unused by the exclusive scan's output)
    k_tk_binary<<<(unsigned)((ctx->d + 255) / 256 < 152 * 8 ? (ctx->d + 255) / 256 : 152 * 8),
                  256, 0, st>>>(ctx->B.rowptr, ctx->d, w);
    count_launch(ctx);
    // TK[k] = sum over k' <= k: the exclusive prefix shifted by one.
    if ((rs = scan_exclusive_u64(ctx, (const uint64_t*)w, (uint64_t*)(ctx->TK), (uint64_t)ctx->d,
                                 (uint64_t*)part, st)) != MAD_OK)
      return rs;
    cudaMemcpyAsync(total_dev, ctx->TK + ctx->d, sizeof(unsigned long long),
                    cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(ek_dev, 0, sizeof(int), st);
    ctx->TK_shift = 1;
  }
  unsigned long long host[2] = {0, 0};
  cudaMemcpyAsync(host, total_dev, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  ctx->tk_total = host[0];
  ctx->ek = (int)(host[1] & 0xFFFFFFFFull);
  if (ctx->tk_total == 0) return MAD_ERR_EMPTY;
  if (ctx->tk_total >= (1ull << 63)) return MAD_ERR_OVERFLOW;
  return MAD_OK;
}

mad_status wedge_sample_impl(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first,
                             cudaStream_t st) {
  if (s == 0) return MAD_OK;
  SampleParams p = make_params(ctx);
  WedgeTables w = wedge_tables(ctx);
  if (ctx->TK_shift) w.TK = ctx->TK + 1;
  k_wedge<<<wedge_grid(s), 256, 0, st>>>(p, w, seed, first, s);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status wedge_draws_impl(mad_ctx* ctx, uint64_t seed, uint64_t first, const uint64_t* ells,
                            uint64_t count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            uint32_t* okp, int64_t* ov, cudaStream_t st) {
  if (count == 0) return MAD_OK;
  SampleParams p = make_params(ctx);
  WedgeTables w = wedge_tables(ctx);
  if (ctx->TK_shift) w.TK = ctx->TK + 1;
  const unsigned long long blocks = (count + 255) / 256;
  k_wedge_draws<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(
      p, w, seed, first, (const unsigned long long*)ells, count, oi, ok, oj, okp,
      (long long*)ov);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

}  // namespace mad
