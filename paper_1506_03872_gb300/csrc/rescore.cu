// Exact dot products of the candidates (Alg. 3): c_ij = a_i . b_j.
//
// Dense inputs: one warp per candidate; lane L accumulates k = L, L+32, ...
// in FP64 with fused multiply-add (products of FP32 inputs are exact in
// FP64), then the 32 partials are folded in halves by XOR shuffles.  Row i
// of A and row j of B^T (built with the tables) are read contiguously.
// 0/1 CSR inputs: c_ij = |{k in row i of A : b_kj = 1}|, counted exactly,
// one warp per candidate, one binary search of j in row k of B per lane.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(double v) { return v; }

template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_rescore_dense(const mad_pair* __restrict__ cand, unsigned long long ncand_max,
                const TA* __restrict__ A, int64_t lda, const TB* __restrict__ Bt, int64_t d,
                int64_t m, int64_t n, double* __restrict__ cvals, Item* __restrict__ items,
                DevScalars* sc, const unsigned long long* n_dev) {
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < ncand; q += warps) {
    const uint32_t i = cand[q].i, j = cand[q].j;
    if (i >= m || j >= n) {  // outside the matrices: report, do not read
      if (lane == 0) {
        atomicOr(&sc->err, DERR_SEARCH);
        cvals[q] = 0.0;
        Item it;
        it.p = 0;
        it.key = ((unsigned long long)i << 32) | j;
        it.aux = q;
        items[q] = it;
      }
      continue;
    }
    const TA* __restrict__ a = A + (int64_t)i * lda;
    const TB* __restrict__ b = Bt + (int64_t)j * d;
    double acc = 0.0;
    for (int64_t k = lane; k < d; k += 32) acc = __fma_rn(to_f64(a[k]), to_f64(b[k]), acc);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
    if (lane == 0) {
      cvals[q] = acc;
      Item it;
      it.p = (unsigned long long)__double_as_longlong(fabs(acc));
      it.key = ((unsigned long long)i << 32) | j;
      it.aux = q;
      items[q] = it;
    }
  }
}

__global__ void __launch_bounds__(256)
k_rescore_binary(const mad_pair* __restrict__ cand, unsigned long long ncand_max,
                 const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_col,
                 const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col, int64_t m,
                 int64_t n, double* __restrict__ cvals, Item* __restrict__ items,
                 DevScalars* sc, const unsigned long long* n_dev) {
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < ncand; q += warps) {
    const uint32_t i = cand[q].i, j = cand[q].j;
    if (i >= m || j >= n) {
      if (lane == 0) {
        atomicOr(&sc->err, DERR_SEARCH);
        cvals[q] = 0.0;
        Item it;
        it.p = 0;
        it.key = ((unsigned long long)i << 32) | j;
        it.aux = q;
        items[q] = it;
      }
      continue;
    }
    const int64_t a0 = a_ptr[i], a1 = a_ptr[i + 1];
    long long count = 0;
    for (int64_t e = a0 + lane; e < a1; e += 32) {
      const int32_t k = a_col[e];
      const int64_t b0 = b_ptr[k];
      if (contains_sorted(b_col + b0, b_ptr[k + 1] - b0, (int32_t)j)) ++count;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, off);
    if (lane == 0) {
      const double c = (double)count;
      cvals[q] = c;
      Item it;
      it.p = (unsigned long long)__double_as_longlong(c);
      it.key = ((unsigned long long)i << 32) | j;
      it.aux = q;
      items[q] = it;
    }
  }
}

// MAD_GRAM on 0/1 rows (B = A^T): c_ij = |row i of A ∩ row j of A|, an
// exact count.  One warp per candidate picks the cheaper of two parallel
// intersections: when one row is much shorter, lanes look its entries up in
// the longer row by binary search; otherwise the two rows are merged along
// 32 equal diagonals of their merge path (ties taken from the shorter row
// first), each lane counting the entries of the shorter row it consumes
// that equal the next entry of the longer row.
__device__ __forceinline__ int ceil_log2_i(int64_t v) {
  int r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}

__global__ void __launch_bounds__(256)
k_rescore_gram_binary(const mad_pair* __restrict__ cand, unsigned long long ncand_max,
                      const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_col,
                      int64_t m, double* __restrict__ cvals, Item* __restrict__ items,
                      DevScalars* sc, const unsigned long long* n_dev) {
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < ncand; q += warps) {
    const uint32_t i = cand[q].i, j = cand[q].j;
    long long count = 0;
    const bool ok = i < m && j < m;
    if (ok) {
      const int64_t i0 = __ldg(a_ptr + i), i1 = __ldg(a_ptr + i + 1);
      const int64_t j0 = __ldg(a_ptr + j), j1 = __ldg(a_ptr + j + 1);
      const bool i_short = (i1 - i0) <= (j1 - j0);
      const int32_t* S = a_col + (i_short ? i0 : j0);
      const int32_t* L = a_col + (i_short ? j0 : i0);
      const int64_t ps = i_short ? i1 - i0 : j1 - j0;
      const int64_t ql = i_short ? j1 - j0 : i1 - i0;
      const int lgq = ceil_log2_i(ql + 1);
      if ((ps + 31) / 32 * lgq <= (ps + ql + 31) / 32 + ceil_log2_i(ps + 1)) {
        for (int64_t e = lane; e < ps; e += 32) {
          const int32_t x = __ldg(S + e);
          int64_t lo = 0, len = ql;
          while (len > 0) {
            const int64_t half = len >> 1;
            if (__ldg(L + lo + half) < x) {
              lo += half + 1;
              len -= half + 1;
            } else {
              len = half;
            }
          }
          count += (lo < ql && __ldg(L + lo) == x) ? 1 : 0;
        }
      } else {
        const int64_t total = ps + ql;
        const int64_t per = (total + 31) / 32;
        const int64_t d0 = min(total, per * lane), d1 = min(total, per * (lane + 1));
        // number of S entries among the first d0 merged entries
        int64_t lo = d0 > ql ? d0 - ql : 0, hi = d0 < ps ? d0 : ps;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (__ldg(S + mid) <= __ldg(L + (d0 - mid - 1))) lo = mid + 1;
          else hi = mid;
        }
        int64_t a = lo, b = d0 - lo;
        for (int64_t dd = d0; dd < d1; ++dd) {
          const int32_t sv = a < ps ? __ldg(S + a) : 0x7FFFFFFF;
          const int32_t lv = b < ql ? __ldg(L + b) : 0x7FFFFFFF;
          if (a < ps && (b >= ql || sv <= lv)) {
            count += (b < ql && sv == lv) ? 1 : 0;
            ++a;
          } else {
            ++b;
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, off);
    if (lane == 0) {
      if (!ok) atomicOr(&sc->err, DERR_SEARCH);
      const double c = ok ? (double)count : 0.0;
      cvals[q] = c;
      Item it;
      it.p = (unsigned long long)__double_as_longlong(c);
      it.key = ((unsigned long long)i << 32) | j;
      it.aux = q;
      items[q] = it;
    }
  }
}

template <typename TA, typename TB>
void launch_dense(mad_ctx* ctx, const mad_pair* cand, uint64_t ncand, Item* items, double* cvals,
                  const unsigned long long* n_dev, cudaStream_t st) {
  const unsigned long long blocks = (ncand * 32 + 255) / 256;
  k_rescore_dense<TA, TB><<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
      cand, ncand, (const TA*)ctx->A.values, ctx->A.ld, (const TB*)ctx->bt, ctx->d, ctx->m, ctx->n,
      cvals, items, ctx->sc, n_dev);
  count_launch(ctx);
}

}  // namespace

mad_status rescore_items(mad_ctx* ctx, const mad_pair* cand, uint64_t ncand, Item* items,
                         double* cvals, cudaStream_t st, const unsigned long long* n_dev) {
  if (ncand == 0) return MAD_OK;
  if (ctx->integer && (ctx->flags & MAD_GRAM)) {
    const unsigned long long blocks = (ncand * 32 + 255) / 256;
    k_rescore_gram_binary<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
        cand, ncand, ctx->A.rowptr, ctx->A.colidx, ctx->m, cvals, items, ctx->sc, n_dev);
    count_launch(ctx);
  } else if (ctx->integer) {
    const unsigned long long blocks = (ncand * 32 + 255) / 256;
    k_rescore_binary<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
        cand, ncand, ctx->A.rowptr, ctx->A.colidx, ctx->B.rowptr, ctx->B.colidx, ctx->m, ctx->n,
        cvals, items, ctx->sc, n_dev);
    count_launch(ctx);
  } else {
    const bool a64 = ctx->A.dt == MAD_F64, b64 = ctx->B.dt == MAD_F64;
    if (a64 && b64) launch_dense<double, double>(ctx, cand, ncand, items, cvals, n_dev, st);
    else if (a64) launch_dense<double, float>(ctx, cand, ncand, items, cvals, n_dev, st);
    else if (b64) launch_dense<float, double>(ctx, cand, ncand, items, cvals, n_dev, st);
    else launch_dense<float, float>(ctx, cand, ncand, items, cvals, n_dev, st);
  }
  return cuda_status(cudaGetLastError());
}

}  // namespace mad
