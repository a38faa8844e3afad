// Exact dot products of the candidates (Alg. 3): c_ij = a_i . b_j.
//
// Dense inputs: one warp per candidate; lane L accumulates k = L, L+32, ...
// in FP64 with fused multiply-add (products of FP32 inputs are exact in
// FP64), then the 32 partials are folded in halves by XOR shuffles.  Row i
// of A and row j of B^T (built with the tables) are read contiguously.
// 0/1 CSR inputs: c_ij = |{k in row i of A : b_kj = 1}|, counted exactly,
// one warp per candidate, one binary search of j in row k of B per lane.
// 0/1 Gram inputs (B = A^T): c_ij = |row i of A ∩ row j of A|.  When a
// bitmap over the d columns fits in shared memory, the candidates are
// grouped by their endpoint of larger degree (the hub) and one block per SM
// takes 64 of them at a time (from a counter): it sets the hub's row as
// bits, then each warp counts the other endpoint's row against them with
// independent 16-byte loads.  Otherwise one warp per candidate intersects the two sorted rows.
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

// ---- Grouped 0/1 Gram rescoring -------------------------------------------
// A candidate's record in hub order: its index q and pair (i, j), its hub
// (the endpoint of larger degree, the smaller index on a tie; m for a pair
// outside the matrix), and the extents of the hub's row and of the other
// endpoint's row in the column array.
struct __align__(16) GramRec {
  uint32_t q, i, j, hub;
  uint32_t lo_len, hub_len, pad0, pad1;
  long long lo_start, hub_start;
};

constexpr int kRgUnit = 64;        // candidates a block takes at a time
constexpr int kRgThreads = 1024;
constexpr int kRgKeep = 8;         // hub columns a thread keeps between set and clear

__device__ __forceinline__ GramRec gram_rec(const mad_pair* __restrict__ cand, unsigned long long q,
                                            const int64_t* __restrict__ a_ptr, int64_t m) {
  GramRec r;
  r.q = (uint32_t)q;
  r.i = cand[q].i;
  r.j = cand[q].j;
  r.pad0 = r.pad1 = 0;
  if (r.i < m && r.j < m) {
    const int64_t i0 = __ldg(a_ptr + r.i), i1 = __ldg(a_ptr + r.i + 1);
    const int64_t j0 = __ldg(a_ptr + r.j), j1 = __ldg(a_ptr + r.j + 1);
    const bool hub_i = i1 - i0 > j1 - j0 || (i1 - i0 == j1 - j0 && r.i <= r.j);
    r.hub = hub_i ? r.i : r.j;
    r.hub_start = hub_i ? i0 : j0;
    r.hub_len = (uint32_t)(hub_i ? i1 - i0 : j1 - j0);
    r.lo_start = hub_i ? j0 : i0;
    r.lo_len = (uint32_t)(hub_i ? j1 - j0 : i1 - i0);
  } else {
    r.hub = (uint32_t)m;
    r.hub_start = r.lo_start = 0;
    r.hub_len = r.lo_len = 0;
  }
  return r;
}

// Candidates per hub (cnt[m] counts the pairs outside the matrix).
__global__ void __launch_bounds__(256)
k_rg_count(const mad_pair* __restrict__ cand, unsigned long long ncand_max,
           const unsigned long long* n_dev, const int64_t* __restrict__ a_ptr, int64_t m,
           uint32_t* __restrict__ cnt) {
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncand;
       q += (unsigned long long)gridDim.x * blockDim.x)
    atomicAdd(cnt + gram_rec(cand, q, a_ptr, m).hub, 1u);
}

// Records in hub order (off: the exclusive scan of the counts; the order
// within a hub is immaterial).
__global__ void __launch_bounds__(256)
k_rg_scatter(const mad_pair* __restrict__ cand, unsigned long long ncand_max,
             const unsigned long long* n_dev, const int64_t* __restrict__ a_ptr, int64_t m,
             uint32_t* __restrict__ off, GramRec* __restrict__ rec) {
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < ncand;
       q += (unsigned long long)gridDim.x * blockDim.x) {
    const GramRec r = gram_rec(cand, q, a_ptr, m);
    rec[atomicAdd(off + r.hub, 1u)] = r;
  }
}

__device__ __forceinline__ uint32_t bit_of(const uint32_t* bits, int32_t c, int64_t d) {
  return (uint32_t)c < (uint64_t)d ? (bits[(uint32_t)c >> 5] >> ((uint32_t)c & 31u)) & 1u : 0u;
}

// Entries of row P[0..len) whose bit is set, summed over the warp's lanes
// (lane-strided 16-byte loads, four in flight per lane).
__device__ __forceinline__ uint32_t count_row_in_bits(const uint32_t* bits, int64_t d,
                                                      const int32_t* __restrict__ P, uint32_t len,
                                                      int lane) {
  uint32_t count = 0;
  const uint32_t mis = (uint32_t)(((uintptr_t)P >> 2) & 3u);
  uint32_t head = (4u - mis) & 3u;
  head = head < len ? head : len;
  if ((uint32_t)lane < head) count += bit_of(bits, __ldg(P + lane), d);
  const int32_t* Q = P + head;
  const uint32_t rest = len - head, nv = rest >> 2;
  const int4* V = reinterpret_cast<const int4*>(Q);
  for (uint32_t v = lane; v < nv; v += 128) {
    int4 x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      x[u] = v + 32u * u < nv ? __ldg(V + v + 32u * u) : make_int4(-1, -1, -1, -1);
#pragma unroll
    for (int u = 0; u < 4; ++u)
      count += bit_of(bits, x[u].x, d) + bit_of(bits, x[u].y, d) + bit_of(bits, x[u].z, d) +
               bit_of(bits, x[u].w, d);
  }
  for (uint32_t e = 4 * nv + lane; e < rest; e += 32) count += bit_of(bits, __ldg(Q + e), d);
  return count;
}

// The exact counts of the grouped candidates: units of kRgUnit records;
// within a unit, each run of one hub sets the hub's row in the shared bitmap
// over the d columns, each warp counts one candidate's other row against it,
// and the hub's bits are cleared again.  Column indices at or above d are
// never set or counted.
__global__ void __launch_bounds__(kRgThreads, 1)
k_rescore_bitmap(const GramRec* __restrict__ rec, unsigned long long ncand_max,
                 const unsigned long long* n_dev, const int32_t* __restrict__ a_col, int64_t m,
                 int64_t d, double* __restrict__ cvals, Item* __restrict__ items,
                 DevScalars* sc, unsigned long long* next_unit) {
  extern __shared__ uint32_t bits[];
  __shared__ GramRec s_rec[kRgUnit];
  __shared__ int s_start[kRgUnit + 1];
  __shared__ int s_nrun;
  __shared__ unsigned long long s_unit;
  const unsigned long long ncand = dev_len(ncand_max, n_dev);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t words = (uint32_t)((d + 31) >> 5);
  for (uint32_t w = tid; w < words; w += kRgThreads) bits[w] = 0u;
  const unsigned long long units = (ncand + kRgUnit - 1) / kRgUnit;
  // Units from a counter: their cost varies with the number of hubs in
  // them (one bitmap per hub), so a fixed assignment left some blocks
  // twice the mean work.
  for (;;) {
    __syncthreads();   // the bitmap is clear and the previous unit's records are done
    if (tid == 0) s_unit = atomicAdd(next_unit, 1ull);
    __syncthreads();
    const unsigned long long u = s_unit;
    if (u >= units) break;
    const unsigned long long p0 = u * kRgUnit;
    const int n = (int)(ncand - p0 < (unsigned long long)kRgUnit ? ncand - p0 : kRgUnit);
    if (tid < n) {
      const uint4* src = reinterpret_cast<const uint4*>(rec + p0 + tid);
      uint4* dst = reinterpret_cast<uint4*>(s_rec + tid);
      dst[0] = __ldg(src);
      dst[1] = __ldg(src + 1);
      dst[2] = __ldg(src + 2);
    }
    __syncthreads();
    if (warp == 0) {   // where each run of one hub starts
      int nrun = 0;
      for (int h = 0; h < kRgUnit; h += 32) {
        const int p = h + lane;
        const bool st = p < n && (p == 0 || s_rec[p].hub != s_rec[p - 1].hub);
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, st);
        if (st) s_start[nrun + __popc(bal & ((1u << lane) - 1u))] = p;
        nrun += __popc(bal);
      }
      if (lane == 0) {
        s_start[nrun] = n;
        s_nrun = nrun;
      }
    }
    __syncthreads();
    const int nrun = s_nrun;
    for (int r = 0; r < nrun; ++r) {
      const int a = s_start[r], b = s_start[r + 1];
      const bool valid = s_rec[a].hub < (uint64_t)m;
      const int32_t* H = a_col + s_rec[a].hub_start;
      const uint32_t hl = valid ? s_rec[a].hub_len : 0u;
      // The hub's columns this thread sets, kept to clear them again (rows
      // longer than kRgKeep x kRgThreads are read a second time).
      int32_t keep[kRgKeep];
#pragma unroll
      for (int k = 0; k < kRgKeep; ++k) {
        const uint32_t e = (uint32_t)tid + (uint32_t)k * kRgThreads;
        keep[k] = e < hl ? __ldg(H + e) : -1;
      }
#pragma unroll
      for (int k = 0; k < kRgKeep; ++k) {
        const int32_t c = keep[k];
        if ((uint32_t)c < (uint64_t)d) atomicOr(&bits[(uint32_t)c >> 5], 1u << ((uint32_t)c & 31u));
      }
      for (uint32_t e = tid + kRgKeep * kRgThreads; e < hl; e += kRgThreads) {
        const int32_t c = __ldg(H + e);
        if ((uint32_t)c < (uint64_t)d) atomicOr(&bits[(uint32_t)c >> 5], 1u << ((uint32_t)c & 31u));
      }
      __syncthreads();
      for (int x = a + warp; x < b; x += 32) {
        uint32_t count =
            valid ? count_row_in_bits(bits, d, a_col + s_rec[x].lo_start, s_rec[x].lo_len, lane) : 0u;
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, off);
        if (lane == 0) {
          if (!valid) atomicOr(&sc->err, DERR_SEARCH);
          const double c = (double)count;
          const uint32_t q = s_rec[x].q;
          cvals[q] = c;
          Item it;
          it.p = (unsigned long long)__double_as_longlong(c);
          it.key = ((unsigned long long)s_rec[x].i << 32) | s_rec[x].j;
          it.aux = q;
          items[q] = it;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kRgKeep; ++k) {
        const int32_t c = keep[k];
        if ((uint32_t)c < (uint64_t)d) bits[(uint32_t)c >> 5] = 0u;
      }
      for (uint32_t e = tid + kRgKeep * kRgThreads; e < hl; e += kRgThreads) {
        const int32_t c = __ldg(H + e);
        if ((uint32_t)c < (uint64_t)d) bits[(uint32_t)c >> 5] = 0u;
      }
      __syncthreads();   // cleared before the next run sets its bits
    }
  }
}

// Shared memory of k_rescore_bitmap's bitmap, and the largest allowed.
size_t gram_bitmap_bytes(int64_t d) { return (size_t)((d + 31) >> 5) * sizeof(uint32_t); }
constexpr size_t kBitmapMaxBytes = 200 * 1024;

// Layout of the grouping buffer: hub counts and offsets (m + 1 each), the
// scan's partials, then the records.
struct RgLayout {
  size_t cnt, off, part, next, rec, bytes;
};
RgLayout rg_layout(int64_t m, uint64_t ncand) {
  auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
  RgLayout L;
  L.cnt = 0;
  L.off = up((size_t)(m + 1) * sizeof(uint32_t));
  L.part = L.off + up((size_t)(m + 1) * sizeof(uint32_t));
  L.next = L.part + up(scan_partial_elems((uint64_t)m + 1) * sizeof(uint32_t));
  L.rec = L.next + 256;
  L.bytes = L.rec + (size_t)ncand * sizeof(GramRec);
  return L;
}

bool gram_bitmap_applies(const mad_ctx* ctx) {
  return ctx->integer && (ctx->flags & MAD_GRAM) && gram_bitmap_bytes(ctx->d) <= kBitmapMaxBytes;
}

int rescore_bitmap_grid(size_t smem) {
  static size_t attr = 0;
  if (attr < kBitmapMaxBytes) {
    cudaFuncSetAttribute(k_rescore_bitmap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kBitmapMaxBytes);
    attr = kBitmapMaxBytes;
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rescore_bitmap, kRgThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return sms * per_sm;
}

mad_status rescore_gram_grouped(mad_ctx* ctx, const mad_pair* cand, uint64_t ncand, Item* items,
                                double* cvals, cudaStream_t st, const unsigned long long* n_dev) {
  const RgLayout L = rg_layout(ctx->m, ncand);
  char* base = (char*)ctx->rg_buf;
  uint32_t* cnt = (uint32_t*)(base + L.cnt);
  uint32_t* off = (uint32_t*)(base + L.off);
  uint32_t* part = (uint32_t*)(base + L.part);
  GramRec* rec = (GramRec*)(base + L.rec);
  unsigned long long* next_unit = (unsigned long long*)(base + L.next);
  const uint64_t hubs = (uint64_t)ctx->m + 1;
  cudaMemsetAsync(cnt, 0, hubs * sizeof(uint32_t), st);
  cudaMemsetAsync(next_unit, 0, sizeof(unsigned long long), st);
  const unsigned long long blocks = (ncand + 255) / 256;
  const unsigned grid = (unsigned)(blocks < 152 * 8 ? blocks : 152 * 8);
  k_rg_count<<<grid, 256, 0, st>>>(cand, ncand, n_dev, ctx->A.rowptr, ctx->m, cnt);
  count_launch(ctx);
  mad_status rs = scan_exclusive_u32(ctx, cnt, off, hubs, part, st);
  if (rs != MAD_OK) return rs;
  k_rg_scatter<<<grid, 256, 0, st>>>(cand, ncand, n_dev, ctx->A.rowptr, ctx->m, off, rec);
  count_launch(ctx);
  const size_t smem = gram_bitmap_bytes(ctx->d);
  const unsigned long long units = (ncand + kRgUnit - 1) / kRgUnit;
  const int full = rescore_bitmap_grid(smem);
  k_rescore_bitmap<<<(unsigned)(units < (unsigned long long)full ? units : full), kRgThreads, smem,
                     st>>>(rec, ncand, n_dev, ctx->A.colidx, ctx->m, ctx->d, cvals, items,
                           ctx->sc, next_unit);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
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

// The grouping buffer of the 0/1 Gram rescoring for up to ncand candidates
// (nothing for other inputs); allocated on the context's stream.
mad_status rescore_reserve(mad_ctx* ctx, uint64_t ncand, cudaStream_t st) {
  if (!gram_bitmap_applies(ctx) || ncand <= ctx->rg_cap) return MAD_OK;
  if (ctx->scratch_fixed) return MAD_ERR_STATE;
  if (ctx->rg_buf) cudaFreeAsync(ctx->rg_buf, st);
  ctx->rg_buf = nullptr;
  ctx->rg_cap = 0;
  const mad_status rs = pool_malloc(ctx, &ctx->rg_buf, rg_layout(ctx->m, ncand).bytes, st);
  if (rs != MAD_OK) return rs;
  ctx->rg_cap = ncand;
  return MAD_OK;
}

mad_status rescore_items(mad_ctx* ctx, const mad_pair* cand, uint64_t ncand, Item* items,
                         double* cvals, cudaStream_t st, const unsigned long long* n_dev) {
  if (ncand == 0) return MAD_OK;
  if (gram_bitmap_applies(ctx) && ctx->rg_buf && ctx->rg_cap >= ncand)
    return rescore_gram_grouped(ctx, cand, ncand, items, cvals, st, n_dev);
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
