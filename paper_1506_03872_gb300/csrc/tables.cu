// Weights and cumulative sampling tables (Alg. 2 weight line; Sec. 4.2).
//
// Float mode (dense FP32/FP64 inputs):
//   ||b_k*||_1, ||a_i*||_1 and s_i = sum_k |a_ik| ||b_k*||_1 are FP32 sums in
//   one fixed order: 256 partial sums (partial q takes the indices equal to q
//   mod 256, ascending), folded in halves.  r_i = ||a_i*||_1 * s_i.
//   Row tables (T2 over k of |a_ik| ||b_k*||_1, TA over k of |a_ik|, TB over
//   j of |b_kj|) hold inclusive prefixes of round(w * 2^E) with
//   E = 29 - floor(log2(row sum)), so every prefix stays below 2^31 and bit
//   31 carries the sign of the underlying value of A or B.  T1 holds the
//   uint64 prefix of round(r_i * 2^E1), E1 = 62 - ceil(log2 m) -
//   (floor(log2 max r) + 1).  A nonzero weight that rounds to 0 becomes 1.
// Integer mode (0/1 CSR): T2 holds the prefix of deg_k^B along row i of A,
//   T1 the prefix of r_i = deg_i^A * sum_{k in N(i)} deg_k^B; the uniform
//   endpoint tables TA and TB are implicit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return __double2float_rn(v); }

// Inclusive warp scan of 32-bit values.
__device__ __forceinline__ uint32_t warp_inclusive_u32(uint32_t v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t o = __shfl_up_sync(0xFFFFFFFFu, v, off);
    if (lane >= off) v += o;
  }
  return v;
}

__device__ __forceinline__ unsigned long long warp_inclusive_u64(unsigned long long v, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, v, off);
    if (lane >= off) v += o;
  }
  return v;
}

// Exclusive scan of one 32-bit value per thread over a 256-thread block.
__device__ __forceinline__ uint32_t block_exclusive_u32(uint32_t v, uint32_t* warp_tot,
                                                        uint32_t* block_total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t inc = warp_inclusive_u32(v, lane);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const uint32_t t = lane < 8 ? warp_tot[lane] : 0u;
    const uint32_t ti = warp_inclusive_u32(t, lane);
    if (lane < 8) warp_tot[lane] = ti - t;  // exclusive warp offsets
    if (lane == 7) warp_tot[8] = ti;
  }
  __syncthreads();
  const uint32_t out = warp_tot[warp] + inc - v;
  *block_total = warp_tot[8];
  __syncthreads();
  return out;
}

__device__ __forceinline__ unsigned long long block_exclusive_u64(unsigned long long v,
                                                                  unsigned long long* warp_tot,
                                                                  unsigned long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long inc = warp_inclusive_u64(v, lane);
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long t = lane < 8 ? warp_tot[lane] : 0ull;
    const unsigned long long ti = warp_inclusive_u64(t, lane);
    if (lane < 8) warp_tot[lane] = ti - t;
    if (lane == 7) warp_tot[8] = ti;
  }
  __syncthreads();
  const unsigned long long out = warp_tot[warp] + inc - v;
  *total = warp_tot[8];
  __syncthreads();
  return out;
}

// round(w * 2^e) for a row table (integer round-to-nearest-even, no FP64),
// with the support-preserving bump.
__device__ __forceinline__ uint32_t quantize_row(float w, int e) {
  uint32_t q = (uint32_t)fixed_point(w, e);
  if (w > 0.0f && q == 0u) q = 1u;
  return q;
}

// ---------------------------------------------------------------------------
// Rows of dense B: ||b_k*||_1, max |b|, TB.  One 256-thread block per row.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_b_rows_dense(const T* __restrict__ B, int64_t n, int64_t ldb, float* __restrict__ nb,
               uint32_t* __restrict__ TB, DevScalars* sc) {
  __shared__ float part[256];
  __shared__ uint32_t warp_tot[9];
  const int64_t k = blockIdx.x;
  const T* __restrict__ row = B + k * ldb;
  const int t = threadIdx.x;
  float acc = 0.0f, mx = 0.0f;
  for (int64_t idx = t; idx < n; idx += 256) {
    const float v = fabsf(to_f32(row[idx]));
    acc = __fadd_rn(acc, v);
    mx = fmaxf(mx, v);
  }
  part[t] = acc;
  __syncthreads();
  for (int h = 128; h >= 1; h >>= 1) {
    if (t < h) part[t] = __fadd_rn(part[t], part[t + h]);
    __syncthreads();
  }
  const float total = part[0];
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
  if ((t & 31) == 0 && mx > 0.0f) atomicMax(&sc->maxb_bits, __float_as_uint(mx));
  if (t == 0) nb[k] = total;

  uint32_t* __restrict__ out = TB + k * n;
  const int e = total > 0.0f ? 29 - ilogb_pos(total) : 0;
  constexpr int PER = 16;  // consecutive entries per thread and tile
  uint32_t carry = 0;
  for (int64_t base = 0; base < n; base += 256 * PER) {
    uint32_t q[PER], sg[PER], local = 0;
#pragma unroll
    for (int c = 0; c < PER; ++c) {
      const int64_t idx = base + PER * t + c;
      q[c] = 0;
      sg[c] = 0;
      if (idx < n) {
        const float v = to_f32(row[idx]);
        if (total > 0.0f) local += quantize_row(fabsf(v), e);
        q[c] = local;
        sg[c] = v < 0.0f ? SIGN_BIT : 0u;
      }
    }
    uint32_t tile_total;
    const uint32_t excl = block_exclusive_u32(local, warp_tot, &tile_total);
#pragma unroll
    for (int c = 0; c < PER; ++c) {
      const int64_t idx = base + PER * t + c;
      if (idx < n) out[idx] = (carry + excl + q[c]) | sg[c];
    }
    carry += tile_total;
  }
}

// Rows of dense B with 1024 threads per row, the same results as
// k_b_rows_dense.  Sums: tiles of 8192 entries are loaded by all threads
// (eight independent loads each; the next tile's are issued before the
// current one is used) and staged in shared memory, where the 256 canonical
// partial sums advance in index order.  Table: four consecutive entries per
// thread, quantised and scanned across the block, the next tile prefetched.
// Part 0: sums and table; 1: the sums (nb, max |b|) alone; 2: the table
// alone, from the sums in nb (so that it can run beside the A rows).
template <typename T, int Part>
__global__ void __launch_bounds__(1024)
k_b_rows_wide(const T* __restrict__ B, int64_t n, int64_t ldb, float* __restrict__ nb,
              uint32_t* __restrict__ TB, DevScalars* sc) {
  constexpr int kTileB = 4096;      // table tiles: four consecutive entries per thread
  constexpr int kSumTile = 8192;    // sum tiles: eight loads in flight per thread
  constexpr int kSumPer = kSumTile / 1024;
  __shared__ float tile[kSumTile];
  __shared__ float part[256];
  __shared__ uint32_t wsum[33];
  const int64_t k = blockIdx.x;
  const T* __restrict__ row = B + k * ldb;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  float total;
  if (Part == 2) {
    total = nb[k];
  } else {
    float acc = 0.0f, mx = 0.0f;
    float cur[kSumPer];
#pragma unroll
    for (int r = 0; r < kSumPer; ++r) {
      const int64_t idx = t + 1024 * r;
      cur[r] = idx < n ? fabsf(to_f32(row[idx])) : 0.0f;
    }
    for (int64_t base = 0; base < n; base += kSumTile) {
      float nxt[kSumPer];
#pragma unroll
      for (int r = 0; r < kSumPer; ++r) {
        tile[t + 1024 * r] = cur[r];
        mx = fmaxf(mx, cur[r]);
        const int64_t idx = base + kSumTile + t + 1024 * r;
        nxt[r] = idx < n ? fabsf(to_f32(row[idx])) : 0.0f;
      }
      __syncthreads();
      if (t < 256) {
        const int64_t len = (n - base) < kSumTile ? (n - base) : kSumTile;
#pragma unroll
        for (int j = 0; j < kSumTile / 256; ++j) {
          const int idx = t + 256 * j;
          if (idx < len) acc = __fadd_rn(acc, tile[idx]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kSumPer; ++r) cur[r] = nxt[r];
    }
    if (t < 256) part[t] = acc;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, off));
    if (lane == 0 && mx > 0.0f) atomicMax(&sc->maxb_bits, __float_as_uint(mx));
    __syncthreads();
    for (int h = 128; h >= 1; h >>= 1) {
      if (t < h) part[t] = __fadd_rn(part[t], part[t + h]);
      __syncthreads();
    }
    total = part[0];
    if (t == 0) nb[k] = total;
  }
  if (Part == 1) return;

  uint32_t* __restrict__ out = TB + k * n;
  const int e = total > 0.0f ? 29 - ilogb_pos(total) : 0;
  const bool plain = e >= -126 && e <= 127;   // one exact scaling per entry
  const float scale = plain ? pow2f(e) : 0.0f;
  float v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int64_t idx = 4 * t + c;
    v[c] = idx < n ? to_f32(row[idx]) : 0.0f;
  }
  uint32_t carry = 0;
  for (int64_t base = 0; base < n; base += kTileB) {
    float vn[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t idx = base + kTileB + 4 * t + c;
      vn[c] = idx < n ? to_f32(row[idx]) : 0.0f;
    }
    uint32_t q[4], local = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t idx = base + 4 * t + c;
      if (idx < n && total > 0.0f) {
        const float w = fabsf(v[c]);
        uint32_t qv;
        if (plain) {
          qv = (uint32_t)__float2int_rn(__fmul_rn(w, scale));   // at most the sum: < 2^30
          qv += (w > 0.0f && qv == 0u) ? 1u : 0u;
        } else {
          qv = quantize_row(w, e);
        }
        local += qv;
      }
      q[c] = local;
    }
    const uint32_t inc = warp_inclusive_u32(local, lane);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const uint32_t x = wsum[lane];
      const uint32_t xi = warp_inclusive_u32(x, lane);
      wsum[lane] = xi - x;
      if (lane == 31) wsum[32] = xi;
    }
    __syncthreads();
    const uint32_t off = carry + wsum[warp] + inc - local;
    carry += wsum[32];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t idx = base + 4 * t + c;
      if (idx < n) out[idx] = (off + q[c]) | (v[c] < 0.0f ? SIGN_BIT : 0u);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = vn[c];
  }
}

// ---------------------------------------------------------------------------
// Rows of dense A: ||a_i*||_1, s_i, r_i, T2, TA.  One warp per row; the
// 256 canonical partials live 8 per lane (partial L + 32c in slot c).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_a_rows_dense(const T* __restrict__ A, int64_t m, int64_t d, int64_t lda,
               const float* __restrict__ nb_g, float* __restrict__ na_out,
               float* __restrict__ r_out, uint32_t* __restrict__ T2, uint32_t* __restrict__ TA,
               DevScalars* sc) {
  extern __shared__ float nb[];
  for (int64_t idx = threadIdx.x; idx < d; idx += blockDim.x) nb[idx] = nb_g[idx];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  float rmax = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * warps + warp; i < m; i += (int64_t)gridDim.x * warps) {
    const T* __restrict__ row = A + i * lda;
    float pa[8], ps[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) pa[c] = ps[c] = 0.0f;
    for (int64_t base = 0; base < d; base += 256) {
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t idx = base + lane + 32 * c;
        if (idx < d) {
          const float a = fabsf(to_f32(row[idx]));
          pa[c] = __fadd_rn(pa[c], a);
          ps[c] = __fadd_rn(ps[c], __fmul_rn(a, nb[idx]));
        }
      }
    }
    // Fold halves: 128 and 64 and 32 inside the lane, 16..1 across lanes.
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pa[c] = __fadd_rn(pa[c], pa[c + 4]);
      ps[c] = __fadd_rn(ps[c], ps[c + 4]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      pa[c] = __fadd_rn(pa[c], pa[c + 2]);
      ps[c] = __fadd_rn(ps[c], ps[c + 2]);
    }
    float na = __fadd_rn(pa[0], pa[1]);
    float s = __fadd_rn(ps[0], ps[1]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      na = __fadd_rn(na, __shfl_xor_sync(0xFFFFFFFFu, na, off));
      s = __fadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
    }
    const float r = __fmul_rn(na, s);
    if (lane == 0) {
      na_out[i] = na;
      r_out[i] = r;
    }
    rmax = fmaxf(rmax, r);

    const bool live = s > 0.0f;
    const int e2 = live ? 29 - ilogb_pos(s) : 0;
    const int ea = live ? 29 - ilogb_pos(na) : 0;
    uint32_t* __restrict__ o2 = T2 + i * d;
    uint32_t* __restrict__ oa = TA + i * d;
    uint32_t c2 = 0, ca = 0;
    for (int64_t base = 0; base < d; base += 32) {
      const int64_t idx = base + lane;
      uint32_t q2 = 0, qa = 0, sg = 0;
      if (idx < d) {
        const float v = to_f32(row[idx]);
        const float a = fabsf(v);
        if (live) {
          q2 = quantize_row(__fmul_rn(a, nb[idx]), e2);
          qa = quantize_row(a, ea);
        }
        sg = v < 0.0f ? SIGN_BIT : 0u;
      }
      const uint32_t i2 = warp_inclusive_u32(q2, lane);
      const uint32_t ia = warp_inclusive_u32(qa, lane);
      if (idx < d) {
        o2[idx] = (c2 + i2) | sg;
        oa[idx] = (ca + ia) | sg;
      }
      c2 += __shfl_sync(0xFFFFFFFFu, i2, 31);
      ca += __shfl_sync(0xFFFFFFFFu, ia, 31);
    }
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1)
    rmax = fmaxf(rmax, __shfl_xor_sync(0xFFFFFFFFu, rmax, off));
  if (lane == 0 && rmax > 0.0f) atomicMax(&sc->maxr_bits, __float_as_uint(rmax));
}

// Rows of dense A with d <= 32 NC <= 256, the same results as
// k_a_rows_dense: each canonical partial then holds at most one entry, so
// lane L keeps entries L + 32c (c < NC) in registers for both the sums and
// the tables.  The next row's entries are loaded before the current row is
// processed; the prefix scans take the entries in consecutive runs of NC
// per lane (through shared memory) and the tables are written 16 bytes at a
// time where the rows allow.
template <typename T, int NC>
__global__ void __launch_bounds__(256)
k_a_rows_short(const T* __restrict__ A, int64_t m, int d, int64_t lda,
               const float* __restrict__ nb_g, float* __restrict__ na_out,
               float* __restrict__ r_out, uint32_t* __restrict__ T2, uint32_t* __restrict__ TA,
               DevScalars* sc) {
  __shared__ float nb[32 * NC];
  __shared__ __align__(16) uint32_t scan_buf[8][2][32 * NC];   // per warp: T2, TA entries
  for (int idx = threadIdx.x; idx < 32 * NC; idx += blockDim.x) nb[idx] = idx < d ? nb_g[idx] : 0.0f;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  uint32_t* const w2 = scan_buf[threadIdx.x >> 5][0];
  uint32_t* const wa = scan_buf[threadIdx.x >> 5][1];
  const int64_t stride = (int64_t)gridDim.x * (blockDim.x >> 5);
  int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float v[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int idx = lane + 32 * c;
    v[c] = (i < m && idx < d) ? to_f32(A[i * lda + idx]) : 0.0f;
  }
  float rmax = 0.0f;
  for (; i < m; i += stride) {
    const int64_t inext = i + stride;
    float vn[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int idx = lane + 32 * c;
      vn[c] = (inext < m && idx < d) ? to_f32(A[inext * lda + idx]) : 0.0f;
    }
    // Partials 0..255 in slots c < 8 (slot c holds partial lane + 32c; the
    // slots at and above NC hold empty partials, exactly 0), folded in
    // halves as in k_a_rows_dense.
    float pa[8], ps[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (c < NC) {
        const float a = fabsf(v[c]);
        pa[c] = __fadd_rn(0.0f, a);
        ps[c] = __fadd_rn(0.0f, __fmul_rn(a, nb[lane + 32 * c]));
      } else {
        pa[c] = 0.0f;
        ps[c] = 0.0f;
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      pa[c] = __fadd_rn(pa[c], pa[c + 4]);
      ps[c] = __fadd_rn(ps[c], ps[c + 4]);
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      pa[c] = __fadd_rn(pa[c], pa[c + 2]);
      ps[c] = __fadd_rn(ps[c], ps[c + 2]);
    }
    float na = __fadd_rn(pa[0], pa[1]);
    float s = __fadd_rn(ps[0], ps[1]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
      na = __fadd_rn(na, __shfl_xor_sync(0xFFFFFFFFu, na, off));
      s = __fadd_rn(s, __shfl_xor_sync(0xFFFFFFFFu, s, off));
    }
    const float r = __fmul_rn(na, s);
    if (lane == 0) {
      na_out[i] = na;
      r_out[i] = r;
    }
    rmax = fmaxf(rmax, r);
    const bool live = s > 0.0f;
    const int e2 = live ? 29 - ilogb_pos(s) : 0;
    const int ea = live ? 29 - ilogb_pos(na) : 0;
    // Both exponents inside the normal range: one exact power-of-two
    // scaling per entry (what quantize_row does in that range).
    const bool plain = e2 >= -126 && e2 <= 127 && ea >= -126 && ea <= 127;
    const float s2 = plain ? pow2f(e2) : 0.0f, sa = plain ? pow2f(ea) : 0.0f;
    uint32_t i2[NC], ia[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int idx = lane + 32 * c;
      uint32_t q2 = 0, qa = 0;
      if (live && idx < d) {
        const float a = fabsf(v[c]);
        const float w2 = __fmul_rn(a, nb[idx]);
        if (plain) {
          // 32-bit conversions: an entry is at most its row's sum, which the
          // scaling puts below 2^30.
          q2 = (uint32_t)__float2int_rn(__fmul_rn(w2, s2));
          qa = (uint32_t)__float2int_rn(__fmul_rn(a, sa));
          q2 += (w2 > 0.0f && q2 == 0u) ? 1u : 0u;
          qa += (a > 0.0f && qa == 0u) ? 1u : 0u;
        } else {
          q2 = quantize_row(w2, e2);
          qa = quantize_row(a, ea);
        }
      }
      i2[c] = q2;
      ia[c] = qa;
    }
    // The scans run over consecutive entries: the warp's entries (sign in
    // bit 31, every quantised weight is below 2^31) pass through shared
    // memory so that lane L holds entries NC L ... NC L + NC - 1, scans them
    // in registers and adds the exclusive prefix of the lane totals (one
    // warp scan per table).  Integer sums: the order changes nothing.
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const uint32_t sg = v[c] < 0.0f ? SIGN_BIT : 0u;
      w2[lane + 32 * c] = i2[c] | sg;
      wa[lane + 32 * c] = ia[c] | sg;
    }
    __syncwarp();
    uint32_t e2v[NC], eav[NC];
    if constexpr (NC % 4 == 0) {
#pragma unroll
      for (int c = 0; c < NC; c += 4) {
        const uint4 x2 = *(const uint4*)(w2 + NC * lane + c);
        const uint4 xa = *(const uint4*)(wa + NC * lane + c);
        e2v[c] = x2.x; e2v[c + 1] = x2.y; e2v[c + 2] = x2.z; e2v[c + 3] = x2.w;
        eav[c] = xa.x; eav[c + 1] = xa.y; eav[c + 2] = xa.z; eav[c + 3] = xa.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        e2v[c] = w2[NC * lane + c];
        eav[c] = wa[NC * lane + c];
      }
    }
    __syncwarp();
    uint32_t run2 = 0, runa = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      run2 += e2v[c] & ~SIGN_BIT;
      runa += eav[c] & ~SIGN_BIT;
    }
    uint32_t inc2 = run2, inca = runa;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t o2 = __shfl_up_sync(0xFFFFFFFFu, inc2, off);
      const uint32_t oa = __shfl_up_sync(0xFFFFFFFFu, inca, off);
      if (lane >= off) {
        inc2 += o2;
        inca += oa;
      }
    }
    run2 = inc2 - run2;
    runa = inca - runa;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      run2 += e2v[c] & ~SIGN_BIT;
      runa += eav[c] & ~SIGN_BIT;
      e2v[c] = run2 | (e2v[c] & SIGN_BIT);
      eav[c] = runa | (eav[c] & SIGN_BIT);
    }
    uint32_t* __restrict__ o2 = T2 + i * d;
    uint32_t* __restrict__ oa = TA + i * d;
    const int first = NC * lane;
    if (NC % 4 == 0 && (d & 3) == 0) {   // rows start on 16 bytes
#pragma unroll
      for (int c = 0; c < NC; c += 4) {
        if (first + c < d) {   // d a multiple of 4: all four entries exist
          *(uint4*)(o2 + first + c) = make_uint4(e2v[c], e2v[c + 1], e2v[c + 2], e2v[c + 3]);
          *(uint4*)(oa + first + c) = make_uint4(eav[c], eav[c + 1], eav[c + 2], eav[c + 3]);
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (first + c < d) {
          o2[first + c] = e2v[c];
          oa[first + c] = eav[c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = vn[c];
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1)
    rmax = fmaxf(rmax, __shfl_xor_sync(0xFFFFFFFFu, rmax, off));
  if (lane == 0 && rmax > 0.0f) atomicMax(&sc->maxr_bits, __float_as_uint(rmax));
}

// ---------------------------------------------------------------------------
// Rows of 0/1 CSR A (integer mode): T2 = prefix of deg_k^B, r_i.
// ---------------------------------------------------------------------------
// Rows of at most kShortRow entries (most rows of a sparse graph) are
// taken one per lane, their entries' weights loaded eight at a time; the
// warp then works through its lanes' longer rows together.  Lane l of warp
// w (of W) takes rows w + l W + 32 W k, so that heavy rows with neighbouring
// indices (generators often number nodes by weight) go to different warps.
// A warp per row, as for the long rows, spent a chain of dependent loads on
// every short row in turn.
constexpr int64_t kShortRow = 32;

__global__ void __launch_bounds__(256)
k_a_rows_binary(const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_col,
                const int64_t* __restrict__ b_ptr, int64_t m, uint32_t* __restrict__ T2,
                unsigned long long* __restrict__ r64, DevScalars* sc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool over = false;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t base = 0; base < m; base += warps * 32) {
    const int64_t i = base + (int64_t)lane * warps + w;
    int64_t a0 = 0, a1 = 0;
    if (i < m) {
      a0 = a_ptr[i];
      a1 = a_ptr[i + 1];
    }
    const bool longrow = a1 - a0 > kShortRow;
    if (i < m && !longrow) {
      unsigned long long acc = 0;
      for (int64_t e0 = a0; e0 < a1; e0 += 8) {
        unsigned long long q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          q[u] = 0;
          if (e0 + u < a1) {
            const int32_t k = a_col[e0 + u];
            q[u] = (unsigned long long)(b_ptr[k + 1] - b_ptr[k]);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (e0 + u < a1) {
            acc += q[u];
            if (acc > 0xFFFFFFFFull) over = true;
            T2[e0 + u] = (uint32_t)acc;
          }
        }
      }
      r64[i] = (unsigned long long)(a1 - a0) * acc;
    }
    unsigned lm = __ballot_sync(0xFFFFFFFFu, i < m && longrow);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int64_t r0 = __shfl_sync(0xFFFFFFFFu, a0, src), r1 = __shfl_sync(0xFFFFFFFFu, a1, src);
      unsigned long long carry = 0;
      for (int64_t b = r0; b < r1; b += 32) {
        const int64_t e = b + lane;
        unsigned long long q = 0;
        if (e < r1) {
          const int32_t k = a_col[e];
          q = (unsigned long long)(b_ptr[k + 1] - b_ptr[k]);
        }
        const unsigned long long inc = warp_inclusive_u64(q, lane) + carry;
        if (e < r1) {
          if (inc > 0xFFFFFFFFull) over = true;
          T2[e] = (uint32_t)inc;
        }
        carry = __shfl_sync(0xFFFFFFFFu, inc, 31);
      }
      if (lane == 0) r64[base + (int64_t)src * warps + w] = (unsigned long long)(r1 - r0) * carry;
    }
  }
  if (__any_sync(0xFFFFFFFFu, over) && lane == 0) atomicOr(&sc->err, DERR_OVERFLOW);
}

// ---------------------------------------------------------------------------
// Guides of long 0/1 T2 rows.  Row i (L >= kGuideMin entries, total tot)
// gets buckets of width 2^sh, sh the smallest shift leaving at most about
// L/4 buckets, and nb + 1 guide entries: entry b is the number of the row's
// prefix entries below b << sh, so the first entry above a target t lies
// between guide entries t >> sh and (t >> sh) + 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int bitlen_u32(uint32_t x) { return x ? 32 - __clz(x) : 0; }

__global__ void __launch_bounds__(256)
k_guide_sizes(const int64_t* __restrict__ a_ptr, const uint32_t* __restrict__ T2, int64_t m,
              unsigned long long* __restrict__ sizes, uint8_t* __restrict__ shift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a0 = a_ptr[i], len = a_ptr[i + 1] - a0;
    unsigned long long size = 0;
    int sh = 0;
    if (len >= kGuideMin) {
      const uint32_t tot = T2[a0 + len - 1];
      if (tot > 0) {
        const int want = bitlen_u32((uint32_t)(len / 8));
        sh = bitlen_u32(tot - 1) - want;
        if (sh < 0) sh = 0;
        size = (unsigned long long)((tot - 1) >> sh) + 2;   // nb + 1
      }
    }
    sizes[i] = size;
    shift[i] = (uint8_t)sh;
  }
}

__global__ void __launch_bounds__(256)
k_guide_fill(const int64_t* __restrict__ a_ptr, const uint32_t* __restrict__ T2, int64_t m,
             const unsigned long long* __restrict__ gptr, const uint8_t* __restrict__ shift,
             uint32_t* __restrict__ G) {
  // A warp looks at 32 rows at once (lane l of warp w of W: rows
  // w + l W + 32 W k) and fills the guides of those that have one together.
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t base = 0; base < m; base += warps * 32) {
    const int64_t r = base + (int64_t)lane * warps + w;
    unsigned long long g0r = 0, nr = 0;
    if (r < m) {
      g0r = gptr[r];
      nr = gptr[r + 1] - g0r;
    }
    unsigned gm = __ballot_sync(0xFFFFFFFFu, nr != 0);
    while (gm) {
      const int src = __ffs(gm) - 1;
      gm &= gm - 1;
      const int64_t i = base + (int64_t)src * warps + w;
      const unsigned long long g0 = __shfl_sync(0xFFFFFFFFu, g0r, src);
      const unsigned long long n = __shfl_sync(0xFFFFFFFFu, nr, src);
      const int64_t a0 = a_ptr[i], len = a_ptr[i + 1] - a0;
      const int sh = shift[i];
      for (unsigned long long b = lane; b < n; b += 32) {
        const unsigned long long thr = b << sh;   // count the entries below thr
        uint32_t cnt;
        if (thr == 0) cnt = 0;
        else if (thr > 0xFFFFFFFFull) cnt = (uint32_t)len;
        else cnt = (uint32_t)ub_u32(T2 + a0, (int)len, (uint32_t)(thr - 1), 0xFFFFFFFFu);
        G[g0 + b] = cnt;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// T1: scale exponent, per-chunk sums, chunk offsets, inclusive prefix.
// ---------------------------------------------------------------------------
constexpr int T1_CHUNK = 2048;  // 256 threads x 8 elements

__device__ __forceinline__ int t1_exponent(const DevScalars* sc, int clog2m) {
  const float maxr = __uint_as_float(sc->maxr_bits);
  return 62 - clog2m - (ilogb_pos(maxr) + 1);
}

__device__ __forceinline__ unsigned long long t1_weight(const float* r, const unsigned long long* r64,
                                                        int64_t i, int e1) {
  if (r64) return r64[i];
  const float v = r[i];
  unsigned long long q = (unsigned long long)fixed_point(v, e1);
  if (v > 0.0f && q == 0ull) q = 1ull;
  return q;
}

__global__ void __launch_bounds__(256)
k_t1_chunk_sums(const float* __restrict__ r, const unsigned long long* __restrict__ r64,
                int64_t m, int clog2m, unsigned long long* __restrict__ partial, DevScalars* sc) {
  __shared__ unsigned long long warp_tot[9];
  int scale = 0;
  if (!r64) {
    if (sc->maxr_bits == 0u) return;  // ||W||_1 == 0, reported by the host
    scale = t1_exponent(sc, clog2m);
  }
  const int64_t base = (int64_t)blockIdx.x * T1_CHUNK + threadIdx.x * 8;
  unsigned long long acc = 0;
  bool over = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t i = base + c;
    if (i < m) {
      const unsigned long long q = t1_weight(r, r64, i, scale);
      const unsigned long long nx = acc + q;
      if (nx < acc || q >= (1ull << 63)) over = true;
      acc = nx;
    }
  }
  unsigned long long total;
  // 256 values of at most 2^63 each: detect wrap on the chunk sum.
  const unsigned long long excl = block_exclusive_u64(acc, warp_tot, &total);
  if (over || excl + acc < excl) atomicOr(&sc->err, DERR_OVERFLOW);
  if (threadIdx.x == 255 && total < excl) atomicOr(&sc->err, DERR_OVERFLOW);
  if (threadIdx.x == 0) partial[blockIdx.x] = total;
  if (blockIdx.x == 0 && threadIdx.x == 0 && !r64) sc->e1 = t1_exponent(sc, clog2m);
}

// One warp: exclusive offsets of the chunk totals and T1's total, then the
// scalars the sampler derives from it: the bucket shifts of T1's guide
// (about 2^bl_m buckets) and of the row-order sort (at most 2^lgm buckets),
// and F = 62 - lg_s - (floor(log2 max |b|) + 1) for dense inputs.  The
// total is exact when below 2^63: the high and low 32-bit halves of the
// chunk totals are summed separately to detect a larger one.
__global__ void k_t1_chunk_offsets(unsigned long long* __restrict__ partial, int64_t chunks,
                                   int bl_m, int lgm, int lg_s, int dense, DevScalars* sc) {
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32 || blockIdx.x != 0) return;
  unsigned long long carry = 0, hi = 0, lo = 0;
  for (int64_t base = 0; base < chunks; base += 32) {
    const int64_t b = base + lane;
    const unsigned long long v = b < chunks ? partial[b] : 0ull;
    hi += v >> 32;
    lo += v & 0xFFFFFFFFull;
    const unsigned long long inc = warp_inclusive_u64(v, lane) + carry;
    if (b < chunks) partial[b] = inc - v;
    carry = __shfl_sync(0xFFFFFFFFu, inc, 31);
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    hi += __shfl_xor_sync(0xFFFFFFFFu, hi, off);
    lo += __shfl_xor_sync(0xFFFFFFFFu, lo, off);
  }
  if (lane != 0) return;
  const unsigned long long acc = carry;
  if (hi + (lo >> 32) >= (1ull << 31)) atomicOr(&sc->err, DERR_OVERFLOW);
  if (acc == 0ull) atomicOr(&sc->err, DERR_EMPTY);
  sc->t1_total = acc;
  const int bl_t = acc > 1ull ? 64 - __clzll((long long)(acc - 1)) : 0;
  sc->t1g_sh = bl_t > bl_m ? bl_t - bl_m : 0;
  sc->sort_shift = bl_t > lgm ? bl_t - lgm : 0;
  int f = 0;
  if (dense) {
    if (sc->maxb_bits == 0u || sc->maxr_bits == 0u) atomicOr(&sc->err, DERR_EMPTY);
    else f = 62 - lg_s - (ilogb_pos(__uint_as_float(sc->maxb_bits)) + 1);
  }
  sc->f_exp = f;
}

__global__ void __launch_bounds__(256)
k_t1_write(const float* __restrict__ r, const unsigned long long* __restrict__ r64, int64_t m,
           int clog2m, const unsigned long long* __restrict__ offset, uint64_t* __restrict__ T1,
           const DevScalars* sc) {
  __shared__ unsigned long long warp_tot[9];
  int scale = 0;
  if (!r64) {
    if (sc->maxr_bits == 0u) return;
    scale = t1_exponent(sc, clog2m);
  }
  const int64_t base = (int64_t)blockIdx.x * T1_CHUNK + threadIdx.x * 8;
  unsigned long long q[8], acc = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t i = base + c;
    q[c] = (i < m) ? t1_weight(r, r64, i, scale) : 0ull;
    acc += q[c];
    q[c] = acc;
  }
  unsigned long long total;
  const unsigned long long excl = block_exclusive_u64(acc, warp_tot, &total);
  const unsigned long long off = offset[blockIdx.x] + excl;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int64_t i = base + c;
    if (i < m) T1[i] = off + q[c];
  }
}

// Dense B (d x n) to B^T (n x d) for coalesced rescoring.
template <typename T>
__global__ void k_transpose(const T* __restrict__ B, int64_t d, int64_t n, int64_t ldb,
                            T* __restrict__ Bt) {
  __shared__ T tile[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, j = j0 + threadIdx.x;
    if (k < d && j < n) tile[r][threadIdx.x] = B[k * ldb + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, k = k0 + threadIdx.x;
    if (k < d && j < n) Bt[j * d + k] = tile[threadIdx.x][r];
  }
}

// Home-region size of row i: the smallest power of two >= factor x the
// row's expected number of diamonds among s_max (factor 1.5 unless a test
// asks for less), at least 4 (every region starts on a 4-slot group).
__global__ void __launch_bounds__(256)
k_region_sizes(const uint64_t* __restrict__ T1, int64_t m, unsigned long long s_max, float factor,
               const DevScalars* sc, unsigned long long* __restrict__ sizes) {
  const float scale = factor * ((float)s_max / (float)(sc->t1_total ? sc->t1_total : 1ull));
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long q = T1[i] - (i ? T1[i - 1] : 0ull);
    const float want = (float)q * scale;
    // smallest power of two >= want, between 2^2 and 2^40
    int e = 2;
    if (want > 4.0f) {
      const uint32_t b = __float_as_uint(want);
      e = (int)((b >> 23) & 0xFF) - 127 + ((b & 0x7FFFFF) ? 1 : 0);
      e = e < 40 ? e : 40;
    }
    sizes[i] = 1ull << e;
  }
}

// hreg[m+1] = hreg[m] + the overflow table's slots.
__global__ void k_overflow_end(unsigned long long* hreg_m, unsigned long long hov) {
  if (threadIdx.x == 0) hreg_m[1] = hreg_m[0] + hov;
}

int ceil_log2_host(uint64_t x) {
  int e = 0;
  while (e < 64 && (1ull << e) < x) ++e;
  return e;
}

template <typename T>
void launch_b_rows(mad_ctx* ctx, cudaStream_t st, cudaStream_t table_st = nullptr) {
  if (ctx->n >= 8192 && table_st) {   // sums on st, then the table on table_st
    k_b_rows_wide<T, 1><<<(unsigned)ctx->d, 1024, 0, st>>>(
        (const T*)ctx->B.values, ctx->n, ctx->B.ld, ctx->nb, ctx->TB, ctx->sc);
    cudaEventRecord(ctx->ev_fork2, st);
    cudaStreamWaitEvent(table_st, ctx->ev_fork2, 0);
    k_b_rows_wide<T, 2><<<(unsigned)ctx->d, 1024, 0, table_st>>>(
        (const T*)ctx->B.values, ctx->n, ctx->B.ld, ctx->nb, ctx->TB, ctx->sc);
    count_launch(ctx, 2);
    return;
  }
  if (ctx->n >= 8192) {
    k_b_rows_wide<T, 0><<<(unsigned)ctx->d, 1024, 0, st>>>(
        (const T*)ctx->B.values, ctx->n, ctx->B.ld, ctx->nb, ctx->TB, ctx->sc);
  } else {
    k_b_rows_dense<T><<<(unsigned)ctx->d, 256, 0, st>>>((const T*)ctx->B.values, ctx->n,
                                                         ctx->B.ld, ctx->nb, ctx->TB, ctx->sc);
  }
  count_launch(ctx);
}

template <typename T>
void launch_a_rows(mad_ctx* ctx, cudaStream_t st) {
  const int64_t blocks64 = (ctx->m + 7) / 8;
  const unsigned blocks = (unsigned)(blocks64 < 152 * 16 ? blocks64 : 152 * 16);
  if (ctx->d <= 256) {
    const T* A = (const T*)ctx->A.values;
    const int d = (int)ctx->d;
    switch ((d + 31) / 32) {
#define MAD_A_ROWS_SHORT(NC)                                                                    \
  case NC:                                                                                      \
    k_a_rows_short<T, NC><<<blocks, 256, 0, st>>>(A, ctx->m, d, ctx->A.ld, ctx->nb, ctx->na,   \
                                                  ctx->r, ctx->T2, ctx->TA, ctx->sc);           \
    break;
      MAD_A_ROWS_SHORT(1) MAD_A_ROWS_SHORT(2) MAD_A_ROWS_SHORT(3) MAD_A_ROWS_SHORT(4)
      MAD_A_ROWS_SHORT(5) MAD_A_ROWS_SHORT(6) MAD_A_ROWS_SHORT(7) MAD_A_ROWS_SHORT(8)
#undef MAD_A_ROWS_SHORT
    }
    count_launch(ctx);
    return;
  }
  k_a_rows_dense<T><<<blocks, 256, (size_t)ctx->d * sizeof(float), st>>>(
      (const T*)ctx->A.values, ctx->m, ctx->d, ctx->A.ld, ctx->nb, ctx->na, ctx->r, ctx->T2,
      ctx->TA, ctx->sc);
  count_launch(ctx);
}

template <typename T>
void launch_transpose(mad_ctx* ctx, cudaStream_t st) {
  dim3 grid((unsigned)((ctx->n + 31) / 32), (unsigned)((ctx->d + 31) / 32));
  k_transpose<T><<<grid, dim3(32, 8), 0, st>>>((const T*)ctx->B.values, ctx->d, ctx->n,
                                               ctx->B.ld, (T*)ctx->bt);
  count_launch(ctx);
}

}  // namespace

// Each region holds at most max(4, 2 x 1.5 x its expected diamonds) slots,
// the expectation taken in FP32 (relative error below 2^-20).
uint64_t hash_region_bound(uint64_t m, uint64_t s_max) {
  return 4 * m + 3 * s_max + (s_max >> 18) + 16;
}

mad_status t2_guide_offsets(mad_ctx* ctx, cudaStream_t st) {
  const uint64_t m = (uint64_t)ctx->m;
  const size_t sizes_bytes = (m * sizeof(unsigned long long) + 255) & ~(size_t)255;
  mad_status rs = ensure_scratch(ctx, sizes_bytes + scan_partial_elems(m) * 8, st);
  if (rs != MAD_OK) return rs;
  unsigned long long* sizes = (unsigned long long*)ctx->scratch;
  uint64_t* part = (uint64_t*)((char*)ctx->scratch + sizes_bytes);
  const unsigned blocks = (unsigned)((m + 255) / 256 < 152 * 8 ? (m + 255) / 256 : 152 * 8);
  k_guide_sizes<<<blocks, 256, 0, st>>>(ctx->A.rowptr, ctx->T2, ctx->m, sizes, ctx->T2g_sh);
  count_launch(ctx);
  return scan_exclusive_u64(ctx, (const uint64_t*)sizes, (uint64_t*)ctx->T2g_ptr, m, part, st);
}

// One warp per row of the closure matrix; every entry (row, col) sets its
// five bits.
__global__ void __launch_bounds__(256)
k_bloom_build(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col, int64_t rows,
              int shift, unsigned long long* __restrict__ words) {
  // Short rows one per lane, longer ones by the whole warp (lane l of warp
  // w of W: rows w + l W + 32 W k).
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t base = 0; base < rows; base += warps * 32) {
    const int64_t r = base + (int64_t)lane * warps + w;
    int64_t e0 = 0, e1 = 0;
    if (r < rows) {
      e0 = ptr[r];
      e1 = ptr[r + 1];
    }
    const bool longrow = e1 - e0 > 32;
    if (r < rows && !longrow) {
      for (int64_t e = e0; e < e1; ++e) {
        const unsigned long long h = mix64(((unsigned long long)r << 32) | (uint32_t)col[e]);
        atomicOr(words + (h >> shift), bloom_bits(h));
      }
    }
    unsigned lm = __ballot_sync(0xFFFFFFFFu, r < rows && longrow);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const unsigned long long rr = (unsigned long long)(base + (int64_t)src * warps + w);
      const int64_t f0 = __shfl_sync(0xFFFFFFFFu, e0, src), f1 = __shfl_sync(0xFFFFFFFFu, e1, src);
      for (int64_t e = f0 + lane; e < f1; e += 32) {
        const unsigned long long h = mix64((rr << 32) | (uint32_t)col[e]);
        atomicOr(words + (h >> shift), bloom_bits(h));
      }
    }
  }
}

mad_status build_bloom(mad_ctx* ctx, cudaStream_t st) {
  const bool gram = (ctx->flags & MAD_GRAM) != 0;
  const int64_t* ptr = gram ? ctx->A.rowptr : ctx->B.rowptr;
  const int32_t* col = gram ? ctx->A.colidx : ctx->B.colidx;
  const int64_t rows = gram ? ctx->m : ctx->d;
  cudaMemsetAsync(ctx->bloom, 0, (sizeof(unsigned long long) << ctx->bloom_lg), st);
  const int64_t blocks64 = (rows + 7) / 8;
  const unsigned blocks = (unsigned)(blocks64 < 152 * 16 ? blocks64 : 152 * 16);
  k_bloom_build<<<blocks, 256, 0, st>>>(ptr, col, rows, 64 - ctx->bloom_lg, ctx->bloom);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

// Guides of the dense TB rows: row k (n entries, masked total tot) gets
// buckets of width 2^sh, sh = max(0, bitlen(tot - 1) - W) with
// W = tb_guide_width(n), so it has nb = ((tot - 1) >> sh) + 1 <= 2^W
// buckets and its nb + 1 guide entries fit a fixed row stride 2^W + 1
// (no size pass, no host read-back).  Guide entry b is the first position
// whose prefix reaches b << sh.  Built by one pass over the entries: entry
// e writes the guide entries of the bucket starts its step (v_{e-1}, v_e]
// crosses; the last entry also stores the row's sh.
__global__ void __launch_bounds__(256)
k_tbg_fill(const uint32_t* __restrict__ TB, int64_t d, int64_t n, int W, int64_t stride,
           uint8_t* __restrict__ shift, uint32_t* __restrict__ G) {
  // Rows along grid dimension y, entries of a row along x (no division).
  for (int64_t k = blockIdx.y; k < d; k += gridDim.y) {
    const uint32_t* __restrict__ row = TB + k * n;
    const uint32_t tot = __ldg(row + n - 1) & PREFIX_MASK;
    int sh = tot ? bitlen_u32(tot - 1) - W : 0;
    sh = sh > 0 ? sh : 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) shift[k] = (uint8_t)sh;
    if (tot == 0) continue;
    const unsigned long long nb1 = (unsigned long long)((tot - 1) >> sh) + 2;   // nb + 1 entries
    uint32_t* __restrict__ g = G + k * stride;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      const unsigned long long v = row[e] & PREFIX_MASK;
      const unsigned long long b_hi = v >> sh;
      const unsigned long long b_lo = e ? ((unsigned long long)(row[e - 1] & PREFIX_MASK) >> sh) + 1 : 0;
      for (unsigned long long b = b_lo; b <= b_hi && b < nb1; ++b) g[b] = (uint32_t)e;
      if (e == n - 1)   // bucket starts past the last prefix: no entry reaches them
        for (unsigned long long b = b_hi + 1; b < nb1; ++b) g[b] = (uint32_t)n;
    }
  }
}

// Guide of T1 (one 64-bit prefix row), filled like the TB guides: entry e
// writes the guide entries of the bucket starts in (T1[e-1], T1[e]].
__global__ void __launch_bounds__(256)
k_t1g_fill(const uint64_t* __restrict__ T1, int64_t m, const DevScalars* sc,
           uint32_t* __restrict__ G) {
  const unsigned long long total = sc->t1_total;
  if (total == 0ull) return;
  const int sh = sc->t1g_sh;
  const unsigned long long nb1 = ((total - 1) >> sh) + 2;   // nb + 1 entries
  // Lane l of warp w of W takes entries w + l W + 32 W k; ranges of more
  // than 32 guide entries (the heaviest rows) are written by the whole warp.
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int64_t base = 0; base < m; base += warps * 32) {
    const int64_t e = base + (int64_t)lane * warps + w;
    unsigned long long b_lo = 0, b_end = 0;   // guide entries [b_lo, b_end) get e
    if (e < m) {
      const unsigned long long b_hi = T1[e] >> sh;
      b_lo = e ? (T1[e - 1] >> sh) + 1 : 0;
      b_end = b_hi + 1 < nb1 ? b_hi + 1 : nb1;
      if (e == m - 1) b_end = nb1;   // and every later one gets m
      if (b_end < b_lo) b_end = b_lo;
    }
    const bool wide = b_end - b_lo > 32;
    if (e < m && !wide) {
      const unsigned long long b_last = e == m - 1 ? ((T1[e] >> sh) + 1 < nb1 ? (T1[e] >> sh) + 1 : nb1) : b_end;
      for (unsigned long long b = b_lo; b < b_end; ++b) G[b] = b < b_last ? (uint32_t)e : (uint32_t)m;
    }
    unsigned wm = __ballot_sync(0xFFFFFFFFu, e < m && wide);
    while (wm) {
      const int src = __ffs(wm) - 1;
      wm &= wm - 1;
      const int64_t ee = base + (int64_t)src * warps + w;
      const unsigned long long lo = __shfl_sync(0xFFFFFFFFu, b_lo, src);
      const unsigned long long end = __shfl_sync(0xFFFFFFFFu, b_end, src);
      const unsigned long long hi_t = T1[ee] >> sh;
      const unsigned long long last = ee == m - 1 ? (hi_t + 1 < nb1 ? hi_t + 1 : nb1) : end;
      for (unsigned long long b = lo + lane; b < end; b += 32)
        G[b] = b < last ? (uint32_t)ee : (uint32_t)m;
    }
  }
}

// Empties the slots [*lo_dev, min(cap, *n_dev)) of the hash (keys to
// EMPTY_KEY, values to 0) with 16-byte stores.
__global__ void __launch_bounds__(256)
k_clear_slots(unsigned long long* __restrict__ keys, long long* __restrict__ vals, uint64_t cap,
              const unsigned long long* lo_dev, const unsigned long long* n_dev) {
  const uint64_t n = dev_len(cap, n_dev);
  uint64_t lo = lo_dev ? *lo_dev : 0;
  if (lo >= n) return;
  if (lo & 1) {   // an odd first slot alone, then 16-byte stores
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      keys[lo] = EMPTY_KEY;
      vals[lo] = 0;
    }
    ++lo;
  }
  const uint64_t stride = 2ull * gridDim.x * blockDim.x;
  for (uint64_t q = lo + 2ull * (blockIdx.x * blockDim.x + threadIdx.x); q < n; q += stride) {
    if (q + 1 < n) {
      *(ulonglong2*)(keys + q) = make_ulonglong2(EMPTY_KEY, EMPTY_KEY);
      *(longlong2*)(vals + q) = make_longlong2(0, 0);
    } else {
      keys[q] = EMPTY_KEY;
      vals[q] = 0;
    }
  }
}

mad_status clear_slots(mad_ctx* ctx, const unsigned long long* lo_dev,
                       const unsigned long long* hi_dev, cudaStream_t st) {
  const uint64_t bound = hash_slot_bound(ctx);
  const uint64_t blocks64 = (bound + 511) / 512;
  k_clear_slots<<<(unsigned)(blocks64 < 152 * 8 ? (blocks64 ? blocks64 : 1) : 152 * 8), 256, 0,
                  st>>>(ctx->hkeys, ctx->hvals, bound, lo_dev, hi_dev);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

int t1_guide_width(int64_t m) {
  int w = 0;
  while (w < 63 && (((uint64_t)m) >> w)) ++w;
  return w;
}

mad_status t1_guide_fill(mad_ctx* ctx, cudaStream_t st) {
  const int64_t blocks64 = (ctx->m + 255) / 256;
  k_t1g_fill<<<(unsigned)(blocks64 < 152 * 16 ? blocks64 : 152 * 16), 256, 0, st>>>(
      ctx->T1, ctx->m, ctx->sc, ctx->T1g);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

// About one bucket per entry (measured: the draws of the dense factor
// workload ran 0.05 ms faster than with n/8 buckets), but at most 2^17
// buckets per row once a row is long.
int tb_guide_width(int64_t n) {
  auto bitlen = [](uint64_t x) {
    int w = 0;
    while (w < 63 && (x >> w)) ++w;
    return w;
  };
  const int full = bitlen((uint64_t)(n > 0 ? n : 1));
  const int coarse = bitlen((uint64_t)(n / 8 > 0 ? n / 8 : 1));
  const int cap = coarse > 17 ? coarse : 17;
  return full < cap ? full : cap;
}

mad_status tb_guide_build(mad_ctx* ctx, cudaStream_t st) {
  const int W = tb_guide_width(ctx->n);
  const int64_t xblocks = (ctx->n + 1023) / 1024;   // four entries per thread
  const dim3 grid((unsigned)(xblocks < 64 ? xblocks : 64),
                  (unsigned)(ctx->d < 65535 ? ctx->d : 65535));
  k_tbg_fill<<<grid, 256, 0, st>>>(ctx->TB, ctx->d, ctx->n, W, ctx->tbg_stride, ctx->TBg_sh,
                                   ctx->TBg);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status build_item_tables(mad_ctx* ctx, cudaStream_t st) {
  launch_b_rows<float>(ctx, st);
  launch_transpose<float>(ctx, st);
  return cuda_status(cudaGetLastError());
}

mad_status build_query_rows(mad_ctx* ctx, cudaStream_t st) {
  launch_a_rows<float>(ctx, st);
  return cuda_status(cudaGetLastError());
}

mad_status t2_guide_fill(mad_ctx* ctx, cudaStream_t st) {
  const int64_t warps_needed = ctx->m;
  const int64_t blocks64 = (warps_needed + 7) / 8;
  const unsigned blocks = (unsigned)(blocks64 < 152 * 16 ? blocks64 : 152 * 16);
  k_guide_fill<<<blocks, 256, 0, st>>>(ctx->A.rowptr, ctx->T2, ctx->m, ctx->T2g_ptr, ctx->T2g_sh,
                                       ctx->T2g);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

mad_status build_hash_regions(mad_ctx* ctx, cudaStream_t st) {
  const uint64_t m = (uint64_t)ctx->m;
  const size_t sizes_bytes = (m * sizeof(unsigned long long) + 255) & ~(size_t)255;
  mad_status rs = ensure_scratch(ctx, sizes_bytes + scan_partial_elems(m) * 8, st);
  if (rs != MAD_OK) return rs;
  unsigned long long* sizes = (unsigned long long*)ctx->scratch;
  uint64_t* part = (uint64_t*)((char*)ctx->scratch + sizes_bytes);
  const unsigned blocks = (unsigned)((m + 255) / 256 < 152 * 8 ? (m + 255) / 256 : 152 * 8);
  k_region_sizes<<<blocks, 256, 0, st>>>(ctx->T1, ctx->m, ctx->s_max, ctx->region_factor, ctx->sc,
                                         sizes);
  count_launch(ctx);
  rs = scan_exclusive_u64(ctx, (const uint64_t*)sizes, (uint64_t*)ctx->hreg, m, part, st);
  if (rs != MAD_OK) return rs;
  k_overflow_end<<<1, 32, 0, st>>>(ctx->hreg + m, ctx->hov);
  count_launch(ctx);
  return cuda_status(cudaGetLastError());
}

uint64_t hash_overflow_slots(uint64_t s_max) {
  uint64_t o = 1ull << 14;
  while (o < (s_max >> 6)) o <<= 1;
  return o;
}

mad_status build_tables_impl(mad_ctx* ctx, cudaStream_t st, bool side_branch) {
  const int64_t chunks = (ctx->m + T1_CHUNK - 1) / T1_CHUNK;
  mad_status rs = ensure_scratch(ctx, (size_t)chunks * sizeof(unsigned long long), st);
  if (rs != MAD_OK) return rs;
  unsigned long long* partial = (unsigned long long*)ctx->scratch;
  const int clog2m = ceil_log2_host((uint64_t)ctx->m);

  if (ctx->integer) {
    const int64_t blocks64 = (ctx->m + 7) / 8;
    const unsigned blocks = (unsigned)(blocks64 < 152 * 16 ? blocks64 : 152 * 16);
    k_a_rows_binary<<<blocks, 256, 0, st>>>(ctx->A.rowptr, ctx->A.colidx, ctx->B.rowptr, ctx->m,
                                            ctx->T2, ctx->r64, ctx->sc);
    count_launch(ctx);
  } else {
    if (side_branch) {
      // Second stream: B^T at once (it needs only B), then, after B's row
      // sums, the TB table (wide rows) and its guides, beside the A rows
      // and T1 on st.  Narrow rows build TB with their sums on st.
      cudaStream_t sd = ctx->side;
      cudaEventRecord(ctx->ev_fork, st);
      cudaStreamWaitEvent(sd, ctx->ev_fork, 0);
      if (ctx->B.dt == MAD_F64) launch_transpose<double>(ctx, sd); else launch_transpose<float>(ctx, sd);
      if (ctx->B.dt == MAD_F64) launch_b_rows<double>(ctx, st, sd); else launch_b_rows<float>(ctx, st, sd);
      if (ctx->n < 8192) {
        cudaEventRecord(ctx->ev_fork2, st);
        cudaStreamWaitEvent(sd, ctx->ev_fork2, 0);
      }
      const mad_status gs = tb_guide_build(ctx, sd);
      if (gs != MAD_OK) return gs;
      cudaEventRecord(ctx->ev_join, sd);
    } else {
      if (ctx->B.dt == MAD_F64) launch_b_rows<double>(ctx, st); else launch_b_rows<float>(ctx, st);
      if (ctx->B.dt == MAD_F64) launch_transpose<double>(ctx, st); else launch_transpose<float>(ctx, st);
    }
    if (ctx->A.dt == MAD_F64) launch_a_rows<double>(ctx, st); else launch_a_rows<float>(ctx, st);
  }
  const float* r = ctx->integer ? nullptr : ctx->r;
  const unsigned long long* r64 = ctx->integer ? ctx->r64 : nullptr;
  k_t1_chunk_sums<<<(unsigned)chunks, 256, 0, st>>>(r, r64, ctx->m, clog2m, partial, ctx->sc);
  const int bl_m = t1_guide_width(ctx->m);
  k_t1_chunk_offsets<<<1, 32, 0, st>>>(partial, chunks, bl_m, sort_bits(ctx->m),
                                       ceil_log2_host(ctx->s_max), ctx->dense ? 1 : 0, ctx->sc);
  k_t1_write<<<(unsigned)chunks, 256, 0, st>>>(r, r64, ctx->m, clog2m, partial, ctx->T1, ctx->sc);
  count_launch(ctx, 3);
  return cuda_status(cudaGetLastError());
}

}  // namespace mad
