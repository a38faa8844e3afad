// Alias tables for constant-time draws (Sec. 4.1 names the alias method):
// built over the same integer weights as the prefix tables of Alg. 2 (the
// differences of consecutive prefix entries), so a draw from them follows
// exactly the same law.
//
// Construction: Vose's method in exact integers.  Over weights x_0..x_{n-1}
// with total X, column c starts with p_c = n x_c; columns below X are
// "small", the others "large", each kept as a stack filled in column order.
// The top small column s keeps itself with threshold t_s = p_s and takes the
// top large column l as its alias; l's weight becomes p_l - (X - p_s) and l
// is classified again.  Columns left at the end keep themselves (t = X).
// Then column c receives t_c + sum over columns aliased to it of (X - t_c'),
// which equals p_c = n x_c: P(c) = x_c / X exactly.
//
// One warp per table (a segment of up to kAliasSeg entries of a row, or a
// row's table over its segment totals): the lanes load the weights into the
// warp's shared memory and lane 0 runs the sequential method; rows of at
// most 128 entries of a 32-bit prefix table take one thread per table.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int kAliasWarps = 4;   // tables per 128-thread block

// Per-warp shared memory for a table of up to `cap` entries: p (PT), then
// the small and large stacks (16-bit column indices), rounded up to 16 bytes
// so that every warp's p stays 16-byte aligned.  PT is 128-bit for the
// 64-bit T1 weights and 64-bit for the 32-bit tables (their weights are
// below 2^31, a segment total below 2^41 and n <= 1024, so n x < 2^51).
template <typename PT>
__host__ __device__ constexpr size_t alias_warp_bytes(int cap) {
  return ((size_t)cap * (sizeof(PT) + 4) + 15) & ~(size_t)15;
}

// level 0: tables of the row segments, weights from a prefix table (u64
// entries when prefix64, else u32 entries whose bit 31 is masked off);
// level 1: tables over the segment totals of the rows with nseg > 1.
template <typename PT>
__global__ void __launch_bounds__(32 * kAliasWarps)
k_alias_build(const void* __restrict__ prefix, int prefix64, int64_t rows, int64_t L, int nseg,
              int level, int cap, AliasEnt* __restrict__ ent, unsigned long long* __restrict__ seg,
              unsigned long long* __restrict__ rowX) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* mine = sm + (size_t)w * alias_warp_bytes<PT>(cap);
  PT* p = reinterpret_cast<PT*>(mine);
  uint16_t* small = reinterpret_cast<uint16_t*>(mine + (size_t)cap * sizeof(PT));
  uint16_t* large = small + cap;
  const int64_t tasks = level == 0 ? rows * nseg : rows;
  const int64_t task = (int64_t)blockIdx.x * kAliasWarps + w;
  if (task >= tasks) return;
  const int64_t r = level == 0 ? task / nseg : task;
  const int64_t sg = level == 0 ? task % nseg : 0;
  const int64_t c0 = sg * kAliasSeg;
  const int n = level == 0 ? (int)(L - c0 < kAliasSeg ? L - c0 : kAliasSeg) : nseg;
  AliasEnt* out = ent + r * (L + nseg) + (level == 0 ? c0 : L);
  // Weights, and their total by a warp sum.
  unsigned long long part = 0;
  for (int c = lane; c < n; c += 32) {
    unsigned long long x;
    if (level == 1) {
      x = seg[r * nseg + c];
    } else if (prefix64) {
      const unsigned long long* P = (const unsigned long long*)prefix + r * L;
      const int64_t e = c0 + c;
      x = P[e] - (e ? P[e - 1] : 0ull);
    } else {
      const uint32_t* P = (const uint32_t*)prefix + r * L;
      const int64_t e = c0 + c;
      x = (unsigned long long)(P[e] & PREFIX_MASK) - (e ? (unsigned long long)(P[e - 1] & PREFIX_MASK) : 0ull);
    }
    p[c] = (PT)x * (PT)n;
    part += x;
  }
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, off);
  const unsigned long long X = part;
  __syncwarp();
  if (lane == 0) {
    int ns = 0, nl = 0;
    for (int c = 0; c < n; ++c) {
      if (p[c] < (PT)X) small[ns++] = (uint16_t)c;
      else large[nl++] = (uint16_t)c;
    }
    while (ns > 0 && nl > 0) {
      const int sc = small[--ns];
      const int lc = large[--nl];
      const unsigned long long ps = (unsigned long long)p[sc];
      AliasEnt e;
      e.t = ps;
      e.a = (uint32_t)lc;
      e.pad = 0;
      out[sc] = e;
      p[lc] -= (PT)(X - ps);
      if (p[lc] < (PT)X) small[ns++] = (uint16_t)lc;
      else large[nl++] = (uint16_t)lc;
    }
    AliasEnt keep;
    keep.t = X;
    keep.pad = 0;
    while (nl > 0) {
      keep.a = large[--nl];
      out[keep.a] = keep;
    }
    while (ns > 0) {
      keep.a = small[--ns];
      out[keep.a] = keep;
    }
    if (level == 0) {
      seg[r * nseg + sg] = X;
      if (nseg == 1) {
        rowX[r] = X;
        AliasEnt top;
        top.t = X;
        top.a = 0;
        top.pad = 0;
        ent[r * (L + nseg) + L] = top;
      }
    } else {
      rowX[r] = X;
    }
  }
}

// Short rows of a 32-bit prefix table (L <= kSmallAlias entries, one
// segment): one thread per table runs the same construction, in the same
// order, with 64-bit p (a weight is below 2^31 and n <= 128, so n x and X
// stay below 2^38).  A warp per table left 31 of its lanes idle while lane 0
// ran the sequential part.
constexpr int kSmallAlias = 128;
constexpr int kSmallThreads = 128;

// Per-thread shared memory: p (8 bytes per entry), then the small and large
// stacks (1 byte per entry); the stride is an odd number of 8-byte words so
// that the threads' p arrays start in different banks.
__host__ __device__ constexpr size_t small_alias_stride(int n) {
  return ((((size_t)n * 10 + 7) & ~(size_t)7) | 8);
}

__global__ void __launch_bounds__(kSmallThreads)
k_alias_build_small(const uint32_t* __restrict__ prefix, int64_t rows, int n,
                    AliasEnt* __restrict__ ent, unsigned long long* __restrict__ seg,
                    unsigned long long* __restrict__ rowX) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  unsigned char* mine = sm + (size_t)threadIdx.x * small_alias_stride(n);
  unsigned long long* p = reinterpret_cast<unsigned long long*>(mine);
  uint8_t* small = mine + (size_t)n * 8;
  uint8_t* large = small + n;
  const uint32_t* P = prefix + r * n;
  unsigned long long X = 0;
  uint32_t prev = 0;
  for (int c = 0; c < n; ++c) {
    const uint32_t cur = __ldg(P + c) & PREFIX_MASK;
    const unsigned long long x = (unsigned long long)(cur - prev);
    prev = cur;
    p[c] = x * (unsigned long long)n;
    X += x;
  }
  AliasEnt* out = ent + r * (n + 1);
  int ns = 0, nl = 0;
  for (int c = 0; c < n; ++c) {
    if (p[c] < X) small[ns++] = (uint8_t)c;
    else large[nl++] = (uint8_t)c;
  }
  while (ns > 0 && nl > 0) {
    const int sc = small[--ns];
    const int lc = large[--nl];
    const unsigned long long ps = p[sc];
    AliasEnt e;
    e.t = ps;
    e.a = (uint32_t)lc;
    e.pad = 0;
    out[sc] = e;
    p[lc] -= X - ps;
    if (p[lc] < X) small[ns++] = (uint8_t)lc;
    else large[nl++] = (uint8_t)lc;
  }
  AliasEnt keep;
  keep.t = X;
  keep.pad = 0;
  while (nl > 0) {
    keep.a = large[--nl];
    out[keep.a] = keep;
  }
  while (ns > 0) {
    keep.a = small[--ns];
    out[keep.a] = keep;
  }
  seg[r] = X;
  rowX[r] = X;
  AliasEnt top;
  top.t = X;
  top.a = 0;
  top.pad = 0;
  out[n] = top;
}

// The warp kernels of a family: level 0 over its row segments, then level
// 1 over the segment totals of rows with more than one segment.
template <typename PT>
void launch_warp_family(mad_ctx* ctx, int fam, const void* prefix, int prefix64, int64_t rows,
                        int64_t L, int64_t nseg, cudaStream_t st) {
  static size_t attr = 0;
  const int cap0 = (int)(L < kAliasSeg ? L : kAliasSeg);
  const size_t smem_max = kAliasWarps * alias_warp_bytes<PT>((int)kAliasSeg);
  if (attr < smem_max) {
    cudaFuncSetAttribute(k_alias_build<PT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_max);
    attr = smem_max;
  }
  const int64_t t0 = rows * nseg;
  k_alias_build<PT><<<(unsigned)((t0 + kAliasWarps - 1) / kAliasWarps), 32 * kAliasWarps,
                      kAliasWarps * alias_warp_bytes<PT>(cap0), st>>>(
      prefix, prefix64, rows, L, (int)nseg, 0, cap0, ctx->al[fam], ctx->al_seg[fam],
      ctx->al_row[fam]);
  count_launch(ctx);
  if (nseg > 1) {
    k_alias_build<PT><<<(unsigned)((rows + kAliasWarps - 1) / kAliasWarps), 32 * kAliasWarps,
                        kAliasWarps * alias_warp_bytes<PT>((int)nseg), st>>>(
        prefix, prefix64, rows, L, (int)nseg, 1, (int)nseg, ctx->al[fam], ctx->al_seg[fam],
        ctx->al_row[fam]);
    count_launch(ctx);
  }
}

// The family over `rows` rows of length L of a prefix table.
mad_status build_family(mad_ctx* ctx, int fam, const void* prefix, int prefix64, int64_t rows,
                        int64_t L, cudaStream_t st) {
  const int64_t nseg = (L + kAliasSeg - 1) / kAliasSeg;
  if (nseg > kAliasSeg) return MAD_ERR_UNSUPPORTED;   // two levels reach 2^20 entries
  mad_status rs;
  if ((rs = pool_malloc(ctx, (void**)&ctx->al[fam], (size_t)(rows * (L + nseg)) * sizeof(AliasEnt),
                        st)) != MAD_OK)
    return rs;
  if ((rs = pool_malloc(ctx, (void**)&ctx->al_seg[fam],
                        (size_t)(rows * nseg) * sizeof(unsigned long long), st)) != MAD_OK)
    return rs;
  if ((rs = pool_malloc(ctx, (void**)&ctx->al_row[fam], (size_t)rows * sizeof(unsigned long long),
                        st)) != MAD_OK)
    return rs;
  ctx->al_nseg[fam] = (int)nseg;
  if (!prefix64 && L <= kSmallAlias) {
    const size_t smem = (size_t)kSmallThreads * small_alias_stride((int)L);
    static size_t small_attr = 0;
    if (small_attr < smem) {
      cudaFuncSetAttribute(k_alias_build_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
      small_attr = smem;
    }
    k_alias_build_small<<<(unsigned)((rows + kSmallThreads - 1) / kSmallThreads), kSmallThreads,
                          smem, st>>>((const uint32_t*)prefix, rows, (int)L, ctx->al[fam],
                                      ctx->al_seg[fam], ctx->al_row[fam]);
    count_launch(ctx);
    return cuda_status(cudaGetLastError());
  }
  if (prefix64)
    launch_warp_family<unsigned __int128>(ctx, fam, prefix, prefix64, rows, L, nseg, st);
  else
    launch_warp_family<unsigned long long>(ctx, fam, prefix, prefix64, rows, L, nseg, st);
  return cuda_status(cudaGetLastError());
}

}  // namespace

mad_status build_alias_tables(mad_ctx* ctx, cudaStream_t st) {
  if (!ctx->dense || ctx->integer) return MAD_ERR_UNSUPPORTED;
  mad_status rs;
  if ((rs = build_family(ctx, kAlT1, ctx->T1, 1, 1, ctx->m, st)) != MAD_OK) return rs;
  if ((rs = build_family(ctx, kAlT2, ctx->T2, 0, ctx->m, ctx->d, st)) != MAD_OK) return rs;
  if ((rs = build_family(ctx, kAlTA, ctx->TA, 0, ctx->m, ctx->d, st)) != MAD_OK) return rs;
  return build_family(ctx, kAlTB, ctx->TB, 0, ctx->d, ctx->n, st);
}

}  // namespace mad
