// One pass of the loop body of Alg. 2 for a single diamond, shared by the
// sampling kernels (single instance and batched queries).
#ifndef MAD_DRAW_CUH_
#define MAD_DRAW_CUH_

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {

struct Draw {
  uint32_t i, k, j, kp;
  long long v;
};

// Center edge, stage 1: row i of A from T1 (through its guide when built).
__device__ __forceinline__ int64_t draw_row_i(const SampleParams& p, unsigned long long u0,
                                              bool* bad) {
  const unsigned long long target = draw_target(u0, p.t1_total);
  if (p.T1g) {
    const int64_t i = ub_guided_u64(p.T1, p.m, p.T1g, p.t1g_sh, target);
    if (i >= p.m) {
      *bad = true;
      return p.m - 1;
    }
    return i;
  }
  return search_u64(p.T1, p.m, target, bad);
}

// The rest of the loop body for a diamond whose row i is known.
__device__ __forceinline__ Draw draw_given_row(const SampleParams& p, const Uniforms& u,
                                               int64_t i, bool* bad) {
  const uint32_t mask = p.integer ? 0xFFFFFFFFu : PREFIX_MASK;
  int64_t a0, alen;
  if (p.dense) {
    a0 = i * p.d;
    alen = p.d;
  } else {
    a0 = __ldg(p.a_ptr + i);
    alen = __ldg(p.a_ptr + i + 1) - a0;
  }
  // Center edge, stage 2 (k within row i) and k' within row i: the two
  // searches run over rows of the same length, side by side.
  int64_t pk, pkp;
  uint32_t e_k, e_kp = 0;
  if (p.integer) {
    const uint32_t t2tot = __ldg(p.T2 + a0 + alen - 1);
    const uint32_t target = (uint32_t)draw_target(u.u1, t2tot);
    if (p.T2g && alen >= kGuideMin) {
      pk = ub_guided_u32(p.T2 + a0, p.T2g + __ldg(p.T2g_ptr + i), (int)__ldg(p.T2g_sh + i), target);
    } else {
      pk = ub_u32(p.T2 + a0, (int)alen, target, mask);
    }
    pkp = (int64_t)draw_target(u.u3, (unsigned long long)alen);
  } else {
    const uint32_t t2tot = __ldg(p.T2 + a0 + alen - 1) & mask;
    const uint32_t tatot = __ldg(p.TA + a0 + alen - 1) & mask;
    int a, b;
    ub2_u32(p.T2 + a0, p.TA + a0, (int)alen, (uint32_t)draw_target(u.u1, t2tot),
            (uint32_t)draw_target(u.u3, tatot), mask, &a, &b);
    pk = a;
    pkp = b;
  }
  if (pk >= alen) { *bad = true; pk = alen - 1; }
  if (pkp >= alen) { *bad = true; pkp = alen - 1; }
  e_k = __ldg(p.T2 + a0 + pk);
  if (!p.integer) e_kp = __ldg(p.TA + a0 + pkp);
  const int64_t k = p.dense ? pk : (int64_t)__ldg(p.a_col + a0 + pk);
  // j from row k of B.
  int64_t b0, blen;
  if (p.dense) {
    b0 = k * p.n;
    blen = p.n;
  } else {
    b0 = __ldg(p.b_ptr + k);
    blen = __ldg(p.b_ptr + k + 1) - b0;
  }
  int64_t pj;
  uint32_t e_j = 0;
  if (p.integer) {
    pj = (int64_t)draw_target(u.u2, (unsigned long long)blen);
  } else {
    const uint32_t tbtot = __ldg(p.TB + b0 + blen - 1) & mask;
    const uint32_t target = (uint32_t)draw_target(u.u2, tbtot);
    if (p.TBg) {
      pj = ub_guided_u32(p.TB + b0, p.TBg + k * p.tbg_stride, (int)__ldg(p.TBg_sh + k), target,
                         mask);
      if (pj >= blen) { *bad = true; pj = blen - 1; }
    } else {
      pj = ub_u32(p.TB + b0, (int)blen, target, mask);
      if (pj >= blen) { *bad = true; pj = blen - 1; }
    }
    e_j = __ldg(p.TB + b0 + pj);
  }
  const int64_t j = p.dense ? pj : (int64_t)__ldg(p.b_col + b0 + pj);
  const int64_t kp = p.dense ? pkp : (int64_t)__ldg(p.a_col + a0 + pkp);
  // Increment.
  long long v;
  if (p.integer) {
    // b_k'j != 0: the entry (j, k') of A under MAD_GRAM, else (k', j) of B.
    // The filter settles most tests with one load; the rest search rows.
    const unsigned long long ekey = (p.flags & MAD_GRAM)
                                        ? (((unsigned long long)j << 32) | (unsigned long long)kp)
                                        : (((unsigned long long)kp << 32) | (unsigned long long)j);
    bool hit = false;
    if (p.bloom && !bloom_may_contain(p.bloom, p.bloom_shift, ekey)) {
      hit = false;
    } else if (p.flags & MAD_GRAM) {
      const int64_t c0 = __ldg(p.b_ptr + kp), clen = __ldg(p.b_ptr + kp + 1) - c0;
      // B = A^T: b_k'j = a_jk'; search the shorter of the two sorted rows.
      const int64_t r0 = __ldg(p.a_ptr + j), rlen = __ldg(p.a_ptr + j + 1) - r0;
      hit = (rlen < clen) ? contains_sorted(p.a_col + r0, rlen, (int32_t)kp)
                          : contains_sorted(p.b_col + c0, clen, (int32_t)j);
    } else {
      const int64_t c0 = __ldg(p.b_ptr + kp), clen = __ldg(p.b_ptr + kp + 1) - c0;
      hit = contains_sorted(p.b_col + c0, clen, (int32_t)j);
    }
    v = hit ? 1 : 0;
  } else {
    const int64_t off = kp * p.ldb + j;
    const float b = p.b_f64 ? __double2float_rn(__ldg((const double*)p.b_val + off))
                            : __ldg((const float*)p.b_val + off);
    v = fixed_point(b, p.f_exp);
    if (!(p.flags & MAD_NONNEG) && ((e_k ^ e_j ^ e_kp) & SIGN_BIT)) v = -v;
  }
  Draw dr;
  dr.i = (uint32_t)i;
  dr.k = (uint32_t)k;
  dr.j = (uint32_t)j;
  dr.kp = (uint32_t)kp;
  dr.v = v;
  return dr;
}

// One alias draw over entries e[0..n) of total X with the uniform u: column
// floor(u n / 2^64); the low 64 bits f of u n keep the column when
// floor(f X / 2^64) < t, else its alias is returned.
__device__ __forceinline__ int64_t alias_pick(const AliasEnt* e, unsigned long long n,
                                              unsigned long long X, unsigned long long u) {
  const unsigned long long col = __umul64hi(u, n);
  const unsigned long long f = u * n;
  const unsigned long long hi = __umul64hi(f, X);
  const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(e + col));
  return hi < v.x ? (int64_t)col : (int64_t)(uint32_t)v.y;
}

// Position in row r of alias family fam (rows of length L): the segment from
// u_top (two levels only), then the column inside it from u_in (u_top when
// the row has one segment).
__device__ __forceinline__ int64_t alias_draw(const SampleParams& p, int fam, int64_t L, int64_t r,
                                              unsigned long long u_top, unsigned long long u_in) {
  const int nseg = p.al_nseg[fam];
  const AliasEnt* row = p.al[fam] + r * (L + nseg);
  if (nseg == 1) return alias_pick(row, (unsigned long long)L, __ldg(p.al_seg[fam] + r), u_top);
  const int64_t sg = alias_pick(row + L, (unsigned long long)nseg, __ldg(p.al_row[fam] + r), u_top);
  const int64_t c0 = sg * kAliasSeg;
  const int64_t len = L - c0 < kAliasSeg ? L - c0 : kAliasSeg;
  return c0 + alias_pick(row + c0, (unsigned long long)len,
                         __ldg(p.al_seg[fam] + r * nseg + sg), u_in);
}

// The loop body with the four draws from alias tables (dense float inputs):
// the same laws as the prefix-table draws, another map from the uniforms.
__device__ __forceinline__ Draw draw_alias(const SampleParams& p, unsigned long long seed,
                                           unsigned long long ell) {
  const Uniforms u = diamond_uniforms(seed, ell);
  const Uniforms v = alias_uniforms(seed, ell);
  const int64_t i = alias_draw(p, kAlT1, p.m, 0, u.u0, v.u0);
  const int64_t k = alias_draw(p, kAlT2, p.d, i, u.u1, v.u1);
  const int64_t j = alias_draw(p, kAlTB, p.n, k, u.u2, v.u2);
  const int64_t kp = alias_draw(p, kAlTA, p.d, i, u.u3, v.u3);
  const uint32_t e_k = __ldg(p.T2 + i * p.d + k);
  const uint32_t e_kp = __ldg(p.TA + i * p.d + kp);
  const uint32_t e_j = __ldg(p.TB + k * p.n + j);
  const int64_t off = kp * p.ldb + j;
  const float b = p.b_f64 ? __double2float_rn(__ldg((const double*)p.b_val + off))
                          : __ldg((const float*)p.b_val + off);
  long long val = fixed_point(b, p.f_exp);
  if (!(p.flags & MAD_NONNEG) && ((e_k ^ e_j ^ e_kp) & SIGN_BIT)) val = -val;
  Draw dr;
  dr.i = (uint32_t)i;
  dr.k = (uint32_t)k;
  dr.j = (uint32_t)j;
  dr.kp = (uint32_t)kp;
  dr.v = val;
  return dr;
}

// kAlias selects the alias-table draws at compile time, so that the
// prefix-table kernels carry none of their code; draw_one picks at run time
// (diagnostic kernels only).
template <bool kAlias>
__device__ __forceinline__ Draw draw_one_as(const SampleParams& p, unsigned long long seed,
                                            unsigned long long ell, bool* bad) {
  if (kAlias) return draw_alias(p, seed, ell);
  const Uniforms u = diamond_uniforms(seed, ell);
  return draw_given_row(p, u, draw_row_i(p, u.u0, bad), bad);
}

__device__ __forceinline__ Draw draw_one(const SampleParams& p, unsigned long long seed,
                                         unsigned long long ell, bool* bad) {
  return p.alias ? draw_one_as<true>(p, seed, ell, bad) : draw_one_as<false>(p, seed, ell, bad);
}

}  // namespace mad

#endif  // MAD_DRAW_CUH_
