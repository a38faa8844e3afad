// Diamond-sampling oracle: a plain, slow, single-threaded CPU statement of
// what the GPU library computes.  TEST INFRASTRUCTURE ONLY: the tests, the
// smoke check and the CPU-baseline leg of the benchmark load it; the product
// path never does.  It shares no source with the CUDA library.
//
// Paper: Ballard, Kolda, Pinar, Seshadhri, "Diamond Sampling for Approximate
// Maximum All-pairs Dot-product (MAD) Search", arXiv:1506.03872.
//
// Orientation.  A is m x d with rows a_i, B is d x n with rows b_k* and
// columns b_j, C = AB, c_ij = sum_k a_ik b_kj.  The paper writes A^T B with
// vectors as columns (Sec. 2); its a_ki is our a_ik.
//
// Every step below follows Alg. 2 (general diamond sampling) and Alg. 3
// (postprocessing), with the numeric readings that the paper leaves open
// written out where they are used:
//   * weights are FP32, row sums use one fixed summation order
//     (canonical_sum_f32), products are rounded to FP32 before summing;
//   * the sampling distributions are held as integer prefix tables whose
//     entries are the FP32 weights scaled by a power of two and rounded to
//     nearest-even (a nonzero weight that rounds to 0 becomes 1);
//   * the center edge (i,k) ~ w_ik/||W||_1 is drawn in two stages: row i with
//     probability r_i/sum r, r_i = ||a_i*||_1 * sum_k |a_ik| ||b_k*||_1, then
//     k within row i proportional to |a_ik| ||b_k*||_1 (same joint law);
//   * a draw maps a 64-bit uniform u to target = floor(u*T/2^64) and returns
//     the first position whose inclusive prefix exceeds target;
//   * uniforms come from Philox4x32-10 with key = seed, counter =
//     (l_lo, l_hi, instance, block) for diamond index l;
//   * the increment sgn(a_ik b_kj a_ik') b_k'j is accumulated in int64 fixed
//     point: b_k'j (as FP32) times 2^F rounded to nearest-even;
//   * 0/1 CSR inputs run in exact integer mode (no scaling at all);
//   * with FL_ALIAS (dense float inputs) the four draws take the same laws
//     from alias tables over the same integer weights (Vose's method in
//     exact integers, two levels above 1024 entries, the second level's
//     uniforms from Philox blocks 2 and 3).
//
// Parity is pinned by the tests: Philox known-answer vectors, Lemma 1 and
// Lemma 2 closed forms, the binary diamond count c_ij^2, brute-force top-t
// and long-double dot products.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace {

enum { FMT_DENSE = 0, FMT_CSR = 1 };
enum { DT_F32 = 0, DT_F64 = 1, DT_BINARY = 2 };
enum { FL_NONNEG = 1u, FL_GRAM = 2u, FL_EXCLUDE_DIAG = 4u, FL_SQSYM = 8u, FL_WEDGE = 16u,
       FL_ALIAS = 32u };
enum {
  ST_OK = 0, ST_ARG = 1, ST_OVERFLOW = 4, ST_EMPTY = 5, ST_UNSUPPORTED = 8
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
// easy as 1, 2, 3", SC'11).  Ten rounds; each round multiplies words 0 and 2
// by the two round multipliers, swaps in the high halves XORed with the other
// words and the round key; the key is bumped by the two Weyl constants
// between rounds.
// ---------------------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    const uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t y0 = hi1 ^ x1 ^ k0;
    const uint32_t y1 = lo1;
    const uint32_t y2 = hi0 ^ x3 ^ k1;
    const uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

// The four 64-bit uniforms of diamond l: u[0] picks i, u[1] picks k,
// u[2] picks j, u[3] picks k'.
void diamond_uniforms(uint64_t seed, uint64_t ell, uint32_t instance, uint64_t u[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t block = 0; block < 2; ++block) {
    const uint32_t ctr[4] = {(uint32_t)ell, (uint32_t)(ell >> 32), instance, block};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    u[2 * block + 0] = ((uint64_t)w[1] << 32) | w[0];
    u[2 * block + 1] = ((uint64_t)w[3] << 32) | w[2];
  }
}

// floor(u * total / 2^64): the draw target in [0, total).
uint64_t draw_target(uint64_t u, uint64_t total) {
  return (uint64_t)(((unsigned __int128)u * (unsigned __int128)total) >> 64);
}

// Inverse-CDF search (Sec. 4.1): first position whose inclusive prefix
// exceeds target.  std::upper_bound is the library search primitive.
template <typename T>
int64_t inverse_cdf(const T* prefix, int64_t len, uint64_t target) {
  const T* p = std::upper_bound(prefix, prefix + len, (T)target,
                                [](T t, T v) { return (uint64_t)t < (uint64_t)v; });
  return (int64_t)(p - prefix);
}

// Fixed FP32 summation order used for every L1 norm and row sum: 256
// partial sums, partial q taking the elements whose index is q mod 256 in
// ascending order, then folded in halves (q += q+128, then q += q+64, ...,
// q += q+1).  FP32 round-to-nearest-even, no fused operations.
float canonical_sum_f32(const std::vector<float>& w) {
  float part[256];
  for (int q = 0; q < 256; ++q) part[q] = 0.0f;
  for (size_t idx = 0; idx < w.size(); ++idx) {
    part[idx % 256] = part[idx % 256] + w[idx];
  }
  for (int h = 128; h >= 1; h /= 2)
    for (int q = 0; q < h; ++q) {
      part[q] = part[q] + part[q + h];
    }
  return part[0];
}

// ceil(log2(x)) for x >= 1.
int ceil_log2(uint64_t x) {
  int e = 0;
  while (e < 64 && ((uint64_t)1 << e) < x) ++e;
  return e;
}

// Row table exponent: the largest power of two keeping the scaled row sum
// below 2^30, so the row's prefix stays below 2^31 (bit 31 stays free).
int row_exponent(float rowsum) { return 29 - std::ilogb(rowsum); }

uint32_t quantize_row(float w, int e) {
  const double q = std::rint(std::ldexp((double)w, e));
  uint32_t v = (uint32_t)q;
  if (w > 0.0f && v == 0) v = 1;  // keep the support of the paper's distribution
  return v;
}

struct Mat {
  int64_t rows = 0, cols = 0;
  std::vector<int64_t> ptr;    // rows+1
  std::vector<int32_t> col;    // stored entries, ascending within a row
  std::vector<double> val;     // values as given (1.0 for binary)
  std::vector<float> valf;     // values rounded to FP32
  bool dense = false, binary = false;
};

bool load_matrix(int fmt, int dt, int64_t rows, int64_t cols, int64_t ld, const void* values,
                 const int64_t* rowptr, const int32_t* colidx, Mat& M) {
  M.rows = rows;
  M.cols = cols;
  M.ptr.assign(rows + 1, 0);
  M.dense = (fmt == FMT_DENSE);
  M.binary = (dt == DT_BINARY);
  if (fmt == FMT_DENSE) {
    if (dt == DT_BINARY || ld < cols) return false;
    for (int64_t r = 0; r < rows; ++r) {
      M.ptr[r + 1] = M.ptr[r] + cols;
      for (int64_t c = 0; c < cols; ++c) {
        const double v = (dt == DT_F64) ? ((const double*)values)[r * ld + c]
                                        : (double)((const float*)values)[r * ld + c];
        M.col.push_back((int32_t)c);
        M.val.push_back(v);
        M.valf.push_back((float)v);
      }
    }
    return true;
  }
  if (fmt != FMT_CSR || dt != DT_BINARY || rowptr[0] != 0) return false;
  for (int64_t r = 0; r < rows; ++r) {
    M.ptr[r + 1] = rowptr[r + 1];
    for (int64_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
      M.col.push_back(colidx[e]);
      M.val.push_back(1.0);
      M.valf.push_back(1.0f);
    }
  }
  return true;
}

// Alias tables (Sec. 4.1 names the alias method for constant-time draws
// from a discrete distribution).  A table over weights x_0..x_{n-1} with
// total X holds, per column c, a threshold t_c in [0, X] and an alias a_c:
// a draw takes column c uniformly and keeps c with probability t_c / X,
// else returns a_c.  Built by Vose's method in exact integers, so that
// P(c) = x_c / X holds exactly.  Tables longer than kAliasSeg entries have
// two levels: segments of kAliasSeg entries, each with its own table, and
// one table over the segment totals.
constexpr int64_t kAliasSeg = 1024;

struct AliasEnt {
  uint64_t t;
  uint32_t a;
  uint32_t pad;
};

// A family of alias tables of the same length L, one per row.  Row r holds
// its segments' entries (L of them) followed by the table over its segments
// (nseg entries); segX and rowX hold the segment and row totals.
struct AliasFam {
  int64_t rows = 0, L = 0, nseg = 0;
  std::vector<AliasEnt> ent;
  std::vector<uint64_t> segX, rowX;
};

struct Oracle {
  uint32_t flags = 0;
  bool integer = false;
  uint64_t s_max = 0;
  Mat A, B;
  int64_t m = 0, d = 0, n = 0;
  // Float-mode norms and row weights.
  std::vector<float> na, nb, srow, r;
  // Tables: T1 over rows of A; T2, TA aligned with A's entries; TB with B's.
  std::vector<uint64_t> T1;
  std::vector<uint32_t> T2, TA, TB;
  int E1 = 0, F = 0;
  uint64_t bumps = 0;
  // Wedge sampling (FL_WEDGE): the columns of A (entry q of column k is
  // row Acol_row[q], FP32 value Acol_val[q], rows ascending), their
  // cumulative tables TAc, the column norms, and the center table TK over k
  // with its scale exponent EK.
  bool wedge = false;
  std::vector<int64_t> Acol_ptr;
  std::vector<int32_t> Acol_row;
  std::vector<float> Acol_val;
  std::vector<uint32_t> TAc;
  std::vector<float> nac, wk;
  std::vector<uint64_t> TK;
  int EK = 0;
  // Alias draws (FL_ALIAS): tables over the weights of T1, of every row of
  // T2 and TA, and of every row of TB.
  bool alias = false;
  AliasFam T1al, T2al, TAal, TBal;
  // Sampling state.
  std::unordered_map<uint64_t, int64_t> X;
  uint64_t sampled = 0, inserted = 0, diag_skipped = 0;
};

int build_tables(Oracle& o) {
  const Mat& A = o.A;
  const Mat& B = o.B;
  o.m = A.rows;
  o.d = A.cols;
  o.n = B.cols;
  if (B.rows != o.d || o.m <= 0 || o.d <= 0 || o.n <= 0) return ST_ARG;
  if (o.m > 0xFFFFFFFFll || o.n > 0xFFFFFFFFll) return ST_ARG;
  o.T1.assign(o.m, 0);
  o.T2.assign(A.col.size(), 0);
  o.TA.assign(A.col.size(), 0);
  o.TB.assign(B.col.size(), 0);

  if (o.integer) {
    // Exact integer mode for 0/1 inputs (Alg. 1): w_ik = deg_i^A deg_k^B.
    // T2 holds deg_k^B along row i, TA and TB hold 1 per neighbour.
    unsigned __int128 total = 0;
    for (int64_t k = 0; k < o.d; ++k) {
      uint32_t p = 0;
      for (int64_t e = B.ptr[k]; e < B.ptr[k + 1]; ++e) o.TB[e] = ++p;
    }
    for (int64_t i = 0; i < o.m; ++i) {
      uint64_t p2 = 0;
      uint32_t pa = 0;
      for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
        const int32_t k = A.col[e];
        p2 += (uint64_t)(B.ptr[k + 1] - B.ptr[k]);
        if (p2 > 0xFFFFFFFFull) return ST_OVERFLOW;
        o.T2[e] = (uint32_t)p2;
        o.TA[e] = ++pa;
      }
      const uint64_t ri = (uint64_t)(A.ptr[i + 1] - A.ptr[i]) * p2;
      total += ri;
      if (total >= ((unsigned __int128)1 << 63)) return ST_OVERFLOW;
      o.T1[i] = (uint64_t)total;
    }
    if (total == 0) return ST_EMPTY;
    o.E1 = 0;
    o.F = 0;
    return ST_OK;
  }

  // Float mode.  L1 norms (Alg. 2 weight line): ||b_k*||_1 and ||a_i*||_1.
  o.nb.assign(o.d, 0.0f);
  float maxb = 0.0f;
  for (int64_t k = 0; k < o.d; ++k) {
    std::vector<float> w;
    for (int64_t e = B.ptr[k]; e < B.ptr[k + 1]; ++e) {
      w.push_back(std::fabs(B.valf[e]));
      maxb = std::max(maxb, std::fabs(B.valf[e]));
    }
    o.nb[k] = canonical_sum_f32(w);
    if (o.nb[k] > 0.0f) {
      const int e = row_exponent(o.nb[k]);
      uint32_t p = 0;
      for (size_t q = 0; q < w.size(); ++q) {
        const uint32_t v = quantize_row(w[q], e);
        if (w[q] > 0.0f && std::rint(std::ldexp((double)w[q], e)) == 0.0) ++o.bumps;
        p += v;
        o.TB[B.ptr[k] + q] = p;
      }
    }
  }
  o.na.assign(o.m, 0.0f);
  o.srow.assign(o.m, 0.0f);
  o.r.assign(o.m, 0.0f);
  float maxr = 0.0f;
  for (int64_t i = 0; i < o.m; ++i) {
    std::vector<float> wa, w2;
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const float a = std::fabs(A.valf[e]);
      const float prod = a * o.nb[A.col[e]];
      wa.push_back(a);
      w2.push_back(prod);
    }
    o.na[i] = canonical_sum_f32(wa);
    o.srow[i] = canonical_sum_f32(w2);
    o.r[i] = o.na[i] * o.srow[i];
    maxr = std::max(maxr, o.r[i]);
    if (o.srow[i] > 0.0f) {
      const int e2 = row_exponent(o.srow[i]);
      const int ea = row_exponent(o.na[i]);
      uint32_t p2 = 0, pa = 0;
      for (size_t q = 0; q < w2.size(); ++q) {
        if (w2[q] > 0.0f && std::rint(std::ldexp((double)w2[q], e2)) == 0.0) ++o.bumps;
        if (wa[q] > 0.0f && std::rint(std::ldexp((double)wa[q], ea)) == 0.0) ++o.bumps;
        p2 += quantize_row(w2[q], e2);
        pa += quantize_row(wa[q], ea);
        o.T2[A.ptr[i] + q] = p2;
        o.TA[A.ptr[i] + q] = pa;
      }
    }
  }
  if (maxr == 0.0f || maxb == 0.0f) return ST_EMPTY;
  // T1: r_i scaled so that every entry is below 2^(62 - ceil(log2 m)); the
  // whole prefix then stays below 2^62.
  o.E1 = 62 - ceil_log2((uint64_t)o.m) - (std::ilogb(maxr) + 1);
  uint64_t p1 = 0;
  for (int64_t i = 0; i < o.m; ++i) {
    const double q = std::rint(std::ldexp((double)o.r[i], o.E1));
    uint64_t v = (uint64_t)q;
    if (o.r[i] > 0.0f && v == 0) {
      v = 1;
      ++o.bumps;
    }
    p1 += v;
    o.T1[i] = p1;
  }
  // Increment scale: |b| 2^F < 2^(62 - ceil(log2 s_max)), so s_max
  // increments cannot overflow int64.
  o.F = 62 - ceil_log2(std::max<uint64_t>(o.s_max, 1)) - (std::ilogb(maxb) + 1);
  return ST_OK;
}

// Tables of wedge sampling (the appendix's Alg. "MAD wedge sampling"): with
// A m x d (rows a_i) and B d x n, the center k is drawn with probability
// w_k / ||w||_1, w_k = ||a_*k||_1 ||b_k*||_1, then i within column k of A
// with probability |a_ik| / ||a_*k||_1 and j within row k of B with
// probability |b_kj| / ||b_k*||_1 (the TB table of Alg. 2 above).  Float
// mode quantises as the diamond tables do: column tables like row tables
// (scaled so the column's prefix stays below 2^31), TK like T1 with d in
// place of m.  0/1 inputs: w_k = (entries of column k of A) x (entries of
// row k of B), exact.
int build_wedge_tables(Oracle& o) {
  const Mat& A = o.A;
  const Mat& B = o.B;
  // Columns of A, rows ascending.
  o.Acol_ptr.assign(o.d + 1, 0);
  for (size_t e = 0; e < A.col.size(); ++e) ++o.Acol_ptr[A.col[e] + 1];
  for (int64_t k = 0; k < o.d; ++k) o.Acol_ptr[k + 1] += o.Acol_ptr[k];
  o.Acol_row.assign(A.col.size(), 0);
  o.Acol_val.assign(A.col.size(), 0.0f);
  std::vector<int64_t> fill(o.Acol_ptr.begin(), o.Acol_ptr.end() - 1);
  for (int64_t i = 0; i < o.m; ++i)
    for (int64_t e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int64_t q = fill[A.col[e]]++;
      o.Acol_row[q] = (int32_t)i;
      o.Acol_val[q] = A.valf[e];
    }
  o.TAc.assign(A.col.size(), 0);
  o.TK.assign(o.d, 0);
  if (o.integer) {
    uint64_t total = 0;
    for (int64_t k = 0; k < o.d; ++k) {
      uint32_t p = 0;
      for (int64_t q = o.Acol_ptr[k]; q < o.Acol_ptr[k + 1]; ++q) o.TAc[q] = ++p;
      const uint64_t w = (uint64_t)(o.Acol_ptr[k + 1] - o.Acol_ptr[k]) *
                         (uint64_t)(B.ptr[k + 1] - B.ptr[k]);
      if (total + w < total || total + w >= (1ull << 63)) return ST_OVERFLOW;
      total += w;
      o.TK[k] = total;
    }
    o.EK = 0;
    return total == 0 ? ST_EMPTY : ST_OK;
  }
  o.nac.assign(o.d, 0.0f);
  o.wk.assign(o.d, 0.0f);
  float maxw = 0.0f;
  for (int64_t k = 0; k < o.d; ++k) {
    std::vector<float> w;
    for (int64_t q = o.Acol_ptr[k]; q < o.Acol_ptr[k + 1]; ++q) w.push_back(std::fabs(o.Acol_val[q]));
    o.nac[k] = canonical_sum_f32(w);
    if (o.nac[k] > 0.0f) {
      const int e = row_exponent(o.nac[k]);
      uint32_t p = 0;
      for (size_t q = 0; q < w.size(); ++q) {
        p += quantize_row(w[q], e);
        o.TAc[o.Acol_ptr[k] + q] = p;
      }
    }
    o.wk[k] = o.nac[k] * o.nb[k];
    maxw = std::max(maxw, o.wk[k]);
  }
  if (maxw == 0.0f) return ST_EMPTY;
  o.EK = 62 - ceil_log2((uint64_t)o.d) - (std::ilogb(maxw) + 1);
  uint64_t p = 0;
  for (int64_t k = 0; k < o.d; ++k) {
    uint64_t v = (uint64_t)std::rint(std::ldexp((double)o.wk[k], o.EK));
    if (o.wk[k] > 0.0f && v == 0) v = 1;
    p += v;
    o.TK[k] = p;
  }
  return ST_OK;
}

// Vose's construction over x[0..n), total X: small and large columns
// (n x_c below X, or not) are stacks filled in column order; the top small
// column s takes its own share n x_s and the top large column l the rest,
// after which l's remaining weight n x_l - (X - n x_s) classifies it again.
// Columns left at the end keep themselves.
void vose(const uint64_t* x, int64_t n, uint64_t X, AliasEnt* out) {
  std::vector<unsigned __int128> p((size_t)n);
  std::vector<int64_t> small, large;
  for (int64_t c = 0; c < n; ++c) {
    p[c] = (unsigned __int128)x[c] * (uint64_t)n;
    if (p[c] < X) small.push_back(c);
    else large.push_back(c);
  }
  while (!small.empty() && !large.empty()) {
    const int64_t sc = small.back();
    small.pop_back();
    const int64_t lc = large.back();
    large.pop_back();
    out[sc].t = (uint64_t)p[sc];
    out[sc].a = (uint32_t)lc;
    out[sc].pad = 0;
    p[lc] -= (unsigned __int128)(X - (uint64_t)p[sc]);
    if (p[lc] < X) small.push_back(lc);
    else large.push_back(lc);
  }
  for (int64_t c : large) out[c] = AliasEnt{X, (uint32_t)c, 0};
  for (int64_t c : small) out[c] = AliasEnt{X, (uint32_t)c, 0};
}

// The family over `rows` rows of length L whose weight c of row r is
// weight(r, c).
template <typename Weight>
void build_alias_family(AliasFam& f, int64_t rows, int64_t L, Weight weight) {
  f.rows = rows;
  f.L = L;
  f.nseg = (L + kAliasSeg - 1) / kAliasSeg;
  f.ent.assign((size_t)(rows * (L + f.nseg)), AliasEnt{0, 0, 0});
  f.segX.assign((size_t)(rows * f.nseg), 0);
  f.rowX.assign((size_t)rows, 0);
  std::vector<uint64_t> w;
  for (int64_t r = 0; r < rows; ++r) {
    AliasEnt* row = f.ent.data() + r * (L + f.nseg);
    uint64_t total = 0;
    for (int64_t sg = 0; sg < f.nseg; ++sg) {
      const int64_t c0 = sg * kAliasSeg, len = std::min(kAliasSeg, L - c0);
      w.assign((size_t)len, 0);
      uint64_t X = 0;
      for (int64_t c = 0; c < len; ++c) {
        w[c] = weight(r, c0 + c);
        X += w[c];
      }
      vose(w.data(), len, X, row + c0);
      f.segX[r * f.nseg + sg] = X;
      total += X;
    }
    f.rowX[r] = total;
    if (f.nseg > 1) vose(f.segX.data() + r * f.nseg, f.nseg, total, row + L);
    else row[L] = AliasEnt{total, 0, 0};
  }
}

// One alias draw over entries e[0..n) of total X with the 64-bit uniform u:
// column floor(u n / 2^64); the low 64 bits f of u n decide between the
// column and its alias, keeping the column when floor(f X / 2^64) < t.
int64_t alias_pick(const AliasEnt* e, int64_t n, uint64_t X, uint64_t u) {
  const unsigned __int128 pr = (unsigned __int128)u * (uint64_t)n;
  const int64_t col = (int64_t)(pr >> 64);
  const uint64_t f = (uint64_t)pr;
  const uint64_t hi = (uint64_t)(((unsigned __int128)f * X) >> 64);
  return hi < e[col].t ? col : (int64_t)e[col].a;
}

// Position in row r of family f: the segment from u_top (two levels only),
// then the column inside it from u_in (u_top when there is one segment).
int64_t alias_draw(const AliasFam& f, int64_t r, uint64_t u_top, uint64_t u_in) {
  const AliasEnt* row = f.ent.data() + r * (f.L + f.nseg);
  if (f.nseg == 1) return alias_pick(row, f.L, f.segX[r], u_top);
  const int64_t sg = alias_pick(row + f.L, f.nseg, f.rowX[r], u_top);
  const int64_t c0 = sg * kAliasSeg, len = std::min(kAliasSeg, f.L - c0);
  return c0 + alias_pick(row + c0, len, f.segX[r * f.nseg + sg], u_in);
}

// Alias tables of the dense float tables: the weights are the differences
// of consecutive prefix entries (T1 over rows, T2 and TA along each row of
// A, TB along each row of B).
int build_alias_tables(Oracle& o) {
  if (o.integer || !o.A.dense || !o.B.dense) return ST_UNSUPPORTED;
  build_alias_family(o.T1al, 1, o.m, [&](int64_t, int64_t c) {
    return o.T1[c] - (c ? o.T1[c - 1] : 0);
  });
  auto row_weight = [](const std::vector<uint32_t>& T, int64_t L) {
    return [&T, L](int64_t r, int64_t c) -> uint64_t {
      const int64_t e = r * L + c;
      return (uint64_t)T[e] - (c ? (uint64_t)T[e - 1] : 0);
    };
  };
  build_alias_family(o.T2al, o.m, o.d, row_weight(o.T2, o.d));
  build_alias_family(o.TAal, o.m, o.d, row_weight(o.TA, o.d));
  build_alias_family(o.TBal, o.d, o.n, row_weight(o.TB, o.n));
  return ST_OK;
}

// Uniforms of Philox blocks 2 and 3 of diamond ell: the segment-level
// uniforms of the two-level alias draws (index q of (i, k, j, k') uses u[q]
// of blocks 0-1 first and the q-th uniform here second).
void alias_uniforms(uint64_t seed, uint64_t ell, uint64_t u[4]) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t block = 2; block < 4; ++block) {
    const uint32_t ctr[4] = {(uint32_t)ell, (uint32_t)(ell >> 32), 0u, block};
    uint32_t w[4];
    philox4x32_10(ctr, key, w);
    u[2 * (block - 2) + 0] = ((uint64_t)w[1] << 32) | w[0];
    u[2 * (block - 2) + 1] = ((uint64_t)w[3] << 32) | w[2];
  }
}

// Value b_{k'j} of B (0 when absent).
double b_value(const Oracle& o, int64_t kp, int64_t j, float* valf) {
  const Mat& B = o.B;
  if (B.dense) {
    const int64_t e = B.ptr[kp] + j;
    *valf = B.valf[e];
    return B.val[e];
  }
  const int32_t* lo = B.col.data() + B.ptr[kp];
  const int32_t* hi = B.col.data() + B.ptr[kp + 1];
  const int32_t* p = std::lower_bound(lo, hi, (int32_t)j);
  if (p != hi && *p == (int32_t)j) {
    *valf = B.valf[p - B.col.data()];
    return B.val[p - B.col.data()];
  }
  *valf = 0.0f;
  return 0.0;
}

struct Draw {
  uint32_t i, k, j, kp;
  int64_t v;
};

// One iteration of the wedge sampling loop for wedge index ell: the first
// three uniforms of the index's Philox counter pick k, i and j; the
// increment is sgn(a_ik b_kj) (1 for 0/1 and nonnegative inputs).  The
// paper prints sgn(a_ki b_ki); its Lemma on E[x_ij] uses a_ki b_kj, which
// is what is added.  kp is 0.
Draw draw_wedge(const Oracle& o, uint64_t seed, uint64_t ell) {
  uint64_t u[4];
  diamond_uniforms(seed, ell, 0, u);
  const Mat& B = o.B;
  const int64_t k = inverse_cdf(o.TK.data(), o.d, draw_target(u[0], o.TK[o.d - 1]));
  const int64_t c0 = o.Acol_ptr[k], clen = o.Acol_ptr[k + 1] - c0;
  const int64_t pi = inverse_cdf(o.TAc.data() + c0, clen, draw_target(u[1], o.TAc[c0 + clen - 1]));
  const int64_t b0 = B.ptr[k], blen = B.ptr[k + 1] - b0;
  const int64_t pj = inverse_cdf(o.TB.data() + b0, blen, draw_target(u[2], o.TB[b0 + blen - 1]));
  Draw dr;
  dr.i = (uint32_t)o.Acol_row[c0 + pi];
  dr.k = (uint32_t)k;
  dr.j = (uint32_t)B.col[b0 + pj];
  dr.kp = 0;
  dr.v = 1;
  if (!o.integer && !(o.flags & FL_NONNEG)) {
    if (o.Acol_val[c0 + pi] < 0.0f) dr.v = -dr.v;
    if (B.valf[b0 + pj] < 0.0f) dr.v = -dr.v;
  }
  return dr;
}

// One iteration of the sampling loop of Alg. 2 for diamond index ell.
Draw draw_diamond(const Oracle& o, uint64_t seed, uint64_t ell) {
  uint64_t u[4];
  diamond_uniforms(seed, ell, 0, u);
  const Mat& A = o.A;
  const Mat& B = o.B;
  Draw dr;
  int64_t i, a0, alen, pk, k, b0, blen, pj, j, pkp, kp;
  if (o.alias) {
    // The same four laws, each drawn from its alias table.
    uint64_t v[4];
    alias_uniforms(seed, ell, v);
    i = alias_draw(o.T1al, 0, u[0], v[0]);
    a0 = A.ptr[i];
    alen = A.ptr[i + 1] - a0;
    pk = alias_draw(o.T2al, i, u[1], v[1]);
    k = A.col[a0 + pk];
    b0 = B.ptr[k];
    blen = B.ptr[k + 1] - b0;
    pj = alias_draw(o.TBal, k, u[2], v[2]);
    j = B.col[b0 + pj];
    pkp = alias_draw(o.TAal, i, u[3], v[3]);
    kp = A.col[a0 + pkp];
  } else {
    // Center edge (i,k) with probability w_ik / ||W||_1, in two stages.
    i = inverse_cdf(o.T1.data(), o.m, draw_target(u[0], o.T1[o.m - 1]));
    a0 = A.ptr[i];
    alen = A.ptr[i + 1] - A.ptr[i];
    pk = inverse_cdf(o.T2.data() + a0, alen, draw_target(u[1], o.T2[a0 + alen - 1]));
    k = A.col[a0 + pk];
    // j with probability |b_kj| / ||b_k*||_1.
    b0 = B.ptr[k];
    blen = B.ptr[k + 1] - B.ptr[k];
    pj = inverse_cdf(o.TB.data() + b0, blen, draw_target(u[2], o.TB[b0 + blen - 1]));
    j = B.col[b0 + pj];
    // k' with probability |a_ik'| / ||a_i*||_1.
    pkp = inverse_cdf(o.TA.data() + a0, alen, draw_target(u[3], o.TA[a0 + alen - 1]));
    kp = A.col[a0 + pkp];
  }
  // Increment sgn(a_ik b_kj a_ik') b_k'j.
  float bf = 0.0f;
  b_value(o, kp, j, &bf);
  int64_t v;
  if (o.integer) {
    v = (bf != 0.0f) ? 1 : 0;
  } else {
    v = (int64_t)std::llrint(std::ldexp((double)bf, o.F));
    if (!(o.flags & FL_NONNEG)) {
      int sgn = 1;
      if (A.valf[a0 + pk] < 0.0f) sgn = -sgn;
      if (B.valf[b0 + pj] < 0.0f) sgn = -sgn;
      if (A.valf[a0 + pkp] < 0.0f) sgn = -sgn;
      v *= sgn;
    }
  }
  dr.i = (uint32_t)i;
  dr.k = (uint32_t)k;
  dr.j = (uint32_t)j;
  dr.kp = (uint32_t)kp;
  dr.v = v;
  return dr;
}

uint64_t pair_key(const Oracle& o, uint64_t i, uint64_t j) {
  if ((o.flags & FL_GRAM) && j < i) std::swap(i, j);
  return (i << 32) | j;
}

// Dot product c_ij in FP64 with the fixed order shared by the library:
// 32 partial sums (partial L takes k = L mod 32, ascending, fused
// multiply-add), folded in halves (L += L+16, ..., L += L+1).
double dense_dot(const Oracle& o, uint32_t i, uint32_t j) {
  double part[32];
  for (int L = 0; L < 32; ++L) part[L] = 0.0;
  for (int64_t k = 0; k < o.d; ++k) {
    const double a = o.A.val[o.A.ptr[i] + k];
    const double b = o.B.val[o.B.ptr[k] + j];
    part[k % 32] = std::fma(a, b, part[k % 32]);
  }
  for (int h = 16; h >= 1; h /= 2)
    for (int L = 0; L < h; ++L) part[L] = part[L] + part[L + h];
  return part[0];
}

// 0/1 CSR: c_ij = |{k : a_ik = 1 and b_kj = 1}|, counted exactly.
double csr_dot(const Oracle& o, uint32_t i, uint32_t j) {
  int64_t count = 0;
  for (int64_t e = o.A.ptr[i]; e < o.A.ptr[i + 1]; ++e) {
    float bf;
    b_value(o, o.A.col[e], j, &bf);
    if (bf != 0.0f) ++count;
  }
  return (double)count;
}

struct Scored {
  uint64_t key;
  double c;
};

bool by_abs_c(const Scored& a, const Scored& b) {
  const double x = std::fabs(a.c), y = std::fabs(b.c);
  if (x != y) return x > y;
  return a.key < b.key;
}

}  // namespace

extern "C" {

void or_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  philox4x32_10(ctr, key, out);
}

void or_diamond_uniforms(uint64_t seed, uint64_t ell, uint32_t instance, uint64_t* u) {
  diamond_uniforms(seed, ell, instance, u);
}

void* or_create(int fmtA, int dtA, int64_t m, int64_t d, int64_t ldA, const void* valA,
                const int64_t* ptrA, const int32_t* colA, int fmtB, int dtB, int64_t dB,
                int64_t n, int64_t ldB, const void* valB, const int64_t* ptrB,
                const int32_t* colB, uint32_t flags, uint64_t s_max, int* status) {
  if ((flags & FL_SQSYM) && !(flags & FL_GRAM)) {  // Sec. 3.2.3 needs B = A^T = A
    *status = ST_UNSUPPORTED;
    return nullptr;
  }
  Oracle* o = new Oracle();
  o->flags = flags;
  o->s_max = s_max;
  if (!load_matrix(fmtA, dtA, m, d, ldA, valA, ptrA, colA, o->A) ||
      !load_matrix(fmtB, dtB, dB, n, ldB, valB, ptrB, colB, o->B) ||
      (dtA == DT_BINARY) != (dtB == DT_BINARY)) {
    *status = ST_UNSUPPORTED;
    delete o;
    return nullptr;
  }
  o->integer = (dtA == DT_BINARY);
  o->wedge = (flags & FL_WEDGE) != 0;
  if (o->wedge && (flags & FL_SQSYM)) {
    *status = ST_UNSUPPORTED;
    delete o;
    return nullptr;
  }
  o->alias = (flags & FL_ALIAS) != 0;
  if (o->alias && o->wedge) {
    *status = ST_UNSUPPORTED;
    delete o;
    return nullptr;
  }
  *status = build_tables(*o);
  if (*status == ST_OK && o->wedge) *status = build_wedge_tables(*o);
  if (*status == ST_OK && o->alias) *status = build_alias_tables(*o);
  if (*status != ST_OK) {
    delete o;
    return nullptr;
  }
  return o;
}

void or_destroy(void* h) { delete (Oracle*)h; }

// Table export.  which: 0 T1 (u64, m), 1 T2 (u32, nnz A), 2 TA (u32, nnz A),
// 3 TB (u32, nnz B), 4 na (f32, m), 5 nb (f32, d), 6 r (f32, m),
// 7 srow (f32, m).  Returns the element count.
int64_t or_table(void* h, int which, void* out) {
  Oracle* o = (Oracle*)h;
  switch (which) {
    case 0: if (out) std::memcpy(out, o->T1.data(), o->T1.size() * 8); return (int64_t)o->T1.size();
    case 1: if (out) std::memcpy(out, o->T2.data(), o->T2.size() * 4); return (int64_t)o->T2.size();
    case 2: if (out) std::memcpy(out, o->TA.data(), o->TA.size() * 4); return (int64_t)o->TA.size();
    case 3: if (out) std::memcpy(out, o->TB.data(), o->TB.size() * 4); return (int64_t)o->TB.size();
    case 4: if (out) std::memcpy(out, o->na.data(), o->na.size() * 4); return (int64_t)o->na.size();
    case 5: if (out) std::memcpy(out, o->nb.data(), o->nb.size() * 4); return (int64_t)o->nb.size();
    case 6: if (out) std::memcpy(out, o->r.data(), o->r.size() * 4); return (int64_t)o->r.size();
    case 7: if (out) std::memcpy(out, o->srow.data(), o->srow.size() * 4); return (int64_t)o->srow.size();
    case 8: if (out) std::memcpy(out, o->TK.data(), o->TK.size() * 8); return (int64_t)o->TK.size();
    case 9: if (out) std::memcpy(out, o->TAc.data(), o->TAc.size() * 4); return (int64_t)o->TAc.size();
    case 10: if (out) std::memcpy(out, o->nac.data(), o->nac.size() * 4); return (int64_t)o->nac.size();
  }
  return -1;
}

// Alias table export: family 0 T1, 1 T2, 2 TA, 3 TB; part 0 the entries
// (16 bytes each: u64 t, u32 a, u32 0; rows x (L + nseg)), 1 the segment
// totals (u64, rows x nseg), 2 the row totals (u64, rows).  Returns the
// element count, -1 without alias tables.
int64_t or_alias(void* h, int fam, int part, void* out) {
  Oracle* o = (Oracle*)h;
  if (!o->alias || fam < 0 || fam > 3) return -1;
  const AliasFam& f = fam == 0 ? o->T1al : fam == 1 ? o->T2al : fam == 2 ? o->TAal : o->TBal;
  switch (part) {
    case 0: if (out) std::memcpy(out, f.ent.data(), f.ent.size() * 16); return (int64_t)f.ent.size();
    case 1: if (out) std::memcpy(out, f.segX.data(), f.segX.size() * 8); return (int64_t)f.segX.size();
    case 2: if (out) std::memcpy(out, f.rowX.data(), f.rowX.size() * 8); return (int64_t)f.rowX.size();
  }
  return -1;
}

// Scalars: E1, F, bumps, T1 total, sampled, inserted, diag_skipped, |X|.
void or_scalars(void* h, int64_t* out) {
  Oracle* o = (Oracle*)h;
  out[0] = o->E1;
  out[1] = o->F;
  out[2] = (int64_t)o->bumps;
  out[3] = (int64_t)o->T1[o->m - 1];
  out[4] = (int64_t)o->sampled;
  out[5] = (int64_t)o->inserted;
  out[6] = (int64_t)o->diag_skipped;
  out[7] = (int64_t)o->X.size();
}

// Draws of diamonds first .. first+count-1 (no accumulation).
void or_draw(void* h, uint64_t seed, uint64_t first, uint64_t count, uint32_t* oi, uint32_t* ok,
             uint32_t* oj, uint32_t* okp, int64_t* ov) {
  Oracle* o = (Oracle*)h;
  for (uint64_t q = 0; q < count; ++q) {
    const Draw dr = o->wedge ? draw_wedge(*o, seed, first + q) : draw_diamond(*o, seed, first + q);
    oi[q] = dr.i;
    ok[q] = dr.k;
    oj[q] = dr.j;
    okp[q] = dr.kp;
    ov[q] = dr.v;
  }
}

// Draws of an arbitrary list of diamond indices (sampled parity checks).
void or_draw_list(void* h, uint64_t seed, uint64_t count, const uint64_t* ells, uint32_t* oi,
                  uint32_t* ok, uint32_t* oj, uint32_t* okp, int64_t* ov) {
  Oracle* o = (Oracle*)h;
  for (uint64_t q = 0; q < count; ++q) {
    const Draw dr = o->wedge ? draw_wedge(*o, seed, ells[q]) : draw_diamond(*o, seed, ells[q]);
    oi[q] = dr.i;
    ok[q] = dr.k;
    oj[q] = dr.j;
    okp[q] = dr.kp;
    ov[q] = dr.v;
  }
}

// The sampling loop of Alg. 2 for diamonds first .. first+s-1, accumulating
// into X.  Gram inputs (B = A^T, Sec. 3.2.2) accumulate into the unordered
// pair, which is twice the symmetrised X of Eq. (xsym) and orders the same;
// the diagonal is skipped when asked (Sec. 6.2, distinct pairs only).
//
// Squared symmetric inputs (FL_SQSYM with FL_GRAM, A = B = A^T, Sec. 3.2.3):
// the diamond (k', i, k, j) is also a diamond of the pair (k, k'), whose
// roles it swaps with (i, j), so its value is added to both pairs.  The
// paper adds half to each; adding the whole value to each scales every x by
// the same factor 2 and orders them the same.  Each of the two additions is
// skipped on the diagonal when asked (counted in diag_skipped).
int or_sample(void* h, uint64_t s, uint64_t seed, uint64_t first) {
  Oracle* o = (Oracle*)h;
  if (o->sampled + s > o->s_max) return ST_OVERFLOW;
  const bool sqsym = (o->flags & FL_SQSYM) != 0;
  for (uint64_t q = 0; q < s; ++q) {
    const Draw dr = o->wedge ? draw_wedge(*o, seed, first + q) : draw_diamond(*o, seed, first + q);
    if ((o->flags & FL_EXCLUDE_DIAG) && dr.i == dr.j) {
      ++o->diag_skipped;
    } else if (dr.v != 0) {
      o->X[pair_key(*o, dr.i, dr.j)] += dr.v;
      ++o->inserted;
    }
    if (!sqsym) continue;
    if ((o->flags & FL_EXCLUDE_DIAG) && dr.k == dr.kp) {
      ++o->diag_skipped;
    } else if (dr.v != 0) {
      o->X[pair_key(*o, dr.k, dr.kp)] += dr.v;
      ++o->inserted;
    }
  }
  o->sampled += s;
  return ST_OK;
}

void or_reset(void* h) {
  Oracle* o = (Oracle*)h;
  o->X.clear();
  o->sampled = o->inserted = o->diag_skipped = 0;
}

// X in ascending key order; returns |X| (entries with x = 0 included).
int64_t or_x_export(void* h, uint64_t* keys, int64_t* vals) {
  Oracle* o = (Oracle*)h;
  std::vector<std::pair<uint64_t, int64_t>> all(o->X.begin(), o->X.end());
  std::sort(all.begin(), all.end());
  if (keys)
    for (size_t q = 0; q < all.size(); ++q) {
      keys[q] = all[q].first;
      vals[q] = all[q].second;
    }
  return (int64_t)all.size();
}

// Alg. 3, first step: Omega_s = {x > 0}; the t' largest by (x desc,
// key asc).  Returns |Omega_t'| <= t'.
int64_t or_topk(void* h, uint64_t tprime, uint64_t* keys, int64_t* xs) {
  Oracle* o = (Oracle*)h;
  std::vector<std::pair<uint64_t, int64_t>> pos;
  for (const auto& kv : o->X)
    if (kv.second > 0) pos.push_back(kv);
  std::sort(pos.begin(), pos.end(), [](const std::pair<uint64_t, int64_t>& a,
                                       const std::pair<uint64_t, int64_t>& b) {
    if (a.second != b.second) return a.second > b.second;
    return a.first < b.first;
  });
  const size_t cnt = std::min<size_t>(pos.size(), tprime);
  for (size_t q = 0; q < cnt; ++q) {
    keys[q] = pos[q].first;
    xs[q] = pos[q].second;
  }
  return (int64_t)cnt;
}

// Alg. 3, dot products of the candidates: FP64 for dense inputs, exact
// counts for 0/1 CSR inputs.
void or_rescore(void* h, int64_t count, const uint64_t* keys, double* c) {
  Oracle* o = (Oracle*)h;
  for (int64_t q = 0; q < count; ++q) {
    const uint32_t i = (uint32_t)(keys[q] >> 32), j = (uint32_t)keys[q];
    c[q] = o->integer ? csr_dot(*o, i, j) : dense_dot(*o, i, j);
  }
}

// Alg. 3, last step: the t largest by (|c| desc, key asc).
int64_t or_topt(int64_t count, const uint64_t* keys, const double* c, uint64_t t,
                uint64_t* out_keys, double* out_c) {
  std::vector<Scored> v(count);
  for (int64_t q = 0; q < count; ++q) v[q] = {keys[q], c[q]};
  std::sort(v.begin(), v.end(), by_abs_c);
  const int64_t cnt = std::min<int64_t>(count, (int64_t)t);
  for (int64_t q = 0; q < cnt; ++q) {
    out_keys[q] = v[q].key;
    out_c[q] = v[q].c;
  }
  return cnt;
}

// Exact top-t by brute force over all pairs (ground truth of Defn. 1):
// long-double sequential dot products, (|c| desc, key asc).  Gram inputs
// enumerate unordered pairs; the diagonal is skipped when asked.
int64_t or_bruteforce(void* h, uint64_t t, uint64_t* out_keys, double* out_c) {
  Oracle* o = (Oracle*)h;
  std::vector<long double> bcol(o->d);
  std::vector<Scored> best;
  std::vector<long double> dense_b;
  // Column j of B as a dense vector (both formats).
  std::vector<std::vector<std::pair<int32_t, double>>> bcols(o->n);
  for (int64_t k = 0; k < o->d; ++k)
    for (int64_t e = o->B.ptr[k]; e < o->B.ptr[k + 1]; ++e)
      if (o->B.val[e] != 0.0) bcols[o->B.col[e]].push_back({(int32_t)k, o->B.val[e]});
  std::vector<long double> arow(o->d, 0.0L);
  for (int64_t i = 0; i < o->m; ++i) {
    std::fill(arow.begin(), arow.end(), 0.0L);
    for (int64_t e = o->A.ptr[i]; e < o->A.ptr[i + 1]; ++e) arow[o->A.col[e]] = o->A.val[e];
    for (int64_t j = 0; j < o->n; ++j) {
      if ((o->flags & FL_GRAM) && j < i) continue;
      if ((o->flags & FL_EXCLUDE_DIAG) && j == i) continue;
      long double acc = 0.0L;
      for (const auto& kb : bcols[j]) acc += arow[kb.first] * (long double)kb.second;
      best.push_back({((uint64_t)i << 32) | (uint64_t)j, (double)acc});
    }
    if (best.size() > 4 * t + 4096) {
      std::nth_element(best.begin(), best.begin() + t, best.end(), by_abs_c);
      best.resize(t);
    }
  }
  std::sort(best.begin(), best.end(), by_abs_c);
  const int64_t cnt = std::min<int64_t>((int64_t)best.size(), (int64_t)t);
  for (int64_t q = 0; q < cnt; ++q) {
    out_keys[q] = best[q].key;
    out_c[q] = best[q].c;
  }
  return cnt;
}

// Exact top-t by the row-wise sparse product (the paper's exact computation
// for comparison, Sec. 4.3, written for sparse inputs): row i of C is the
// sum over the stored entries a_ik of a_ik times row k of B, accumulated in
// a dense vector over j; every stored c_ij of the row (an entry that some k
// reaches) is a candidate, with the same pair rules as or_bruteforce (Gram:
// unordered pairs, j >= i; the diagonal skipped when asked).  Pairs that no
// k reaches have c_ij = 0 and are candidates only when fewer than t stored
// entries exist; they are not enumerated, so the result holds
// min(t, #stored candidates) pairs.  Sums are long double in ascending k
// (exact integers for 0/1 inputs).  Order (|c| desc, key asc).
int64_t or_sparse_exact(void* h, uint64_t t, uint64_t* out_keys, double* out_c) {
  Oracle* o = (Oracle*)h;
  std::vector<long double> acc(o->n, 0.0L);
  std::vector<char> seen(o->n, 0);
  std::vector<int64_t> touched;
  std::vector<Scored> best;
  for (int64_t i = 0; i < o->m; ++i) {
    touched.clear();
    for (int64_t e = o->A.ptr[i]; e < o->A.ptr[i + 1]; ++e) {
      const int64_t k = o->A.col[e];
      const long double a = (long double)o->A.val[e];
      for (int64_t f = o->B.ptr[k]; f < o->B.ptr[k + 1]; ++f) {
        const int64_t j = o->B.col[f];
        if (!seen[j]) {
          seen[j] = 1;
          touched.push_back(j);
        }
        acc[j] += a * (long double)o->B.val[f];
      }
    }
    for (const int64_t j : touched) {
      const long double c = acc[j];
      acc[j] = 0.0L;
      seen[j] = 0;
      if ((o->flags & FL_GRAM) && j < i) continue;
      if ((o->flags & FL_EXCLUDE_DIAG) && j == i) continue;
      best.push_back({((uint64_t)i << 32) | (uint64_t)j, (double)c});
    }
    if (best.size() > 4 * t + 4096) {
      std::nth_element(best.begin(), best.begin() + t, best.end(), by_abs_c);
      best.resize(t);
    }
  }
  std::sort(best.begin(), best.end(), by_abs_c);
  const int64_t cnt = std::min<int64_t>((int64_t)best.size(), (int64_t)t);
  for (int64_t q = 0; q < cnt; ++q) {
    out_keys[q] = best[q].key;
    out_c[q] = best[q].c;
  }
  return cnt;
}

// Wedge law for tiny instances (the appendix's Lemma on the wedge event):
// every wedge (i, k, j) with its probability under the oracle's tables and
// its increment.  Returns the number of wedges with nonzero probability.
int64_t or_enumerate_wedges(void* h, int64_t cap, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            double* prob, int64_t* ov) {
  Oracle* o = (Oracle*)h;
  if (!o->wedge) return -1;
  const Mat& B = o->B;
  int64_t cnt = 0;
  const long double tk = (long double)o->TK[o->d - 1];
  for (int64_t k = 0; k < o->d; ++k) {
    const uint64_t qk = o->TK[k] - (k ? o->TK[k - 1] : 0);
    if (qk == 0) continue;
    const int64_t c0 = o->Acol_ptr[k], clen = o->Acol_ptr[k + 1] - c0;
    const int64_t b0 = B.ptr[k], blen = B.ptr[k + 1] - b0;
    const long double ta = (long double)o->TAc[c0 + clen - 1];
    const long double tb = (long double)o->TB[b0 + blen - 1];
    for (int64_t pi = 0; pi < clen; ++pi) {
      const uint32_t qi = o->TAc[c0 + pi] - (pi ? o->TAc[c0 + pi - 1] : 0);
      if (qi == 0) continue;
      for (int64_t pj = 0; pj < blen; ++pj) {
        const uint32_t qj = o->TB[b0 + pj] - (pj ? o->TB[b0 + pj - 1] : 0);
        if (qj == 0) continue;
        if (cnt < cap) {
          int64_t v = 1;
          if (!o->integer && !(o->flags & FL_NONNEG)) {
            if (o->Acol_val[c0 + pi] < 0.0f) v = -v;
            if (B.valf[b0 + pj] < 0.0f) v = -v;
          }
          oi[cnt] = (uint32_t)o->Acol_row[c0 + pi];
          ok[cnt] = (uint32_t)k;
          oj[cnt] = (uint32_t)B.col[b0 + pj];
          prob[cnt] = (double)(((long double)qk / tk) * ((long double)qi / ta) *
                               ((long double)qj / tb));
          ov[cnt] = v;
        }
        ++cnt;
      }
    }
  }
  return cnt;
}

// Lemma 1 / Lemma 2 enumerator for tiny instances: the exact probability of
// every three-path (k', i, k, j) under the oracle's tables and its
// increment.  Writes up to cap rows (i, k, j, k', prob, v) and returns the
// number of three-paths with nonzero probability.
int64_t or_enumerate(void* h, int64_t cap, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                     uint32_t* okp, double* prob, int64_t* ov) {
  Oracle* o = (Oracle*)h;
  const Mat& A = o->A;
  const Mat& B = o->B;
  int64_t cnt = 0;
  const long double T1tot = (long double)o->T1[o->m - 1];
  for (int64_t i = 0; i < o->m; ++i) {
    const uint64_t qi = o->T1[i] - (i ? o->T1[i - 1] : 0);
    if (qi == 0) continue;
    const int64_t a0 = A.ptr[i], alen = A.ptr[i + 1] - a0;
    const long double t2 = (long double)o->T2[a0 + alen - 1];
    const long double ta = (long double)o->TA[a0 + alen - 1];
    for (int64_t pk = 0; pk < alen; ++pk) {
      const uint32_t qk = o->T2[a0 + pk] - (pk ? o->T2[a0 + pk - 1] : 0);
      if (qk == 0) continue;
      const int64_t k = A.col[a0 + pk];
      const int64_t b0 = B.ptr[k], blen = B.ptr[k + 1] - b0;
      const long double tb = (long double)o->TB[b0 + blen - 1];
      for (int64_t pj = 0; pj < blen; ++pj) {
        const uint32_t qj = o->TB[b0 + pj] - (pj ? o->TB[b0 + pj - 1] : 0);
        if (qj == 0) continue;
        const int64_t j = B.col[b0 + pj];
        for (int64_t pkp = 0; pkp < alen; ++pkp) {
          const uint32_t qkp = o->TA[a0 + pkp] - (pkp ? o->TA[a0 + pkp - 1] : 0);
          if (qkp == 0) continue;
          const int64_t kp = A.col[a0 + pkp];
          if (cnt < cap) {
            float bf = 0.0f;
            b_value(*o, kp, j, &bf);
            int64_t v;
            if (o->integer) {
              v = bf != 0.0f ? 1 : 0;
            } else {
              v = (int64_t)std::llrint(std::ldexp((double)bf, o->F));
              if (!(o->flags & FL_NONNEG)) {
                int sgn = 1;
                if (A.valf[a0 + pk] < 0.0f) sgn = -sgn;
                if (B.valf[b0 + pj] < 0.0f) sgn = -sgn;
                if (A.valf[a0 + pkp] < 0.0f) sgn = -sgn;
                v *= sgn;
              }
            }
            oi[cnt] = (uint32_t)i;
            ok[cnt] = (uint32_t)k;
            oj[cnt] = (uint32_t)j;
            okp[cnt] = (uint32_t)kp;
            prob[cnt] = (double)(((long double)qi / T1tot) * ((long double)qk / t2) *
                                 ((long double)qj / tb) * ((long double)qkp / ta));
            ov[cnt] = v;
          }
          ++cnt;
        }
      }
    }
  }
  return cnt;
}

}  // extern "C"
