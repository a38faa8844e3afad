// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mad.h"

namespace mad {

// ---------------------------------------------------------------------------
// Device error bits (sticky per context).
// ---------------------------------------------------------------------------
enum : uint32_t {
  DERR_HASH_FULL = 1u,     // an insert ran past the probe limit
  DERR_SEARCH = 2u,        // an inverse-CDF search left its row (corrupt table)
  DERR_OVERFLOW = 4u,      // an integer table total left its range
  DERR_EMPTY = 8u,         // ||W||_1 == 0
  DERR_SELECT = 16u,       // a per-query selection held more candidates than it keeps
};

constexpr uint64_t EMPTY_KEY = ~0ull;
constexpr uint32_t SIGN_BIT = 0x80000000u;
constexpr uint32_t PREFIX_MASK = 0x7FFFFFFFu;

// Scalars produced and consumed on the device.
struct DevScalars {
  unsigned int maxr_bits;          // FP32 bits of max_i r_i (nonnegative)
  unsigned int maxb_bits;          // FP32 bits of max |b_kj|
  int e1;                          // row-table exponent
  int pad0;
  unsigned long long t1_total;     // last entry of T1
  unsigned int err;                // DERR_* bits
  unsigned int pad1;
  unsigned long long inserted;     // diamonds accumulated
  unsigned long long diag_skipped; // diamonds with i == j (dropped)
  unsigned long long new_keys;     // keys created by sampling
  unsigned long long distinct;     // occupied slots (compaction)
  unsigned long long positive;     // slots with x > 0 (compaction)
  unsigned long long maxp;         // largest select key (compaction)
  // Derived from T1's total on the device, so that nothing between the
  // table build and the sampler waits for the host:
  int f_exp;                       // F of the dense increments
  int t1g_sh;                      // bucket shift of T1's guide
  int sort_shift;                  // bucket shift of the row-order sort
  int pad2;
};

// Everything a sampling kernel needs, passed by value.
// Alias tables (Sec. 4.1): per column a threshold t in [0, X] over the
// table's total X and an alias; a draw takes a column uniformly, keeps it
// with probability t / X, else returns the alias.  Tables longer than
// kAliasSeg entries have two levels (segments of kAliasSeg entries, and a
// table over the segment totals).  A family holds one table per row: row r
// stores its segments' entries (L) and then its top-level entries (nseg).
constexpr int64_t kAliasSeg = 1024;
struct AliasEnt {
  unsigned long long t;
  uint32_t a;
  uint32_t pad;
};
// Families: 0 T1 (one row over the rows of A), 1 T2 and 2 TA (one row per
// row of A), 3 TB (one row per row of B).
enum { kAlT1 = 0, kAlT2 = 1, kAlTA = 2, kAlTB = 3 };

struct SampleParams {
  // A (m x d): dense row-major or 0/1 CSR.
  const void* a_val;
  const int64_t* a_ptr;
  const int32_t* a_col;
  int64_t m, d, lda;
  // B (d x n).
  const void* b_val;
  const int64_t* b_ptr;
  const int32_t* b_col;
  int64_t n, ldb;
  // Tables.
  const uint64_t* T1;
  const uint32_t* T2;
  const uint32_t* TA;
  const uint32_t* TB;
  unsigned long long t1_total;
  // Guides of the long 0/1 T2 rows (null when absent): row i's guide is
  // T2g[T2g_ptr[i] .. T2g_ptr[i+1]) with bucket width 2^T2g_sh[i]; entry b
  // counts the row's prefix entries below b << T2g_sh[i].
  const unsigned long long* T2g_ptr;
  const uint32_t* T2g;
  const uint8_t* T2g_sh;
  // Bloom filter over the entries the 0/1 closure test looks up (null when
  // absent): word mix64(key) >> bloom_shift holds five bits of each key.
  const unsigned long long* bloom;
  int bloom_shift;
  // Guide of T1 (null when absent): entry b counts the prefix entries
  // below b << t1g_sh.
  const uint32_t* T1g;
  int t1g_sh;
  // Guides of the dense TB rows (null when absent): row k's guide starts
  // at TBg + k * tbg_stride, bucket width 2^TBg_sh[k].
  const uint32_t* TBg;
  int64_t tbg_stride;
  const uint8_t* TBg_sh;
  int f_exp;                       // F
  // Hash.  Regioned (dense inputs): the key (a, b) starts probing in the
  // home region of row a, [hreg[a], hreg[a+1]), sized from row a's expected
  // share of the diamonds; otherwise at mix(key) & hmask.  Probing is
  // linear and wraps at hcap (for regioned hashes, the end of the regions,
  // read on the device and kept within the hcap_alloc allocated slots).
  unsigned long long* hkeys;
  long long* hvals;
  const unsigned long long* hreg;
  uint64_t hmask;
  uint64_t hcap;
  uint64_t hcap_alloc;
  uint32_t max_probe;
  int regioned;
  // Modes.
  int dense;                       // 1 dense A and B, 0 CSR
  int a_f64, b_f64;                // dense dtypes
  int integer;                     // 0/1 exact mode
  uint32_t flags;                  // MAD_NONNEG | MAD_GRAM | MAD_EXCLUDE_DIAG
  DevScalars* sc;
  // Alias draws (MAD_ALIAS): the four families, their segment and row
  // totals and segment counts.
  int alias;
  const AliasEnt* al[4];
  const unsigned long long* al_seg[4];
  const unsigned long long* al_row[4];
  int al_nseg[4];
};

// Select item: primary key p (larger first), tie key (smaller first), aux.
struct Item {
  unsigned long long p;
  unsigned long long key;
  unsigned long long aux;
};

}  // namespace mad

// ---------------------------------------------------------------------------
// Context (host side).
// ---------------------------------------------------------------------------
struct mad_ctx {
  uint32_t flags = 0;
  int device = 0;
  // Private stream-ordered pool for every table, the hash and the scratch:
  // it keeps freed memory mapped, so rebuilding tables of the same shape
  // re-uses pages instead of mapping them again.
  cudaMemPool_t pool = nullptr;
  // Second stream of the dense table build: B^T and the TB guides need only
  // TB, so they run beside the A-row tables and T1 (forked and joined with
  // the two events; captured as parallel branches in a CUDA graph).
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_fork2 = nullptr, ev_join = nullptr;
  // Caller events recorded at the sampling phase boundaries (profiling).
  cudaEvent_t phase_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  uint32_t n_phase_ev = 0;
  bool built = false;
  bool integer = false;
  bool dense = false;
  mad_matrix A{}, B{};
  int64_t m = 0, d = 0, n = 0;
  uint64_t nnz_a = 0, nnz_b = 0;
  uint64_t s_max = 0, sampled = 0;
  int e1 = 0, f = 0;
  unsigned long long t1_total = 0;
  // Owned device memory.
  uint64_t* T1 = nullptr;
  uint32_t* T2 = nullptr;
  uint32_t* TA = nullptr;
  uint32_t* TB = nullptr;
  float* na = nullptr;
  float* nb = nullptr;
  float* r = nullptr;
  unsigned long long* r64 = nullptr;
  unsigned long long* T2g_ptr = nullptr;  // guides of long 0/1 T2 rows
  uint32_t* T2g = nullptr;
  uint8_t* T2g_sh = nullptr;
  unsigned long long* bloom = nullptr;    // closure-test filter (0/1 inputs)
  int bloom_lg = 0;
  uint32_t* T1g = nullptr;                // guide of T1
  int t1g_sh = 0;
  unsigned long long t2g_total = 0;       // entries of the 0/1 T2 guides
  uint32_t* TBg = nullptr;                // guides of the TB rows (fixed row stride)
  int64_t tbg_stride = 0;
  uint8_t* TBg_sh = nullptr;
  // Wedge sampling (MAD_WEDGE): the centre table TK over k (its inclusive
  // prefix starts at TK + TK_shift), its total and scale exponent, the
  // column norms of A and, for dense non-Gram inputs, the column tables.
  unsigned long long* TK = nullptr;
  int TK_shift = 0;
  unsigned long long tk_total = 0;
  int ek = 0;
  float* nac = nullptr;
  uint32_t* TAc = nullptr;
  // Alias draws (MAD_ALIAS): per family its entries, segment totals, row
  // totals and segment count.
  mad::AliasEnt* al[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long* al_seg[4] = {nullptr, nullptr, nullptr, nullptr};
  unsigned long long* al_row[4] = {nullptr, nullptr, nullptr, nullptr};
  int al_nseg[4] = {0, 0, 0, 0};
  // Fused pass (mad_pipeline_*): budgets fixed when planned, one buffer
  // for its selection lists.
  bool pipe = false;
  uint64_t pipe_s = 0;
  uint32_t pipe_tprime = 0, pipe_t = 0;
  uint64_t pipe_list_cap = 0;             // compacted candidates the pass holds
  void* pipe_buf = nullptr;
  // The pass's own scratch (a captured run keeps its addresses however the
  // context's shared scratch changes later).
  void* pipe_scratch = nullptr;
  size_t pipe_scratch_bytes = 0;
  bool scratch_fixed = false;       // no reallocation while a pass is enqueued
  // Batched queries: the plan of the current batch.
  bool mips_items = false;
  uint32_t mips_nq = 0, mips_tprime = 0, mips_t = 0;
  uint64_t mips_chunks = 0;
  unsigned long long* mips_s = nullptr;   // nq budgets
  uint32_t* mips_chunk_q = nullptr;       // query of each 256-diamond chunk
  uint32_t* mips_chunk_l0 = nullptr;      // its first diamond
  // Launch shape of batched queries (mad_mips_config): region size factor
  // 2^mips_region_lg, 256 x mips_chunk_mult diamonds per chunk (the plan's
  // value in mips_plan_mult), sampler blocks per SM (0: as many as fit),
  // select threads per query.
  int mips_region_lg = 1;
  int mips_chunk_mult = 1;
  int mips_plan_mult = 1;
  int mips_bps = 0;
  int mips_select_threads = 256;
  void* bt = nullptr;               // dense B^T (n x d), the input dtype
  unsigned long long* hkeys = nullptr;
  long long* hvals = nullptr;
  // Dense inputs: row i's home region is [hreg[i], hreg[i+1]) (m + 2
  // offsets; hreg[m] is the end of the regions, followed by an overflow
  // table of hov slots that only the fused pass's region builder fills;
  // hreg[m+1] = hreg[m] + hov is the end of X).
  unsigned long long* hreg = nullptr;
  bool regioned = false;
  uint64_t hcap = 0, hcap_alloc = 0, hcap_request = 0, hov = 0;
  // Region size factor and overflow table request (0: default) of the
  // dense hash.
  float region_factor = 1.5f;
  uint64_t hov_request = 0;
  mad::DevScalars* sc = nullptr;
  // Scratch (select, scans); grown on demand.
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  // Grouping buffer of the 0/1 Gram rescoring, for up to rg_cap candidates.
  void* rg_buf = nullptr;
  uint64_t rg_cap = 0;
  // Host-side fault injection (MAD_FAULT=oom[:N]): the allocation number
  // from which pool allocations fail (0: off), and allocations so far.
  int64_t fault_oom_at = 0;
  int64_t allocs = 0;
  // Host mirrors.
  uint64_t launches = 0;
  uint64_t distinct = 0, positive = 0;
  uint32_t device_error = 0;
};

namespace mad {

// Launch bookkeeping: every kernel launch of the library goes through this.
inline void count_launch(mad_ctx* ctx, int n = 1) { ctx->launches += (uint64_t)n; }

mad_status cuda_status(cudaError_t e);
// The one device allocation path of a context (its stream-ordered pool),
// with the host-side fault injection of MAD_FAULT=oom[:N].
mad_status pool_malloc(mad_ctx* ctx, void** p, size_t bytes, cudaStream_t st);
mad_status ensure_scratch(mad_ctx* ctx, size_t bytes, cudaStream_t st);

// scan.cu: out[0..n] = exclusive prefix of in[0..n) and the total at
// out[n]; partial holds scan_partial_elems(n) elements.
size_t scan_partial_elems(uint64_t n);
mad_status scan_exclusive_u32(mad_ctx* ctx, const uint32_t* in, uint32_t* out, uint64_t n,
                              uint32_t* partial, cudaStream_t st);
mad_status scan_exclusive_u64(mad_ctx* ctx, const uint64_t* in, uint64_t* out, uint64_t n,
                              uint64_t* partial, cudaStream_t st);
// tables.cu
// Guides of the 0/1 T2 rows of at least kGuideMin entries (integer mode):
// sizes, shifts and offsets into ctx->T2g_ptr / T2g_sh (allocated by the
// caller, m + 1 and m entries; the total lands in T2g_ptr[m]), then the
// entries into ctx->T2g.
constexpr int kGuideMin = 64;
mad_status t2_guide_offsets(mad_ctx* ctx, cudaStream_t st);
// Bloom filter of the entries of the matrix the closure test reads (A under
// MAD_GRAM, else B) into ctx->bloom (2^bloom_lg words, cleared here).
mad_status build_bloom(mad_ctx* ctx, cudaStream_t st);
mad_status t2_guide_fill(mad_ctx* ctx, cudaStream_t st);
// Guides of the dense TB rows into ctx->TBg (d rows of ctx->tbg_stride =
// 2^tb_guide_width(n) + 1 entries) and ctx->TBg_sh (d shifts).
int tb_guide_width(int64_t n);
mad_status tb_guide_build(mad_ctx* ctx, cudaStream_t st);
// Guide of T1 into ctx->T1g, at most 2^t1_guide_width(m) + 1 entries; its
// shift and length come from T1's total on the device.
int t1_guide_width(int64_t m);
mad_status t1_guide_fill(mad_ctx* ctx, cudaStream_t st);
// Batched queries: the item-side tables (TB, nb, maximum |b|, B^T) and the
// query rows (T2, TA).
mad_status build_item_tables(mad_ctx* ctx, cudaStream_t st);
mad_status build_query_rows(mad_ctx* ctx, cudaStream_t st);
// side_branch: dense inputs launch B^T and the TB guides on ctx->side
// (after TB, joined by the caller through ctx->ev_join); otherwise B^T is
// launched on st and the caller builds the TB guides.
mad_status build_tables_impl(mad_ctx* ctx, cudaStream_t st, bool side_branch = false);
// Empties the hash slots [*lo_dev, min(bound, *hi_dev)) with bound =
// hash_slot_bound(ctx) (0 without lo_dev, bound without hi_dev).
mad_status clear_slots(mad_ctx* ctx, const unsigned long long* lo_dev,
                       const unsigned long long* hi_dev, cudaStream_t st);
// Home regions of the dense hash: sizes from T1 and s_max, then offsets.
mad_status build_hash_regions(mad_ctx* ctx, cudaStream_t st);
uint64_t hash_region_bound(uint64_t m, uint64_t s_max);
// End of the dense hash on the device (the end of the home regions and
// their overflow table), else null (the whole ctx->hcap).
inline const unsigned long long* hash_extent(const mad_ctx* ctx) {
  return ctx->regioned ? ctx->hreg + ctx->m + 1 : nullptr;
}
// Slots of the overflow table after the home regions.
uint64_t hash_overflow_slots(uint64_t s_max);
// Host-side bound on the slots a scan of the hash may touch: the
// allocation for regioned hashes (their extent is read on the device).
inline uint64_t hash_slot_bound(const mad_ctx* ctx) {
  return ctx->regioned ? ctx->hcap_alloc : ctx->hcap;
}
// sample.cu
// Diamonds among the first n of a fixed pilot seed that would add to X
// (closed, nonzero, off-diagonal when excluded); synchronises.
mad_status pilot_inserts(mad_ctx* ctx, uint64_t n, uint64_t* hits, cudaStream_t st);
// Whether a sampling call of s diamonds into an empty X may build the home
// regions whole (dense, non-Gram, one sorted batch); X then needs no
// clearing beforehand.
bool x_builder_applies(const mad_ctx* ctx, uint64_t s);
// fresh_x: X is empty and this call is its only filling (the fused pass):
// where x_builder_applies, the home regions are built whole.
mad_status sample_impl(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first,
                       cudaStream_t st, bool fresh_x = false);
mad_status debug_draws_impl(mad_ctx* ctx, uint64_t seed, uint64_t first, const uint64_t* ells,
                            uint64_t count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            uint32_t* okp, int64_t* ov, cudaStream_t st);
SampleParams make_params(const mad_ctx* ctx);
// select.cu
// Workspace of one top-K selection over at most n items.
struct SelectWs {
  Item* l0;          // input list (n items), preserved
  Item* l1;          // ping-pong survivor lists
  Item* l2;
  Item* out;         // K selected items, sorted (padded to a power of two)
  void* state;
  unsigned long long* counter;
  uint64_t cap_n, cap_out;
};
size_t select_ws_bytes(uint64_t n, uint64_t K);
SelectWs select_ws_carve(void* base, uint64_t n, uint64_t K);
// K largest of ws.l0[0..n) by (p desc, key asc), sorted into ws.out.  dp =
// number of significant bytes of the largest p.  Asynchronous.
mad_status select_list(mad_ctx* ctx, const SelectWs& ws, uint64_t n, uint64_t K, int dp,
                       uint64_t* n_sel, cudaStream_t st);
// Omega_t': the K largest positive x of the hash, sorted into ws.out.
// *n_pos receives the number of positive keys.  Synchronises once.
mad_status select_from_hash(mad_ctx* ctx, const SelectWs& ws, uint64_t K, uint64_t* n_sel,
                            uint64_t* n_pos, cudaStream_t st);
mad_status items_to_pairs(mad_ctx* ctx, const Item* items, uint64_t n, const mad_pair* cand,
                          const double* cvals, mad_pair* out, cudaStream_t st);
// Device-driven selection: every length comes from device memory, so the
// host enqueues the whole selection without waiting (CUDA-graph capturable).
// The K largest of the first min(cap, *n_dev) items of `in` (cap <= 2^17)
// are sorted into out[0..min(K, n)); sorted and pos hold cap entries.  When
// over_err is given, a device length above cap sets DERR_SELECT there.
void tile_select_dev(mad_ctx* ctx, const Item* in, uint64_t cap, uint64_t K,
                     const unsigned long long* n_dev, unsigned int* over_err, Item* sorted,
                     uint32_t* pos, Item* out, cudaStream_t st,
                     const unsigned int* gate = nullptr);
// The same set, selected in one block when min(cap, *n_dev) <= 16384 (in no
// particular order unless `sorted` and K <= 2048); longer lists fall back to
// the tile kernels through the device word *gate (sorted output).
void block_select_dev(mad_ctx* ctx, const Item* in, uint64_t cap, uint64_t K,
                      const unsigned long long* n_dev, bool sorted, Item* tile_sorted,
                      uint32_t* pos, Item* out, unsigned int* gate, unsigned int* over_err,
                      cudaStream_t st);
constexpr uint64_t kDevSelectCap = 1ull << 17;
size_t dev_select_state_bytes();
// Omega_t' from the hash whose extent is *hcap_dev slots (at most
// ctx->hcap): the positive x at or above a log-bucket threshold (estimated
// from one 4-slot group in 8, the exact histogram as a gated fallback) are
// compacted into list (kDevSelectCap entries, count at *count), then the K
// largest go to out, in no particular order when one block selects them
// (lists up to 16384 items), else sorted.  count[1..2] are gate words.
void select_hash_dev(mad_ctx* ctx, uint64_t K, const unsigned long long* hcap_dev, void* state,
                     unsigned long long* count, Item* list, Item* sorted, uint32_t* pos,
                     Item* out, cudaStream_t st);
// The same Omega_t' for candidate lists longer than kDevSelectCap (0/1
// inputs, whose small integer x tie in large numbers at the K-th value):
// the x at or above the exact log-bucket threshold are compacted into list
// (list_cap entries; more is reported as DERR_SELECT), the K first by
// (x desc, key asc) are found by an MSB radix select on the device length
// (ping-pong lists l1, l2 of list_cap entries) and collected into topk,
// then sorted into out (K <= kDevSelectCap).  count[0..3] are device words.
void select_hash_dev_long(mad_ctx* ctx, uint64_t K, const unsigned long long* hcap_dev,
                          void* state, unsigned long long* count, Item* list, Item* l1, Item* l2,
                          uint64_t list_cap, Item* topk, Item* sorted, uint32_t* pos, Item* out,
                          cudaStream_t st);
// out[q] for q < min(cap, *n_dev) as in items_to_pairs; *n_out gets that
// length.
void items_to_pairs_dev(mad_ctx* ctx, const Item* items, uint64_t cap,
                        const unsigned long long* n_dev, const mad_pair* cand,
                        const double* cvals, mad_pair* out, uint32_t* n_out, cudaStream_t st);
int significant_bytes(unsigned long long maxp);
mad_status export_x(mad_ctx* ctx, uint64_t* keys, int64_t* vals, uint64_t cap, uint64_t* n,
                    unsigned long long* counter, cudaStream_t st);
// Sharded runs: X's occupied slots grouped by owner rank (offsets_host gets
// world + 1 segment bounds; nothing is written when the total exceeds cap;
// uses 8 (3 world + 1) bytes of scratch), and the K largest x > 0 of a pair
// list by (x desc, key asc), copied from the input pairs.
mad_status export_x_by_owner(mad_ctx* ctx, uint32_t world, uint64_t* keys, int64_t* vals,
                             uint64_t cap, uint64_t* offsets_host, cudaStream_t st);
mad_status select_pairs(mad_ctx* ctx, const mad_pair* pairs, uint64_t n, uint64_t K,
                        mad_pair* out, uint64_t* n_sel, cudaStream_t st);
// wedge.cu: wedge sampling (MAD_WEDGE contexts): the plain hash's slots for
// s_max wedges, the centre and column tables (after the diamond tables;
// synchronises), the sampling loop and its diagnostic draws.
// Alias tables of a built dense float context (MAD_ALIAS); refuses 0/1
// inputs and tables of more than kAliasSeg segments.
mad_status build_alias_tables(mad_ctx* ctx, cudaStream_t st);
uint64_t wedge_hash_slots(uint64_t s_max);
mad_status build_wedge_tables(mad_ctx* ctx, cudaStream_t st);
mad_status wedge_sample_impl(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first,
                             cudaStream_t st);
mad_status wedge_draws_impl(mad_ctx* ctx, uint64_t seed, uint64_t first, const uint64_t* ells,
                            uint64_t count, uint32_t* oi, uint32_t* ok, uint32_t* oj,
                            uint32_t* okp, int64_t* ov, cudaStream_t st);
// sample.cu: (key, value) pairs added to X.
mad_status accumulate_pairs(mad_ctx* ctx, const uint64_t* keys, const int64_t* vals, uint64_t n,
                            cudaStream_t st);
// dense_topt.cu: the comparator; dense_out != NULL writes the full product.
mad_status dense_comparator(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                            uint32_t rescore, mad_pair* out, uint32_t* n_out, float* dense_out,
                            cudaStream_t st);
// api.cu
// Status of the device error word (DERR_* bits).
mad_status device_error_status(uint32_t err);
// Host copy of the device scalars (synchronises; sets ctx->device_error).
mad_status read_device_scalars(mad_ctx* ctx, DevScalars* hs, cudaStream_t st);
// Every slot of X empty, up to the hash's extent (asynchronous).
mad_status clear_x(mad_ctx* ctx, cudaStream_t st);
// Input checks and allocation of the tables of a dense build (frees the
// previous ones).
mad_status plan_dense_tables(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                             uint64_t s_max, cudaStream_t st);
size_t dense_build_scratch_bytes(const mad_ctx* ctx);
// The dense table build enqueued without waiting for the device, and the
// host mirrors read afterwards (synchronises).
mad_status enqueue_dense_build(mad_ctx* ctx, cudaStream_t st, bool clear_x = true);
mad_status finish_dense_build(mad_ctx* ctx, cudaStream_t st);
// sample.cu: scratch of sample_impl for s diamonds, and the number of bits
// of the row-order sort's buckets (at most 16, about log2 m).
size_t sample_scratch_bytes(const mad_ctx* ctx, uint64_t s);
int sort_bits(int64_t m);
// rescore.cu
// Exact c for every candidate: items[q] = (bits |c|, key, q), cvals[q] = c.
// With n_dev, the candidates are the first min(ncand, *n_dev).
mad_status rescore_reserve(mad_ctx* ctx, uint64_t ncand, cudaStream_t st);
mad_status rescore_items(mad_ctx* ctx, const mad_pair* cand, uint64_t ncand, Item* items,
                         double* cvals, cudaStream_t st, const unsigned long long* n_dev = nullptr);

}  // namespace mad
