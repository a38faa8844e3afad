/*
 * mad.h -- C ABI of a GB300 (sm_103a) library for approximate Maximum
 * All-pairs Dot-product (MAD) search by diamond sampling.
 *
 * Paper: G. Ballard, T. G. Kolda, A. Pinar, C. Seshadhri, "Diamond Sampling
 * for Approximate Maximum All-pairs Dot-product (MAD) Search",
 * arXiv:1506.03872.
 *
 * Problem (Defn. 1): given A (m x d, rows a_i) and B (d x n, columns b_j),
 * find the t pairs (i, j) with the largest |a_i . b_j|.  The paper stores
 * vectors as columns (A^T B); here A holds them as rows, so a_ik below is
 * the paper's a_ki.
 *
 * Pipeline (one call per step, all asynchronous on the caller's stream):
 *   mad_build_tables  weights w_ik = |a_ik| ||a_i*||_1 ||b_k*||_1 and the
 *                     cumulative sampling tables (Alg. 2 weight line; Sec. 4.2)
 *   mad_sample        s diamonds: (i,k) ~ w_ik, j ~ |b_kj|, k' ~ |a_ik'|,
 *                     x_ij += sgn(a_ik b_kj a_ik') b_k'j (Alg. 2 loop)
 *   mad_topk          Omega_t': the t' largest positive x_ij (Alg. 3, step 1)
 *   mad_rescore       exact c_ij for the candidates, top t by |c| (Alg. 3)
 *
 * Numeric contract (fixed here because the paper leaves it open):
 *   - Weights are FP32; L1 norms use one fixed summation order (256 strided
 *     partial sums folded in halves).  Sampling tables are integer prefix
 *     sums (uint64 over rows of A, uint32 within a row) of the FP32 weights
 *     scaled by a power of two and rounded to nearest-even.
 *   - Diamond l draws its four 64-bit uniforms from Philox4x32-10 with key =
 *     seed and counter (l_lo, l_hi, 0, block), block 0 -> (i, k), block 1 ->
 *     (j, k'); a uniform u selects the first prefix entry exceeding
 *     floor(u * total / 2^64).
 *   - x_ij is int64 fixed point: b_k'j (FP32) times 2^F, F chosen from s_max
 *     and max|b| so that s_max increments cannot overflow.  0/1 CSR inputs
 *     run in exact integer mode (F = 0, x_ij counts diamonds).
 *   - Rescoring is FP64 (32 strided fused-multiply-add partial sums folded
 *     in halves) for dense inputs and exact integer counts for 0/1 inputs.
 *   Given the same inputs, seed and diamond range, every result is
 *   bit-identical run to run and independent of launch configuration.
 *
 * Memory: the caller owns A, B and every output buffer (device memory unless
 * a parameter says host).  A and B must stay alive and unchanged from
 * mad_build_tables until mad_destroy or the next mad_build_tables: sampling
 * and rescoring read them.  The library owns its tables, hash and scratch,
 * allocated stream-ordered on the stream of mad_build_tables.
 *
 * Errors: every call returns a status and never aborts.  Device-side
 * failures (hash probe limit, bad index) set a sticky flag that the next
 * synchronising call (mad_topk, mad_rescore, mad_stats) reports.
 * Thread safety: one context must not be used from two host threads at once.
 */
#ifndef MAD_H_
#define MAD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (the same type as cudaStream_t); NULL is the legacy
 * default stream. */
struct CUstream_st;
typedef struct CUstream_st* mad_stream;

typedef enum mad_status {
  MAD_OK = 0,
  MAD_ERR_ARG = 1,          /* bad shape, pointer, flag or size */
  MAD_ERR_OOM = 2,          /* device allocation failed */
  MAD_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  MAD_ERR_OVERFLOW = 4,     /* a table total or the diamond count exceeds its range */
  MAD_ERR_EMPTY = 5,        /* ||W||_1 == 0: no three-path exists */
  MAD_ERR_HASH_FULL = 6,    /* an insert exceeded the probe limit */
  MAD_ERR_STATE = 7,        /* call out of order (e.g. sample before tables) */
  MAD_ERR_UNSUPPORTED = 8   /* valid request outside what this build handles */
} mad_status;

typedef enum mad_format { MAD_DENSE_ROWMAJOR = 0, MAD_CSR = 1 } mad_format;
typedef enum mad_dtype { MAD_F32 = 0, MAD_F64 = 1, MAD_BINARY = 2 } mad_dtype;

/* A matrix in device memory.
 *   dense: values[r * ld + c], dtype MAD_F32 or MAD_F64, ld >= cols.
 *   CSR:   rowptr[rows + 1] (rowptr[0] == 0), colidx[rowptr[rows]] sorted
 *          ascending within each row, dtype MAD_BINARY (values == NULL,
 *          every stored entry is 1). */
typedef struct mad_matrix {
  int32_t fmt;              /* mad_format */
  int32_t dt;               /* mad_dtype */
  int64_t rows, cols, ld;
  const void* values;
  const int64_t* rowptr;
  const int32_t* colidx;
} mad_matrix;

/* One candidate or result pair: x is the sampled score (Alg. 2), c the
 * exact dot product a_i . b_j (Alg. 3).  24 bytes, 8-byte aligned. */
typedef struct mad_pair {
  uint32_t i, j;
  int64_t x;
  double c;
} mad_pair;

/* Context flags (mad_create).
 *   MAD_NONNEG        caller asserts A, B >= 0: the sign product of Alg. 2 is
 *                     skipped (Sec. 3.2.1).
 *   MAD_GRAM          caller asserts B = A^T, so C is symmetric: pairs are
 *                     accumulated unordered, key (min(i,j), max(i,j)), which
 *                     is twice the symmetrised X of Sec. 3.2.2 and ranks the
 *                     same.
 *   MAD_EXCLUDE_DIAG  diamonds with i == j are drawn but not accumulated
 *                     (the distinct-pairs application of Sec. 6.2).
 *   MAD_SQUARE_SYM    squared symmetric input (Sec. 3.2.3): with MAD_GRAM
 *                     and A = B = A^T (the caller guarantees symmetry),
 *                     each diamond (k', i, k, j) also adds its value to the
 *                     pair (k, k') (the paper adds half to each pair; the
 *                     whole value scales every x by 2 and orders the same).
 *                     Under MAD_EXCLUDE_DIAG a diagonal addition of either
 *                     kind is skipped.  0/1 inputs only.
 *   MAD_WEDGE         wedge sampling in place of diamond sampling (the
 *                     paper's comparison method, appendix "Previous
 *                     approach: Wedge sampling"): mad_sample draws wedges
 *                     (i, k, j) with k ~ ||a_*k||_1 ||b_k*||_1, i ~ |a_ik|
 *                     within column k of A and j ~ |b_kj| within row k of B
 *                     (the first three Philox uniforms of the wedge index)
 *                     and adds sgn(a_ik b_kj) to x_ij, so E[x_ij] = s c_ij /
 *                     ||w||_1.  mad_topk and mad_rescore apply as for
 *                     diamonds.  Dense inputs (d <= 1024) and 0/1 Gram
 *                     inputs (MAD_ERR_UNSUPPORTED for other 0/1 inputs); X is
 *                     a plain table of at least s_max / 0.6 slots; mad_stats
 *                     reports ||w||_1 in place of ||W||_1; not with
 *                     MAD_SQUARE_SYM or the fused pass. */
/* MAD_ALIAS:         draws from alias tables (Sec. 4.1 names the alias
 *                     method for constant-time draws): mad_build_tables
 *                     also builds, over the same integer weights as T1, the
 *                     rows of T2 and TA and the rows of TB, tables that give
 *                     each entry exactly its weight over the total (Vose's
 *                     method in exact integers; tables longer than 1024
 *                     entries have two levels, segments of 1024 and a table
 *                     over the segment totals).  mad_sample then draws each
 *                     of (i, k, j, k') from its alias table: a column from
 *                     the high bits of u * n, kept against its threshold by
 *                     the low bits, else its alias; the second level of a
 *                     two-level draw takes its uniform from Philox blocks 2
 *                     and 3 of the diamond.  Same law, another map from the
 *                     uniforms.  Dense float inputs with m and n up to 2^20
 *                     (MAD_ERR_UNSUPPORTED otherwise); not with MAD_WEDGE or
 *                     the fused pass. */
enum { MAD_NONNEG = 1u, MAD_GRAM = 2u, MAD_EXCLUDE_DIAG = 4u, MAD_SQUARE_SYM = 8u,
       MAD_WEDGE = 16u, MAD_ALIAS = 32u };

typedef struct mad_stats_t {
  double w1;                /* ||W||_1 as represented by the tables */
  uint64_t t1_total;        /* integer total of the row table */
  int32_t e1;               /* row-table scale exponent */
  int32_t f;                /* increment scale exponent (0 in integer mode) */
  uint64_t sampled;         /* diamonds drawn since the last reset */
  uint64_t inserted;        /* diamonds with a nonzero increment */
  uint64_t diag_skipped;    /* diamonds dropped because i == j */
  uint64_t distinct;        /* occupied hash slots (updated by mad_topk) */
  uint64_t positive;        /* keys with x > 0 (updated by mad_topk) */
  uint64_t hash_capacity;   /* hash slots */
  uint64_t launches;        /* kernels launched by this context so far */
  uint32_t integer_mode;    /* 1 for 0/1 inputs */
  uint32_t device_error;    /* sticky device error bits (0 = none) */
} mad_stats_t;

typedef struct mad_ctx mad_ctx;

/* Create a context on the current CUDA device.  flags: MAD_NONNEG |
 * MAD_GRAM | MAD_EXCLUDE_DIAG.  Returns MAD_ERR_ARG for unknown flags.
 * The context allocates its tables, hash and scratch from a private
 * stream-ordered memory pool that keeps freed pages mapped, so repeated
 * mad_build_tables calls of one shape do not map memory again. */
mad_status mad_create(mad_ctx** ctx, uint32_t flags);

/* Profiling aid (the paper has no counterpart).  From the next mad_sample
 * on, record n caller-created CUDA events (cudaEvent_t handles, n <= 4) on
 * the sampling stream at the phase boundaries of each batch of diamonds:
 * events[0] before the batch; events[1] after the row-order sort (dense
 * inputs; at the start for 0/1 inputs); events[2] after the draw kernel
 * (k_sample_sorted, or k_sample, which also inserts, for 0/1 inputs);
 * events[3] after the hash insert (k_insert; equal to events[2] for 0/1
 * inputs).  With several batches the events mark the last one.  The handles
 * must stay valid while set; n = 0 stops recording.  MAD_ERR_ARG for n > 4
 * or a null array with n > 0. */
mad_status mad_set_phase_events(mad_ctx* ctx, void* const* events, uint32_t n);

/* Free everything the context owns, its memory pool included
 * (synchronises the device). */
void mad_destroy(mad_ctx* ctx);

/* Static description of a status code. */
const char* mad_strerror(mad_status status);

/* Hash capacity in slots for the next mad_build_tables (a power of two,
 * >= 1024), or 0 for the default: the smallest power of two >= s_max / 0.6.
 * Each slot is 16 bytes. */
mad_status mad_set_hash_capacity(mad_ctx* ctx, uint64_t slots);

/* Alg. 2 weight line and the cumulative tables of Sec. 4.2.
 *   A: m x d, B: d x n (B->rows == A->cols).  Both dense (F32/F64, any mix)
 *   or both 0/1 CSR.  Dense inputs need d <= 1024.  m, n < 2^32.
 *   s_max: the most diamonds mad_sample may accumulate before the next
 *   mad_reset_hash; it fixes the increment scale F and the hash size.
 * Synchronises the stream once to read the table totals.  Errors:
 *   MAD_ERR_EMPTY when ||W||_1 == 0, MAD_ERR_OVERFLOW when a 0/1 table total
 *   exceeds its integer range, MAD_ERR_UNSUPPORTED for other formats. */
mad_status mad_build_tables(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                            uint64_t s_max, mad_stream stream);

/* Alg. 2 sampling loop for diamonds first_diamond .. first_diamond+s-1,
 * accumulated into the context's hash.  Calls may be repeated (resume or
 * split a run): any split of a diamond range gives the same X as one call.
 * Errors: MAD_ERR_STATE before mad_build_tables, MAD_ERR_OVERFLOW when the
 * diamonds since the last reset would exceed s_max.  Asynchronous. */
mad_status mad_sample(mad_ctx* ctx, uint64_t s, uint64_t seed, uint64_t first_diamond,
                      mad_stream stream);

/* Clear X (and the sampled count) without rebuilding tables. */
mad_status mad_reset_hash(mad_ctx* ctx, mad_stream stream);

/* Alg. 3, first step: Omega_t' = the min(t', |{x > 0}|) keys with the
 * largest x, ties broken by smaller (i, j); written to out_dev sorted by
 * (x desc, i asc, j asc) with c = 0.  Gram contexts report i < j.
 * *n_out_host receives the count.  Synchronises the stream. */
mad_status mad_topk(mad_ctx* ctx, uint32_t tprime, mad_pair* out_dev, uint32_t* n_out_host,
                    mad_stream stream);

/* Alg. 3, remaining steps: c_ij = a_i . b_j for each of the ncand candidates
 * (cand_dev, device), then the min(t, ncand) pairs with the largest |c|,
 * ties broken by smaller (i, j), sorted, written to out_dev with their x.
 * Uses the A and B given to mad_build_tables.  Candidates must be distinct
 * pairs with i < m, j < n.  For 0/1 Gram inputs the first call after a
 * table build (and a later call with more candidates) allocates,
 * stream-ordered, a buffer that groups the candidates by their endpoint of
 * larger degree (freed with the tables).  Synchronises the stream. */
mad_status mad_rescore(mad_ctx* ctx, const mad_pair* cand_dev, uint32_t ncand, uint32_t t,
                       mad_pair* out_dev, uint32_t* n_out_host, mad_stream stream);

/* ---- Fused pass (Alg. 2 then Alg. 3) ------------------------------------ *
 * mad_pipeline_plan: fixes A and B (both dense row-major, or both 0/1 CSR:
 * their device buffers and shapes), the budget s and t <= t' <= 131072,
 * and allocates every table, the hash (dense: home regions for s diamonds)
 * and the selection lists.  For 0/1 inputs it runs the step-wise build once
 * (its pilot sizes the hash; the graph sizes the T2 guides and the closure
 * filter), so the graph must not change between plan and run; only the
 * contents of the same buffers may.  It replaces any earlier tables of the
 * context.  Synchronises.  Errors as mad_build_tables; MAD_ERR_UNSUPPORTED
 * for mixed formats and for MAD_WEDGE or MAD_ALIAS contexts.
 *
 * mad_pipeline_run: one whole pass over the current contents of A and B:
 * the tables, s diamonds (indices 0 .. s-1 of `seed`), Omega_t' and the
 * exact rescore, with the same results as mad_build_tables, mad_sample,
 * mad_topk and mad_rescore.  Asynchronous and free of host synchronisation
 * and allocation, so it can be captured in a CUDA graph and replayed.
 * out_dev: t pairs (device), sorted as mad_rescore sorts them; counts_dev:
 * two uint32 (device), the number of candidates and of results; cand_dev
 * (optional, t' pairs, device): Omega_t', in no particular order.  Errors
 * found on the device (dense inputs: a compacted candidate list above 131072
 * entries, a full overflow table of the hash; 0/1 inputs: a full hash) go
 * to the device error word.  X after a
 * run (read by mad_export_x, mad_topk, mad_rescore) is the X of the step-wise
 * calls, laid out differently: for dense non-Gram inputs the home regions
 * are built whole and keys that do not fit go to an overflow table after
 * them.  The run samples all s diamonds the plan allows, so a further
 * mad_sample needs mad_reset_hash first (MAD_ERR_OVERFLOW otherwise).
 *
 * mad_pipeline_status: synchronises, refreshes the host-side table scalars
 * (mad_stats) and returns the status of the last run. */
mad_status mad_pipeline_plan(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint64_t s,
                             uint32_t tprime, uint32_t t, mad_stream stream);
mad_status mad_pipeline_run(mad_ctx* ctx, uint64_t seed, mad_pair* out_dev, uint32_t* counts_dev,
                            mad_pair* cand_dev, mad_stream stream);
mad_status mad_pipeline_status(mad_ctx* ctx, mad_stream stream);

/* Exact-computation comparator (Sec. 4.3) rebuilt for tensor cores: the t
 * pairs with the largest |a_i . b_j| by direct computation, for comparison
 * with diamond sampling.  A and B are cast to BF16 (K zero-padded to a
 * multiple of 64), C~ = A B is computed with BF16 tensor-core MMAs accumulating in FP32,
 * the `rescore` largest |c~| (0 selects 8t) are kept by a threshold filter
 * fused into the GEMM (C~ is never stored), rescored exactly in FP32 (32
 * strided fused multiply-add partial sums folded in halves), and the t
 * largest |c| are written to out_dev sorted by (|c| desc, i asc, j asc) with
 * c as the FP32 value and x = 0.  BF16 rounding can reorder near-equal
 * products, so recall against the exact top t grows with `rescore`.
 * Dense A (m x d) and B (d x n), F32 or F64, d <= 640, 1 <= t <= rescore
 * <= 65536.  The context provides scratch only (no tables needed).
 * Synchronises the stream.  MAD_ERR_UNSUPPORTED outside these limits. */
mad_status mad_dense_topt(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                          uint32_t rescore, mad_pair* out_dev, uint32_t* n_out_host,
                          mad_stream stream);

/* Exact comparator for 0/1 inputs (Sec. 4.3, the exact computation for
 * comparison: C formed one sparse row at a time, its top entries kept).
 * A (m x d) and B (d x n) are 0/1 CSR (MAD_BINARY; B = A^T for MAD_GRAM
 * contexts, where pairs are unordered, j >= i; MAD_EXCLUDE_DIAG drops
 * i == j).  Returns the min(t, #stored) largest c_ij = |{k : a_ik = b_kj =
 * 1}| among the stored entries of C (c_ij >= 1), sorted by (c desc, i asc,
 * j asc), with c as an exact integer in the double and x = 0: the same
 * pairs and counts as a full sparse product for any input.
 * Because c_ij <= min(nnz(a_i*), nnz(b_*j)), a pilot product of the ~2048
 * rows and columns of largest degree gives a lower bound theta on the t-th
 * largest count, and the main pass covers only rows and columns with at
 * least theta entries, keeping counts >= theta (MAD_SPARSE_NO_BOUND: every
 * row and column, the threshold filtering entries only).  Counts are
 * accumulated in shared memory, one block per row of C.  t <= 524288.
 * Uses the context's scratch (about 40 bytes per row and column plus 4 per
 * entry of B, and 75 MB of candidate lists); the context needs no tables.
 * Synchronises the stream.  MAD_ERR_UNSUPPORTED for other formats, and
 * for inputs whose t-th count ties beyond the candidate list with counts
 * of 65535 or more. */
#define MAD_SPARSE_NO_BOUND 1u
mad_status mad_sparse_topt(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                           uint32_t options, mad_pair* out_dev, uint32_t* n_out_host,
                           mad_stream stream);

/* ---- Batched queries (maximum |inner product| search) ----------------- *
 * Many small instances against one item matrix: query q is the instance
 * A = Q[q] (1 x d) with B = the items (d x n), sampled with its own budget
 * s_q and seed + q.  Because m = 1, the stage-1 draw of Alg. 2 always gives
 * the query's row, so diamond l of query q draws only k, j and k' (Philox
 * key seed + q, counter l, as in mad_sample); its x accumulates in a hash
 * region of its own, and Alg. 3 runs per query: the t' largest positive x
 * by (x desc, j asc), their exact c = q . b_j (FP64, rescoring order of
 * mad_rescore), the t largest |c| by (|c| desc, j asc).  Each query's result
 * equals mad_build_tables + mad_sample + mad_topk + mad_rescore on that
 * query alone with the same s_max.
 *
 * mad_mips_items: item-side tables (TB with per-row guides, row norms, the
 * items transposed for rescoring) for dense B (d x n, F32, n < 2^31).  B
 * must stay alive and unchanged while the context uses it.  s_max bounds
 * every query budget (it fixes the fixed-point scale F).  Synchronises.
 *
 * mad_mips_plan: the batch shape: nq queries with budgets s_host[q] (host,
 * 1 <= s_q <= s_max), t' (1..1024) and t (1..t').  Allocates the batch's
 * device buffers and uploads the per-query layout.  Synchronises.
 *
 * mad_mips_run: one batch on Q (nq x d dense F32, device), asynchronous
 * and free of host synchronisation and allocation, so it can be captured
 * in a CUDA graph.  out_dev: nq * t pairs (query q's results at q * t, i =
 * q); n_out_dev: nq counts (uint32, device); cand_dev (optional, nq * t'
 * pairs): each query's top-t' candidates.  A query whose candidates above
 * the selection threshold exceed 4096 (ties of x in the thousands) reports
 * MAD_ERR_STATE through the device error word (read by mad_stats). */
mad_status mad_mips_items(mad_ctx* ctx, const mad_matrix* B, uint64_t s_max, mad_stream stream);
/* mad_mips_config (the paper has no counterpart; used by the package's
 * autotuner, paper_1506_03872_gb300/autotune.py): the launch shape of the
 * next mad_mips_plan and mad_mips_run.  region_lg: each query's region is
 * the power of two >= 2^region_lg s_q slots (1..4; 0: 1); chunk_mult: 256
 * x chunk_mult diamonds per chunk (1, 2, 4, 8; 0: 1); blocks_per_sm:
 * sampler blocks per SM (0: as many as fit, at most 8); select_threads:
 * threads of each query's selection (128, 256, 512; 0: 256).  None of
 * these changes a result (the keys and sums of X, Omega_t' and Omega_t are
 * the same): only the time.  MAD_ERR_ARG outside these values. */
mad_status mad_mips_config(mad_ctx* ctx, uint32_t region_lg, uint32_t chunk_mult,
                           uint32_t blocks_per_sm, uint32_t select_threads);
mad_status mad_mips_plan(mad_ctx* ctx, uint32_t nq, const uint64_t* s_host, uint32_t tprime,
                         uint32_t t, mad_stream stream);
mad_status mad_mips_run(mad_ctx* ctx, const mad_matrix* Q, uint64_t seed, mad_pair* out_dev,
                        uint32_t* n_out_dev, mad_pair* cand_dev, mad_stream stream);

/* ---- Learned budget predictor (the paper has no counterpart) ----------- *
 * Theorem 2 bounds the diamonds needed to separate the top entries by a
 * multiple of ||W||_1 / tau^2; the predictor learns the budget from cheap
 * statistics of an instance instead of the unknown tau.
 *
 * mad_budget_features: MAD_BUDGET_FEATURES statistics of the instance of the
 * last mad_build_tables, written to features_host (host): log10 of m, n, d,
 * nnz(A), nnz(B); 1 for 0/1 inputs else 0; log10 ||W||_1; log10 of the
 * largest row 2-norm of A and column 2-norm of B; log10 of sum r_i^2 /
 * (sum r_i)^2 and of max r_i / sum r_i for the row weights r_i of T1; and
 * log10 ||W||_1 - 2 (the two largest-norm logs), a Cauchy-Schwarz stand-in
 * for Theorem 2's ||W||_1 / tau^2.  Synchronises.
 *
 * mad_mlp_train / mad_mlp_predict: a perceptron f -> 64 -> 64 -> 1 (ReLU)
 * with BF16 weights (FP32 master copies for training) and FP32 arithmetic.
 * params_dev (device, MAD_MLP_PARAMS(f) floats, caller-initialised): W1
 * (64 x f, row-major), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3.
 * Training: `epochs` full-batch Adam steps (beta 0.9 / 0.999) on the pinball
 * loss of level `quantile` (0 < quantile < 1; above 0.5 a prediction below
 * the target costs more than one above it) over X_dev (n x f, row-major) and
 * y_dev (n); loss_dev (optional, `epochs` floats) receives the loss before
 * each step.  n <= 4096, f <= 32.  Uses the context's scratch.
 * Prediction: y_dev[i] = network(X_dev row i).  Both are asynchronous. */
#define MAD_BUDGET_FEATURES 12
#define MAD_MLP_HIDDEN 64
#define MAD_MLP_PARAMS(f) (MAD_MLP_HIDDEN * (f) + 3 * MAD_MLP_HIDDEN + MAD_MLP_HIDDEN * MAD_MLP_HIDDEN + 1)
mad_status mad_budget_features(mad_ctx* ctx, float* features_host, mad_stream stream);
mad_status mad_mlp_train(mad_ctx* ctx, float* params_dev, const float* X_dev, const float* y_dev,
                         uint32_t n, uint32_t f, uint32_t epochs, float lr, float quantile,
                         float* loss_dev, mad_stream stream);
mad_status mad_mlp_predict(const float* params_dev, const float* X_dev, uint32_t n, uint32_t f,
                           float* y_dev, mad_stream stream);

/* Diagnostics for mad_dense_topt: the full BF16 tensor-core product C~ as
 * FP32, row-major m x n, written to c_dev (device, m*n floats). */
mad_status mad_debug_dense_product(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B,
                                   float* c_dev, mad_stream stream);

/* Rescoring and top-t without any device allocation.
 *
 * The paper has no counterpart to this entry point.  It returns exactly what
 * mad_rescore returns (same pairs, same bits) for callers that cannot
 * allocate device memory: applications whose GPU memory is reserved up
 * front by another allocator (serving stacks, host frameworks), and loops
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * It needs no context: A and B are the matrices the candidates index (the
 * formats of mad_build_tables; dense B is read in place), and the caller
 * owns every buffer passed in.
 *
 * Limit: ncand <= MAD_NOALLOC_MAX_CANDIDATES; larger requests return
 * MAD_ERR_UNSUPPORTED.  The working memory is one fixed static device array
 * (about 1.8 MB) that each GPU loading the library keeps until the process
 * exits.  The first call on a device looks up that array's device address
 * and keeps it (set-up once per device; make that first call before any
 * stream capture on the device; a device reset after it is not supported).
 * All calls share the array and each clears what must start at zero, so
 * calls that overlap on the GPU (other streams or host threads) race:
 * serialise them.  A candidate outside A or B returns MAD_ERR_ARG, and the
 * next call starts from a cleared status.  Every call copies its status
 * word to the host and synchronises the stream. */
#define MAD_NOALLOC_MAX_CANDIDATES 16384u
mad_status mad_rescore_noalloc(const mad_matrix* A, const mad_matrix* B, const mad_pair* cand_dev,
                               uint32_t ncand, uint32_t t, mad_pair* out_dev,
                               uint32_t* n_out_host, mad_stream stream);

/* ---- Memory-system probes (the paper has no counterpart) --------------- *
 * The sampler's diamonds end in random 32-byte sectors of its tables and,
 * for 0/1 inputs, random 64-bit atomics on its hash; these kernels measure
 * those two rates on buffers of the caller's choosing (sized like the
 * tables and the hash), so the sampler's throughput can be stated against
 * them.  Both are asynchronous on `stream`; time them with events.
 *
 * mad_probe_gather: `count` 4-byte loads, each from a uniformly random
 * 32-byte sector of table_dev (device, `bytes` a multiple of 32, 32-byte
 * aligned), positions from a SplitMix64 hash of `seed` and the load index.
 * sink_dev: 8 bytes of device memory the kernel may write (keeps the loads).
 *
 * mad_probe_atomics: `count` 64-bit atomics on uniformly random words of
 * table_dev (device, `bytes` a multiple of 8, 8-byte aligned): mode 0 adds
 * 1 (a reduction, no value returned), mode 1 compare-and-swaps against 0
 * and uses the old value (a round trip, as a hash insert's key claim).
 * The table's contents change.  MAD_ERR_ARG for bad sizes or modes. */
mad_status mad_probe_gather(const void* table_dev, uint64_t bytes, uint64_t count, uint64_t seed,
                            void* sink_dev, mad_stream stream);
mad_status mad_probe_atomics(void* table_dev, uint64_t bytes, uint64_t count, uint32_t mode,
                             uint64_t seed, void* sink_dev, mad_stream stream);

/* ---- Sharded runs (one rank per GPU) ----------------------------------- *
 * Diamonds are independent and counter-indexed (Alg. 2 with the Philox
 * counter of the diamond index), so a run of s diamonds splits into
 * contiguous diamond ranges, one per rank (mad_sample with first_diamond),
 * over replicated tables.  X is an exact integer sum, so the partial X of
 * the ranges summed by key equal the X of one run; each key is summed by
 * one owner rank, owners select their top t' (mad_topk), and the union of
 * the owners' candidates holds the global Omega_t' (Alg. 3).  These entry
 * points are the compute steps of that exchange; the collectives belong to
 * the caller (paper_1506_03872_gb300/shard.py uses torch.distributed).
 *
 * mad_export_x_by_owner: X's occupied keys and values grouped by owner
 * rank, owner = a SplitMix64 mix of the key modulo `world` (1..65536):
 * owner o's entries are keys_dev/vals_dev[offsets_host[o] .. offsets_host
 * [o + 1]) (device arrays of cap entries; offsets_host: world + 1 host
 * entries).  When the total offsets_host[world] exceeds cap nothing is
 * written (call again with a larger buffer).  Synchronises.
 *
 * mad_accumulate: adds n (key, value) pairs (device arrays) to X, as
 * sampling adds diamonds: X of the keys this rank owns, merged from every
 * rank's partials after mad_reset_hash.  Keys must belong to the
 * context's shape (row < m, column < n, unordered under MAD_GRAM); the
 * hash must hold them (MAD_ERR_HASH_FULL from the next mad_topk otherwise).
 * Asynchronous.
 *
 * mad_select_pairs: the min(K, #{x > 0}) pairs of pairs_dev (n, device)
 * with the largest x, ties broken by smaller (i, j), sorted by (x desc, i
 * asc, j asc) and copied whole to out_dev (K pairs, device): the global
 * Omega_t' from the gathered candidates.  Synchronises. */
mad_status mad_export_x_by_owner(mad_ctx* ctx, uint32_t world, uint64_t* keys_dev,
                                 int64_t* vals_dev, uint64_t cap, uint64_t* offsets_host,
                                 mad_stream stream);
mad_status mad_accumulate(mad_ctx* ctx, const uint64_t* keys_dev, const int64_t* vals_dev,
                          uint64_t n, mad_stream stream);
mad_status mad_select_pairs(mad_ctx* ctx, const mad_pair* pairs_dev, uint64_t n, uint32_t K,
                            mad_pair* out_dev, uint32_t* n_out_host, mad_stream stream);

/* Counters and table scalars (synchronises the device). *//* Counters and table scalars (synchronises the device). */
mad_status mad_stats(mad_ctx* ctx, mad_stats_t* out);

/* ---- Diagnostics (used by the parity tests; not on the hot path) ------- */

/* The draws of diamonds first .. first+count-1 without accumulating: the
 * indices (i, k, j, k') and the increment v (Alg. 2 loop body).  Output
 * arrays are device arrays of count elements. */
mad_status mad_debug_draws(mad_ctx* ctx, uint64_t seed, uint64_t first, uint64_t count,
                           uint32_t* i_dev, uint32_t* k_dev, uint32_t* j_dev, uint32_t* kp_dev,
                           int64_t* v_dev, mad_stream stream);

/* Layout of the dense hash X for the next mad_build_tables or
 * mad_pipeline_plan, for tests of its rarely taken paths.  region_factor:
 * row i's home region is the smallest power of two >= region_factor x its
 * expected diamonds (at least 4 slots); 0 < region_factor <= 1.5, default
 * 1.5.  overflow_slots: slots of the overflow table after the regions (a
 * power of two >= 16), or 0 for the default max(2^14, s_max / 64) rounded
 * up to a power of two.  Regions too small for their keys send them to the
 * overflow table in the fused pass (mad_pipeline_run); a full overflow
 * table is reported as MAD_ERR_HASH_FULL by mad_pipeline_status.  The
 * step-wise mad_sample probes the regions as one table and reports
 * MAD_ERR_HASH_FULL past its probe limit.  MAD_ERR_ARG outside these
 * ranges. */
mad_status mad_debug_set_hash_layout(mad_ctx* ctx, float region_factor, uint64_t overflow_slots);

/* As mad_debug_draws for an arbitrary device list of diamond indices. */
mad_status mad_debug_draws_list(mad_ctx* ctx, uint64_t seed, const uint64_t* ells_dev,
                                uint64_t count, uint32_t* i_dev, uint32_t* k_dev,
                                uint32_t* j_dev, uint32_t* kp_dev, int64_t* v_dev,
                                mad_stream stream);

/* Every occupied key of X and its value (order unspecified).  keys_dev and
 * vals_dev hold cap entries; *n_host receives |X| (the copy stops at cap).
 * Synchronises the stream. */
mad_status mad_export_x(mad_ctx* ctx, uint64_t* keys_dev, int64_t* vals_dev, uint64_t cap,
                        uint64_t* n_host, mad_stream stream);

/* Copy an internal table to out_dev (device, cap elements):
 *   0 T1 (uint64, m)      1 T2 (uint32, nnz(A))   2 TA (uint32, nnz(A))
 *   3 TB (uint32, nnz(B)) 4 ||a_i*||_1 (f32, m)  5 ||b_k*||_1 (f32, d)
 *   6 r_i (f32, m)
 *   wedge contexts: 7 TK (uint64, d, inclusive prefix of the centre
 *   weights), 8 column tables of A (uint32, m x d column-major; dense
 *   non-Gram inputs), 9 ||a_*k||_1 (f32, d; dense inputs)
 *   alias contexts (MAD_ALIAS): 10 + 3 f + part for the families f = 0 T1
 *   (1 row of m), 1 T2 and 2 TA (m rows of d), 3 TB (d rows of n); part 0
 *   the entries (16 bytes: uint64 threshold, uint32 alias, uint32 0; per
 *   row its segments' entries then its nseg top-level entries), 1 the
 *   segment totals (uint64, rows x nseg), 2 the row totals (uint64, rows)
 * Row-table entries carry the sign of the matching value of A or B in bit
 * 31 (float mode).  Tables the mode keeps implicit report 0 elements.
 * *n_host receives the element count.  Synchronises the stream. */
mad_status mad_export_table(mad_ctx* ctx, int which, void* out_dev, uint64_t cap,
                            uint64_t* n_host, mad_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* MAD_H_ */
