// The fused pass of Alg. 2 and Alg. 3: tables, sampling, Omega_t' from X,
// exact rescoring and Omega_t, enqueued by the host without waiting for the
// device.  Dense inputs, and 0/1 CSR inputs: for these the plan runs the
// step-wise table build once, which fixes the sizes that follow from the
// graph (the T2 guides, the closure filter) and the hash capacity (from its
// pilot); a run then rebuilds every table of the same graph on the device
// and samples with the run's seed (the graph must not change between plan
// and run).  Every size is fixed when the pass is planned (by
// m, d, n, s, t' and t); every quantity that depends on the data (T1's
// total, the increment exponent F, the extent of the hash, the list
// lengths of the selections) is read by the kernels from device memory.  A
// run allocates nothing and never synchronises, so a caller can capture it
// in a CUDA graph once and replay it on new contents of the same inputs.
//
// Results are those of the step-wise calls (mad_build_tables, mad_sample
// with first diamond 0, mad_topk, mad_rescore) on the same inputs, seed and
// budgets, bit for bit: the kernels are the same and only where the lengths
// come from differs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "mad_internal.cuh"

using namespace mad;

namespace {

// The pass's own buffers, carved in this order from one allocation.
struct PipeBufs {
  void* state;                  // selection state of Omega_t'
  unsigned long long* count;    // compacted candidates (device length)
  Item* list;                   // compacted items, list_cap
  Item* l1;                     // ping-pong lists of the long selection (0/1
  Item* l2;                     //   inputs), list_cap each
  Item* topk;                   // the K selected, unsorted (0/1 inputs), t'
  Item* sorted;                 // tile-sorted copy, kDevSelectCap
  uint32_t* pos;                // their input positions, kDevSelectCap
  Item* top;                    // Omega_t', t'
  mad_pair* cand;               // Omega_t' as pairs, t'
  Item* rs_items;               // rescored candidates, t'
  Item* rs_sorted;              // tile-sorted copy, t'
  uint32_t* rs_pos;             // t'
  Item* rs_out;                 // Omega_t, t
  double* cvals;                // exact c of each candidate, t'
  size_t bytes;
};

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// long_sel: the 0/1 pass's radix selection over list_cap candidates.
PipeBufs carve(void* base, uint64_t tprime, uint64_t t, uint64_t list_cap, bool long_sel) {
  PipeBufs b;
  char* p = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += up256(bytes);
    return (void*)q;
  };
  b.state = take(dev_select_state_bytes());
  b.count = (unsigned long long*)take(4 * sizeof(unsigned long long));
  b.list = (Item*)take(list_cap * sizeof(Item));
  b.l1 = (Item*)take(long_sel ? list_cap * sizeof(Item) : 0);
  b.l2 = (Item*)take(long_sel ? list_cap * sizeof(Item) : 0);
  b.topk = (Item*)take(long_sel ? tprime * sizeof(Item) : 0);
  b.sorted = (Item*)take(kDevSelectCap * sizeof(Item));
  b.pos = (uint32_t*)take(kDevSelectCap * sizeof(uint32_t));
  b.top = (Item*)take(tprime * sizeof(Item));
  b.cand = (mad_pair*)take(tprime * sizeof(mad_pair));
  b.rs_items = (Item*)take(tprime * sizeof(Item));
  b.rs_sorted = (Item*)take(tprime * sizeof(Item));
  b.rs_pos = (uint32_t*)take(tprime * sizeof(uint32_t));
  b.rs_out = (Item*)take(t * sizeof(Item));
  b.cvals = (double*)take(tprime * sizeof(double));
  b.bytes = off;
  return b;
}

// The 0/1 tables, guides, closure filter and an empty X, on the device.
mad_status enqueue_csr_build(mad_ctx* ctx, cudaStream_t st) {
  cudaMemsetAsync(ctx->sc, 0, sizeof(DevScalars), st);
  mad_status rs;
  if ((rs = build_tables_impl(ctx, st)) != MAD_OK) return rs;
  if ((rs = t2_guide_offsets(ctx, st)) != MAD_OK) return rs;
  if (ctx->t2g_total && (rs = t2_guide_fill(ctx, st)) != MAD_OK) return rs;
  if ((rs = build_bloom(ctx, st)) != MAD_OK) return rs;
  if ((rs = t1_guide_fill(ctx, st)) != MAD_OK) return rs;
  return clear_x(ctx, st);
}

// Scratch of a 0/1 run: T1's chunk totals, then the T2 guide sizes and
// their scan.
size_t csr_build_scratch_bytes(const mad_ctx* ctx) {
  const uint64_t m = (uint64_t)ctx->m;
  const size_t chunks = (size_t)((m + 2047) / 2048) * sizeof(unsigned long long);
  const size_t guides = ((m * sizeof(unsigned long long) + 255) & ~(size_t)255) +
                        scan_partial_elems(m) * 8;
  return chunks > guides ? chunks : guides;
}

mad_status enqueue_pass(mad_ctx* ctx, uint64_t seed, mad_pair* out_dev, uint32_t* counts_dev,
                        mad_pair* cand_dev, cudaStream_t st) {
  const bool long_sel = !ctx->dense;
  const PipeBufs b =
      carve(ctx->pipe_buf, ctx->pipe_tprime, ctx->pipe_t, ctx->pipe_list_cap, long_sel);
  mad_pair* cand = cand_dev ? cand_dev : b.cand;
  mad_status rs;
  // Alg. 2: tables, an empty X, s diamonds.  Where the sampler builds the
  // home regions whole, nothing needs clearing first.
  const bool fresh = ctx->dense && x_builder_applies(ctx, ctx->pipe_s);
  if (!ctx->dense) {
    if ((rs = enqueue_csr_build(ctx, st)) != MAD_OK) return rs;
  } else if ((rs = enqueue_dense_build(ctx, st, !fresh)) != MAD_OK) {
    return rs;
  }
  ctx->sampled = 0;
  if ((rs = sample_impl(ctx, ctx->pipe_s, seed, 0, st, true)) != MAD_OK) return rs;
  ctx->sampled = ctx->pipe_s;
  ctx->built = true;
  // Alg. 3: Omega_t' (its length min(t', compacted) on the device) ...
  if (long_sel)
    select_hash_dev_long(ctx, ctx->pipe_tprime, hash_extent(ctx), b.state, b.count, b.list, b.l1,
                         b.l2, ctx->pipe_list_cap, b.topk, b.sorted, b.pos, b.top, st);
  else
    select_hash_dev(ctx, ctx->pipe_tprime, hash_extent(ctx), b.state, b.count, b.list, b.sorted,
                  b.pos, b.top, st);
  items_to_pairs_dev(ctx, b.top, ctx->pipe_tprime, b.count, nullptr, nullptr, cand, counts_dev, st);
  // ... the exact c of each candidate, and Omega_t.
  if ((rs = rescore_items(ctx, cand, ctx->pipe_tprime, b.rs_items, b.cvals, st, b.count)) != MAD_OK)
    return rs;
  block_select_dev(ctx, b.rs_items, ctx->pipe_tprime, ctx->pipe_t, b.count, true, b.rs_sorted,
                   b.rs_pos, b.rs_out, (unsigned int*)(b.count + 3), nullptr, st);
  items_to_pairs_dev(ctx, b.rs_out, ctx->pipe_t, b.count, cand, b.cvals, out_dev, counts_dev + 1,
                     st);
  return cuda_status(cudaGetLastError());
}

}  // namespace

extern "C" {

mad_status mad_pipeline_plan(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint64_t s,
                             uint32_t tprime, uint32_t t, mad_stream stream) {
  if (!ctx || !A || !B) return MAD_ERR_ARG;
  if (t == 0 || tprime < t || (uint64_t)tprime > kDevSelectCap) return MAD_ERR_ARG;
  const bool csr = A->fmt == MAD_CSR && B->fmt == MAD_CSR;
  if (!csr && (A->fmt != MAD_DENSE_ROWMAJOR || B->fmt != MAD_DENSE_ROWMAJOR))
    return MAD_ERR_UNSUPPORTED;
  if (ctx->flags & (MAD_WEDGE | MAD_ALIAS)) return MAD_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  // 0/1 inputs: the step-wise build, once, sizes the guides, the filter
  // and the hash (its pilot); dense inputs: the sizes from the shapes.
  mad_status rs = csr ? mad_build_tables(ctx, A, B, s, stream) : plan_dense_tables(ctx, A, B, s, st);
  if (rs != MAD_OK) return rs;
  // Candidate lists: the 0/1 counts tie in large numbers at the t'-th x (on
  // the Chung-Lu graph of 1e6 nodes nearly every key of X has x = 1), so the
  // 0/1 list holds every slot of the hash: it cannot overflow.
  ctx->pipe_list_cap = csr ? std::max<uint64_t>(kDevSelectCap, ctx->hcap_alloc) : kDevSelectCap;
  const PipeBufs sizes = carve(nullptr, tprime, t, ctx->pipe_list_cap, csr);
  if ((rs = pool_malloc(ctx, &ctx->pipe_buf, sizes.bytes, st)) != MAD_OK) return rs;
  // The scratch every launch of a run needs, owned by the pass.
  size_t scratch = csr ? csr_build_scratch_bytes(ctx) : dense_build_scratch_bytes(ctx);
  if (sample_scratch_bytes(ctx, s) > scratch) scratch = sample_scratch_bytes(ctx, s);
  if ((rs = pool_malloc(ctx, &ctx->pipe_scratch, scratch, st)) != MAD_OK) return rs;
  ctx->pipe_scratch_bytes = scratch;
  // The rescoring's grouping buffer (0/1 Gram inputs) for t' candidates.
  if ((rs = rescore_reserve(ctx, tprime, st)) != MAD_OK) return rs;
  ctx->pipe = true;
  ctx->pipe_s = s;
  ctx->pipe_tprime = tprime;
  ctx->pipe_t = t;
  return cuda_status(cudaStreamSynchronize(st));
}

mad_status mad_pipeline_run(mad_ctx* ctx, uint64_t seed, mad_pair* out_dev, uint32_t* counts_dev,
                            mad_pair* cand_dev, mad_stream stream) {
  if (!ctx || !out_dev || !counts_dev) return MAD_ERR_ARG;
  if (!ctx->pipe) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  // The pass's scratch stands in for the context's while the run is
  // enqueued (sized by the plan, so nothing is allocated).
  void* const shared_scratch = ctx->scratch;
  const size_t shared_bytes = ctx->scratch_bytes;
  ctx->scratch = ctx->pipe_scratch;
  ctx->scratch_bytes = ctx->pipe_scratch_bytes;
  ctx->scratch_fixed = true;
  const mad_status rs = enqueue_pass(ctx, seed, out_dev, counts_dev, cand_dev, st);
  ctx->scratch_fixed = false;
  ctx->scratch = shared_scratch;
  ctx->scratch_bytes = shared_bytes;
  return rs;
}

mad_status mad_pipeline_status(mad_ctx* ctx, mad_stream stream) {
  if (!ctx) return MAD_ERR_ARG;
  if (!ctx->pipe) return MAD_ERR_STATE;
  cudaStream_t st = (cudaStream_t)stream;
  if (!ctx->dense) {
    DevScalars hs;
    const mad_status rs = read_device_scalars(ctx, &hs, st);
    if (rs != MAD_OK) return rs;
    if (hs.err & DERR_OVERFLOW) return MAD_ERR_OVERFLOW;
    if (hs.t1_total == 0) return MAD_ERR_EMPTY;
    ctx->t1_total = hs.t1_total;
    return device_error_status(ctx->device_error);
  }
  const mad_status rs = finish_dense_build(ctx, st);
  if (rs != MAD_OK) return rs;
  return device_error_status(ctx->device_error);
}

}  // extern "C"
