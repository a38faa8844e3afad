// mad_rescore_noalloc: the exact-rescore-and-top-t step (the same result as
// mad_rescore) for callers that must not allocate device memory.
//
// Who needs it: host applications whose device memory is owned by another
// allocator that reserves the whole GPU up front (serving stacks, embedding
// frameworks), and latency-critical loops in which cudaMalloc/cudaFree would
// stall the device with their implicit synchronisation.  Such callers own A,
// B, the candidates and the output; this entry point allocates nothing.
//
// Its working memory is one file-scope __device__ array of fixed size
// (kScratchBytes, about 1.8 MB) that every GPU loading the library holds
// until the process exits.  The host learns the array's device address once
// per device with cudaGetSymbolAddress (the host-side symbol is only a
// stand-in, never a device address).  All calls share the array: the parts
// that must start at zero are cleared by each call, and calls that overlap
// on the GPU race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <mutex>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr uint32_t kMaxCandidates = 16384;
constexpr size_t kScratchBytes =
    4ull * kMaxCandidates * sizeof(Item) + kMaxCandidates * sizeof(double) + (64u << 10);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the static array on the current device (set up on the
// first call per device and kept: the address stays valid for the life of
// the CUDA context, so a device reset after the first call is not
// supported).
mad_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return MAD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return e != cudaSuccess ? cuda_status(e) : MAD_ERR_CUDA;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return MAD_OK;
}

__device__ __forceinline__ double as_f64(float v) { return (double)v; }
__device__ __forceinline__ double as_f64(double v) { return v; }

__device__ __forceinline__ void bad_candidate(uint32_t i, uint32_t j, unsigned long long q,
                                              double* cvals, Item* items, DevScalars* sc) {
  atomicOr(&sc->err, DERR_SEARCH);
  cvals[q] = 0.0;
  Item it;
  it.p = 0;
  it.key = ((unsigned long long)i << 32) | j;
  it.aux = q;
  items[q] = it;
}

// Dense: reads column j of B in place (stride ldb).  Lane L sums k = L mod 32
// in ascending order with fused multiply-add, then the partials fold in
// halves: the same order, hence the same bits, as mad_rescore.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_rescore_dense_inplace(const mad_pair* __restrict__ cand, unsigned long long ncand,
                        const TA* __restrict__ A, int64_t lda, const TB* __restrict__ B,
                        int64_t ldb, int64_t d, int64_t m, int64_t n,
                        double* __restrict__ cvals, Item* __restrict__ items, DevScalars* sc) {
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < ncand; q += warps) {
    const uint32_t i = cand[q].i, j = cand[q].j;
    if (i >= m || j >= n) {
      if (lane == 0) bad_candidate(i, j, q, cvals, items, sc);
      continue;
    }
    const TA* __restrict__ a = A + (int64_t)i * lda;
    double acc = 0.0;
    for (int64_t k = lane; k < d; k += 32) acc = __fma_rn(as_f64(a[k]), as_f64(B[k * ldb + j]), acc);
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

// 0/1 CSR: c_ij = number of k in row i of A with b_kj = 1, counted exactly.
__global__ void __launch_bounds__(256)
k_rescore_binary_inplace(const mad_pair* __restrict__ cand, unsigned long long ncand,
                         const int64_t* __restrict__ a_ptr, const int32_t* __restrict__ a_col,
                         const int64_t* __restrict__ b_ptr, const int32_t* __restrict__ b_col,
                         int64_t m, int64_t n, double* __restrict__ cvals,
                         Item* __restrict__ items, DevScalars* sc) {
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < ncand; q += warps) {
    const uint32_t i = cand[q].i, j = cand[q].j;
    if (i >= m || j >= n) {
      if (lane == 0) bad_candidate(i, j, q, cvals, items, sc);
      continue;
    }
    long long count = 0;
    for (int64_t e = a_ptr[i] + lane; e < a_ptr[i + 1]; e += 32) {
      const int32_t k = a_col[e];
      if (contains_sorted(b_col + b_ptr[k], b_ptr[k + 1] - b_ptr[k], (int32_t)j)) ++count;
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

template <typename TA, typename TB>
void launch_inplace(const mad_matrix* A, const mad_matrix* B, const mad_pair* cand, uint64_t ncand,
                    double* cvals, Item* items, DevScalars* sc, cudaStream_t st) {
  const unsigned long long blocks = (ncand * 32 + 255) / 256;
  k_rescore_dense_inplace<TA, TB><<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
      cand, ncand, (const TA*)A->values, A->ld, (const TB*)B->values, B->ld, A->cols, A->rows,
      B->cols, cvals, items, sc);
}

bool dense_ok(const mad_matrix* M) {
  return M->fmt == MAD_DENSE_ROWMAJOR && (M->dt == MAD_F32 || M->dt == MAD_F64) && M->values &&
         M->ld >= M->cols && M->rows > 0 && M->cols > 0;
}

bool csr_ok(const mad_matrix* M) {
  return M->fmt == MAD_CSR && M->dt == MAD_BINARY && M->rowptr && M->colidx && M->rows > 0 &&
         M->cols > 0;
}

}  // namespace
}  // namespace mad

using namespace mad;

extern "C" mad_status mad_rescore_noalloc(const mad_matrix* A, const mad_matrix* B,
                                          const mad_pair* cand_dev, uint32_t ncand, uint32_t t,
                                          mad_pair* out_dev, uint32_t* n_out_host,
                                          mad_stream stream) {
  if (!A || !B || !n_out_host || (ncand > 0 && !cand_dev) || (t > 0 && !out_dev))
    return MAD_ERR_ARG;
  *n_out_host = 0;
  if (B->rows != A->cols) return MAD_ERR_ARG;
  const bool dense = dense_ok(A) && dense_ok(B);
  const bool csr = csr_ok(A) && csr_ok(B);
  if (!dense && !csr) return MAD_ERR_UNSUPPORTED;
  if (ncand > kMaxCandidates) return MAD_ERR_UNSUPPORTED;  // beyond the fixed array
  if (ncand == 0 || t == 0) return MAD_OK;
  cudaStream_t st = (cudaStream_t)stream;

  void* base = nullptr;
  mad_status rs = scratch_address(&base);
  if (rs != MAD_OK) return rs;
  const size_t ws_bytes = (select_ws_bytes(ncand, t) + 255) & ~(size_t)255;
  const size_t cv_bytes = ((size_t)ncand * sizeof(double) + 255) & ~(size_t)255;
  if (ws_bytes + cv_bytes + sizeof(DevScalars) > kScratchBytes) return MAD_ERR_UNSUPPORTED;
  const SelectWs ws = select_ws_carve(base, ncand, t);
  double* cvals = (double*)((char*)base + ws_bytes);
  DevScalars* sc = (DevScalars*)((char*)base + ws_bytes + cv_bytes);
  // The array keeps the previous call's contents: reset the error word.
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
  if (e != cudaSuccess) return cuda_status(e);

  if (csr) {
    const unsigned long long blocks = ((unsigned long long)ncand * 32 + 255) / 256;
    k_rescore_binary_inplace<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(
        cand_dev, ncand, A->rowptr, A->colidx, B->rowptr, B->colidx, A->rows, B->cols, cvals,
        ws.l0, sc);
  } else {
    const bool a64 = A->dt == MAD_F64, b64 = B->dt == MAD_F64;
    if (a64 && b64) launch_inplace<double, double>(A, B, cand_dev, ncand, cvals, ws.l0, sc, st);
    else if (a64) launch_inplace<double, float>(A, B, cand_dev, ncand, cvals, ws.l0, sc, st);
    else if (b64) launch_inplace<float, double>(A, B, cand_dev, ncand, cvals, ws.l0, sc, st);
    else launch_inplace<float, float>(A, B, cand_dev, ncand, cvals, ws.l0, sc, st);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e);

  // The select and pair-writing helpers only count launches on the context
  // they are given; a host-side context object owns no device memory.
  mad_ctx bookkeeping;
  uint64_t nsel = 0;
  if ((rs = select_list(&bookkeeping, ws, ncand, t, 8, &nsel, st)) != MAD_OK) return rs;
  if ((rs = items_to_pairs(&bookkeeping, ws.out, nsel, cand_dev, cvals, out_dev, st)) != MAD_OK)
    return rs;
  uint32_t err = 0;
  e = cudaMemcpyAsync(&err, &sc->err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  if (err & DERR_SEARCH) return MAD_ERR_ARG;  // a candidate lies outside A or B
  if (err) return MAD_ERR_STATE;
  *n_out_host = (uint32_t)nsel;
  return MAD_OK;
}
