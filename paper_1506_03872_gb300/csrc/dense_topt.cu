// Exact-computation comparator of Sec. 4.3, rebuilt for GB300 tensor cores:
// the top t of |A B| for dense A (m x d) and B (d x n).
//
// The paper streams dgemm column blocks through a priority queue.  Here:
//  1. A and B^T are cast to BF16, K padded with zeros to a multiple of 64.
//  2. One persistent kernel per SM computes C~ = A B tile by tile with
//     tcgen05.mma (BF16 in, FP32 accumulate in TMEM), operands brought into
//     shared memory by TMA (128-byte swizzle), and never writes C~: its
//     epilogue keeps only entries with |c~| >= theta in a per-CTA buffer.
//     theta starts from a pre-pass (the same kernel over every 16th tile,
//     recording row-segment maxima, whose K_keep-th largest bounds the global
//     K_keep-th largest from below) and rises whenever the buffer is
//     compacted to its K_keep largest entries (the rescore budget, 8t by
//     default; the buffer lives in global memory and holds 4 K_keep
//     entries, at least 4096) (a tile that overflows the buffer is
//     rescanned from TMEM above the new theta); CTAs share theta
//     through an atomicMax, so every kept threshold is a lower bound of the
//     global K_keep-th largest |c~| and no entry of the global top K_keep is
//     ever dropped.
//  3. The K_keep largest |c~| of the merged buffers are rescored exactly in FP32
//     and the t largest |c| returned.
// Warp roles per CTA (352 threads with the default 8 epilogue warps): warp 0 takes work units from a global
// counter (runs of column tiles of one row block, so CTAs whose tiles hold
// many candidates take fewer) and issues TMA; warps 1 and 10 issue the MMAs
// of the even and odd tiles into their own TMEM accumulator (warp 1 also
// allocates the 2 x 256 TMEM columns); warps 2-9 drain the accumulators
// (warp w reads TMEM lane quarter w mod 4 and one half of the columns) and
// release a tile's accumulator as soon as none of their values passes the
// threshold.  The A panel (128 rows x K) of a unit stays in shared memory;
// B arrives one 256-column tile per stage for K <= 128 (3 stages), else one
// 64-wide K slice per stage (32 KB; 3 stages for K = 512, 2 for K = 640).
// Every wait is bounded by a clock limit after which the CTA sets an error
// flag and winds down.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "mad_device.cuh"
#include "mad_internal.cuh"

namespace mad {
namespace {

constexpr int BM = 128;             // rows of A per tile (TMEM lanes)
constexpr int TM = BM;              // rows of C per tile
constexpr int BN = 256;             // columns of C per tile (TMEM columns)
constexpr int KATOM = 64;           // BF16 elements per 128-byte swizzle row
constexpr int A_ATOM_BYTES = BM * KATOM * 2;  // 16 KB: one K slice of the A panel
constexpr int B_ATOM_BYTES = BN * KATOM * 2;  // 32 KB: one K slice of a B tile (a stage)
constexpr int MAX_KATOMS = 10;      // K up to 640 (A panel 160 KB)
constexpr int MAX_STAGES = 8;
constexpr int kSched = 4;           // units in flight between the scheduler and the consumers
constexpr int kSmemOptIn = 232448;  // shared memory one block may opt into (227 KB)
constexpr int kStaticSmem = 2048;   // allowance for the kernel's static shared memory
constexpr int CAND_MIN = 4096;      // smallest per-CTA candidate buffer
constexpr unsigned kKeepMax = 1u << 16;  // largest rescore budget
#ifndef MAD_EPI_WARPS
#define MAD_EPI_WARPS 8
#endif
// 8 measured faster than 16: with 16 the registers drop to 96 a thread and
// the MMA issue slows.
constexpr int kEpiWarps = MAD_EPI_WARPS;       // epilogue warps (8 or 16)
constexpr int kEpi = kEpiWarps * 32;           // epilogue threads
constexpr int kThreads = kEpi + 3 * 32;        // producer, MMA issuer 0, epilogue, MMA issuer 1
constexpr int kCols = BN * 4 / kEpiWarps;      // accumulator columns per epilogue thread
constexpr int kChunks = kCols / 64;
// |c~_ij| <= (1 + K 2^-24) ||a~_i|| ||b~_j|| (Cauchy-Schwarz on the BF16
// vectors plus the FP32 accumulation error); the norms themselves carry
// FP32 rounding.  A generous factor keeps the skip test a proven bound.
constexpr float kBoundSlack = 1.01f;
constexpr long long kWaitCycles = 4000000000ll;  // ~2 s: a wait this long is a fault
constexpr uint32_t kSleepNs = 100000;            // longest sleep inside one try_wait
constexpr long long kDrainCycles = 200000000ll;  // ~0.1 s for copies in flight at an abort

struct GemmArgs {
  int64_t m, n;
  int kp;                            // padded K (a multiple of 64)
  int katoms;                        // kp / 64
  int nstage;                        // B stages
  int spt;                           // K slices per stage (a whole tile when K <= 128)
  int ksteps;                        // MMA K steps of 16 that reach column d
  int64_t tiles_m, tiles_n;
  int kkeep;                         // entries kept per CTA at compaction
  unsigned int* g_theta;             // shared threshold (FP32 bits)
  unsigned int* g_err;
  float* cta_val;                    // per-CTA candidate buffers (cta_cap entries each)
  unsigned long long* cta_key;
  unsigned cta_cap, cta_trigger;     // buffer size; compact before a tile when above trigger
  float* cand_val;                   // merged candidates
  unsigned long long* cand_key;
  unsigned long long* cand_count;
  unsigned long long cand_cap;
  float* dense_out;                  // diagnostics: full C~ (m x n) when set
  long long total_units;             // work units, handed out through g_next
  long long units_per_rb, unit_tiles; // stride 1: a unit is unit_tiles column tiles of a row block
  unsigned long long* g_next;        // next unit to hand out
  const uint32_t* perm_a;            // original row of A at each row position of the product
  const uint32_t* perm_b;            // original column of B at each column position
  const float* anorm;                // ||a~_i||_2 of the BF16 rows of A (m)
  const float* bgmax;                // max ||b~_j||_2 over each kCols-column group of B
  float* max_out;                    // threshold pre-pass: row-segment maxima
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait that lets the thread sleep up to `ns` nanoseconds (it resumes
// as soon as the phase completes): waiting warps then take no issue slots
// from the single threads that issue the MMAs and TMA copies.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the CTA is aborting or the limit passed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_sleep(bar, parity, kSleepNs)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

// Work units.  The main pass hands out runs of unit_tiles column tiles of
// one row block (tens per CTA) through a global counter, so CTAs whose
// tiles hold many candidates take fewer units.  The threshold pre-pass has
// one unit per row block of its corner: column tiles [0, unit_tiles).
struct Unit {
  long long rb, c0, c1;  // row block, column tiles [c0, c1)
};
__device__ __forceinline__ Unit unit_of(const GemmArgs& a, long long u) {
  Unit x;
  if (a.max_out) {
    x.rb = u;
    x.c0 = (u % a.units_per_rb) * a.unit_tiles;
    x.c1 = min(x.c0 + a.unit_tiles, (long long)a.tiles_n);
  } else {
    x.rb = u / a.units_per_rb;
    x.c0 = (u % a.units_per_rb) * a.unit_tiles;
    x.c1 = min(x.c0 + a.unit_tiles, (long long)a.tiles_n);
  }
  return x;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(const void* p) {
  const uint32_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = BM, N = BN.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The registers a tcgen05.ld wrote hold their values only after
// tcgen05.wait::ld; the compiler does not know that.  An empty statement
// that claims to rewrite them, placed after the wait, keeps every use of
// them after it.
template <int N>
__device__ __forceinline__ void tmem_regs_ready(uint32_t* r) {
#pragma unroll
  for (int i = 0; i < N; i += 8)
    asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                 "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7]));
}

__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Barrier among the epilogue threads only.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpi) : "memory"); }

struct Shared {
  uint64_t a_full, a_empty, done;
  uint64_t b_full[MAX_STAGES], b_empty[MAX_STAGES];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t sched_full[kSched], sched_empty[kSched];
  long long sched_unit[kSched];  // unit index, -1 = no more work
  long long epi_unit;
  uint32_t tmem_base;
  int abort_flag;
  int epi_abort;           // uniform exit decision of the four epilogue warps
  unsigned int count;      // candidates in the buffer
  unsigned int overflow;
  float theta;
  unsigned int hist[256];  // compaction
  unsigned int sel_prefix, sel_mask, sel_krem, sel_pick;
};

// The kkeep-th largest value among vals[0..n) (all >= 0) by MSB radix
// select on the FP32 bits; run by the epilogue threads.
__device__ float epi_kth_largest(const float* vals, unsigned n, unsigned kkeep, Shared* sh, int et) {
  if (et == 0) {
    sh->sel_prefix = 0;
    sh->sel_mask = 0;
    sh->sel_krem = kkeep;
  }
  for (int pass = 0; pass < 4; ++pass) {
    for (int b = et; b < 256; b += kEpi) sh->hist[b] = 0;
    epi_sync();
    const unsigned prefix = sh->sel_prefix, mask = sh->sel_mask;
    const int shift = 24 - 8 * pass;
    const unsigned rounds = (n + kEpi - 1) / kEpi;
    for (unsigned r = 0; r < rounds; ++r) {
      const unsigned x = r * kEpi + et;
      const unsigned bits = x < n ? __float_as_uint(vals[x]) : 0u;
      const bool in = x < n && (bits & mask) == prefix;
      const unsigned bin = in ? (bits >> shift) & 0xFFu : 0x100u;
      // one shared-memory atomic per distinct bin per warp
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, bin);
      if (in && (et & 31) == __ffs(peers) - 1) atomicAdd(&sh->hist[bin], __popc(peers));
    }
    epi_sync();
    if (et == 0) {
      unsigned above = 0;
      int b = 255;
      for (; b > 0; --b) {
        if (above + sh->hist[b] >= sh->sel_krem) break;
        above += sh->hist[b];
      }
      sh->sel_krem -= above;
      sh->sel_prefix |= (unsigned)b << shift;
      sh->sel_mask |= 0xFFu << shift;
    }
    epi_sync();
  }
  return __uint_as_float(sh->sel_prefix);
}

// Keep buffer entries [0, n) with value >= theta, in place and in order.
// Rounds of kEpi entries: every read of a round happens before any write of
// it, and a round writes only below its own end, so no entry is overwritten
// before it has been read.
__device__ unsigned epi_compact(float* cv, unsigned long long* ck, unsigned n, float theta,
                                Shared* sh, int et) {
  __shared__ unsigned int warp_keep[kEpi / 32];
  const int w = et >> 5, lane = et & 31;
  unsigned out = 0;
  for (unsigned base = 0; base < n; base += kEpi) {
    const unsigned x = base + et;
    float v = 0.0f;
    unsigned long long k = 0;
    bool keep = false;
    if (x < n) {
      v = cv[x];
      k = ck[x];
      keep = v >= theta;
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, keep);
    if (lane == 0) warp_keep[w] = __popc(mask);
    epi_sync();
    unsigned off = out, total = 0;
    for (int q = 0; q < kEpi / 32; ++q) {
      if (q < w) off += warp_keep[q];
      total += warp_keep[q];
    }
    if (keep) {
      const unsigned dst = off + __popc(mask & ((1u << lane) - 1u));
      cv[dst] = v;
      ck[dst] = k;
    }
    out += total;
    epi_sync();
  }
  if (et == 0) sh->count = out;
  epi_sync();
  return out;
}

// max(|a|, |b|, |c|) in one instruction (three-input max of sm_100 and later).
__device__ __forceinline__ float max3_abs(float a, float b, float c) {
  float r;
  asm("max.abs.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Largest |value| of 64 FP32 bit patterns: eight independent chains of
// three-input maxima (four instructions each), then a three-level fold.
__device__ __forceinline__ float abs_max64(const uint32_t* r) {
  float m[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    m[k] = max3_abs(__uint_as_float(r[k]), __uint_as_float(r[k + 8]), __uint_as_float(r[k + 16]));
    m[k] = max3_abs(m[k], __uint_as_float(r[k + 24]), __uint_as_float(r[k + 32]));
    m[k] = max3_abs(m[k], __uint_as_float(r[k + 40]), __uint_as_float(r[k + 48]));
    m[k] = fmaxf(m[k], fabsf(__uint_as_float(r[k + 56])));
  }
  return max3_abs(max3_abs(m[0], m[1], m[2]), max3_abs(m[3], m[4], m[5]), fmaxf(m[6], m[7]));
}

// Barrier of the epilogue threads that also returns whether any of them
// passed p = true (one barrier for the per-tile overflow and abort checks).
__device__ __forceinline__ bool epi_any(bool p) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "n"(kEpi)
      : "memory");
  return r != 0;
}

__global__ void __launch_bounds__(kThreads, 1)
k_gemm_topk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
            const GemmArgs args) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem =
      (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + args.katoms * A_ATOM_BYTES;
  const unsigned cap = args.cta_cap;
  float* cv = args.cta_val + (size_t)blockIdx.x * cap;
  unsigned long long* ck = args.cta_key + (size_t)blockIdx.x * cap;
  const int nstage = args.nstage;
  const int spt = args.spt;
  __shared__ Shared shared_state;
  Shared* sh = &shared_state;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort_flag = &sh->abort_flag;

  const int katoms = args.katoms;
  // Columns d..kp-1 are zeros: the MMAs stop at the first 16-column step
  // past d (7 steps instead of 8 for d = 100).
  const int ksteps = args.ksteps;

  if (threadIdx.x == 0) {
    mbar_init(&sh->a_full, 1);
    mbar_init(&sh->a_empty, 2);   // both MMA issuers
    mbar_init(&sh->done, 2);
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&sh->b_full[s], 1);
      mbar_init(&sh->b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&sh->acc_full[b], 1);
      mbar_init(&sh->acc_empty[b], kEpi / 32);
    }
    for (int k = 0; k < kSched; ++k) {
      mbar_init(&sh->sched_full[k], 1);
      mbar_init(&sh->sched_empty[k], 3);  // the two MMA issuers and the epilogue
    }
    sh->abort_flag = 0;
    sh->epi_abort = 0;
    sh->count = 0;
    sh->overflow = 0;
    sh->theta = __uint_as_float(*((volatile unsigned int*)args.g_theta));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sh->tmem_base)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem_base = sh->tmem_base;

  if (warp == 0) {
    // ---------------- scheduler and TMA producer ----------------
    if (lane == 0) {
      int s = 0;             // B stage of the next slice
      uint32_t phase = 0;    // parity of that stage's current use
      bool refill = false;   // every stage has been used once
      int ks = 0;            // scheduler slot
      uint32_t kph = 0;
      bool krefill = false;
      long long panel = 0;
      bool quit = false;
      while (!quit) {
        long long u = (long long)atomicAdd(args.g_next, 1ull);
        if (u >= args.total_units || *abort_flag) u = -1;
        if (krefill && !mbar_wait(&sh->sched_empty[ks], kph ^ 1u, abort_flag)) break;
        *((volatile long long*)&sh->sched_unit[ks]) = u;
        mbar_arrive(&sh->sched_full[ks]);
        if (++ks == kSched) {
          ks = 0;
          kph ^= 1u;
          krefill = true;
        }
        if (u < 0) break;
        const Unit x = unit_of(args, u);
        // The A panel of the unit's row block, once the previous unit's MMAs are done.
        if (panel > 0 && !mbar_wait(&sh->a_empty, (uint32_t)((panel - 1) & 1), abort_flag)) break;
        mbar_expect_tx(&sh->a_full, (uint32_t)(katoms * A_ATOM_BYTES));
        for (int ka = 0; ka < katoms; ++ka)
          tma_load_2d(sA + ka * A_ATOM_BYTES, &tmA, &sh->a_full, ka * KATOM, (int)(x.rb * TM));
        ++panel;
        for (long long cb = x.c0; cb < x.c1 && !quit; ++cb) {
          for (int k0 = 0; k0 < katoms; k0 += spt) {
            if (refill && !mbar_wait(&sh->b_empty[s], phase ^ 1u, abort_flag)) {
              quit = true;
              break;
            }
            mbar_expect_tx(&sh->b_full[s], (uint32_t)(spt * B_ATOM_BYTES));
            for (int j = 0; j < spt; ++j)
              tma_load_2d(sB + (s * spt + j) * B_ATOM_BYTES, &tmB, &sh->b_full[s], (k0 + j) * KATOM,
                          (int)(cb * BN));
            if (++s == nstage) {
              s = 0;
              phase ^= 1u;
              refill = true;
            }
          }
        }
      }
      if (*abort_flag) {
        // Winding down: let this CTA's copies in flight land before it
        // exits (stage s2's last load used parity `phase` when it is below
        // s, else the parity before).
        const long long t0 = clock64();
        for (int s2 = 0; s2 < nstage; ++s2) {
          if (s2 >= s && !refill) continue;   // never loaded
          const uint32_t ph = s2 < s ? phase : (phase ^ 1u);
          while (!mbar_try_wait(&sh->b_full[s2], ph) && clock64() - t0 < kDrainCycles) {
          }
        }
        if (panel > 0)
          while (!mbar_try_wait(&sh->a_full, (uint32_t)((panel - 1) & 1)) &&
                 clock64() - t0 < kDrainCycles) {
          }
      }
    }
  } else if (warp == 1 || warp == kThreads / 32 - 1) {
    // ---------------- MMA issuers ----------------
    // Issuer par takes the tiles with (tile index & 1) == par, and with
    // them accumulator par: while one thread waits on its barriers the
    // other's MMAs keep the tensor pipe busy (one thread alone spends as
    // long on its waits and commits as on the 7 MMAs of a K = 100 tile).
    if (lane == 0) {
      const int par = warp == 1 ? 0 : 1;
      const int groups = katoms / spt;   // stages per tile
      int s = 0;
      uint32_t phase = 0;
      int ks = 0;
      uint32_t kph = 0;
      long long panel = 0, it = 0;
      bool quit = false;
      // Descriptors of the first A slice and the first B stage; a K step of
      // 16 adds 32 bytes (2 in the descriptor's 16-byte address units).
      const uint64_t da0 = desc_sw128(sA), db0 = desc_sw128(sB);
      const uint32_t d_tmem = tmem_base + (uint32_t)(par * BN);
      while (!quit) {
        if (!mbar_wait(&sh->sched_full[ks], kph, abort_flag)) break;
        const long long u = *((volatile long long*)&sh->sched_unit[ks]);
        mbar_arrive(&sh->sched_empty[ks]);
        if (++ks == kSched) {
          ks = 0;
          kph ^= 1u;
        }
        if (u < 0) break;
        const Unit x = unit_of(args, u);
        if (!mbar_wait(&sh->a_full, (uint32_t)(panel & 1), abort_flag)) break;
        ++panel;
        for (long long cb = x.c0; cb < x.c1 && !quit; ++cb, ++it) {
          if ((int)(it & 1) != par) {   // the other issuer's tile: skip its stages
            for (int g = 0; g < groups; ++g)
              if (++s == nstage) {
                s = 0;
                phase ^= 1u;
              }
            continue;
          }
          for (int k0 = 0; k0 < katoms; k0 += spt) {
            // B first, then the accumulator: the B wait overlaps the
            // epilogue's drain of this accumulator.
            if (!mbar_wait(&sh->b_full[s], phase, abort_flag) ||
                (k0 == 0 && it >= 2 &&
                 !mbar_wait(&sh->acc_empty[par], (uint32_t)(((it >> 1) - 1) & 1), abort_flag))) {
              quit = true;
              break;
            }
            fence_after_sync();
            for (int j = 0; j < spt; ++j) {
              const int ka = k0 + j;
              const uint64_t da = da0 + (uint64_t)((ka * A_ATOM_BYTES) >> 4);
              const uint64_t db = db0 + (uint64_t)(((s * spt + j) * B_ATOM_BYTES) >> 4);
              // K steps of 16 inside this slice that reach column d (zeros past it).
              const int steps = min(4, ksteps - ka * 4);
              for (int kk = 0; kk < steps; ++kk)
                mma_bf16(d_tmem, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2),
                         (ka > 0 || kk > 0) ? 1u : 0u);
            }
            mma_commit(&sh->b_empty[s]);
            if (++s == nstage) {
              s = 0;
              phase ^= 1u;
            }
          }
          if (quit) break;
          mma_commit(&sh->acc_full[par]);
        }
        if (quit) break;
        mma_commit(&sh->a_empty);   // this issuer's MMAs of the unit done: its A panel may go
      }
    }
  } else {
    // ---------------- epilogue (warps 2..9) ----------------
    const int et = threadIdx.x - 64;          // 0..kEpi-1
    const int quarter = warp & 3;             // TMEM lane quarter of this warp
    const int cq = (warp - 2) >> 2;           // column group of the tile (kCols wide)
    const int row_in_tile = quarter * 32 + lane;
    const bool filter = !args.dense_out && !args.max_out;
    // The shared threshold, loaded one tile ahead so its latency never
    // stalls a tile (any earlier value is a valid, lower bound).
    float g_theta_next = __uint_as_float(*((volatile unsigned int*)args.g_theta));
    int ks = 0;
    uint32_t kph = 0;
    long long it = 0;
    bool quit_all = false;
    while (!quit_all) {
      // Thread 0 takes the next unit from the scheduler and shares it.
      if (et == 0) {
        long long u = -1;
        if (mbar_wait(&sh->sched_full[ks], kph, abort_flag)) {
          u = *((volatile long long*)&sh->sched_unit[ks]);
          mbar_arrive(&sh->sched_empty[ks]);
        }
        *((volatile long long*)&sh->epi_unit) = u;
      }
      if (++ks == kSched) {
        ks = 0;
        kph ^= 1u;
      }
      epi_sync();
      const long long u = *((volatile long long*)&sh->epi_unit);
      epi_sync();   // read by all before thread 0 writes the next one
      if (u < 0) break;
      const Unit x = unit_of(args, u);
      const int64_t urow = x.rb * TM + row_in_tile;
      const float arow = (filter && urow < args.m) ? args.anorm[urow] * kBoundSlack : 0.0f;
      for (long long cb = x.c0; cb < x.c1; ++cb, ++it) {
        const long long rb = x.rb;
        const int buf = (int)(it & 1);
        // The buffer's fill before this tile, the same in every thread: the
        // previous tile's writes all came before its closing barrier, and no
        // thread writes this tile's before the barrier below.  (Read after
        // that barrier, a fast warp's first writes could already be in it.)
        unsigned tile_start = filter ? sh->count : 0u;
        if (filter) epi_sync();
        // Compact first when the buffer is past its trigger.
        if (filter && tile_start > args.cta_trigger) {
          const unsigned held = min(tile_start, cap);
          const float th = epi_kth_largest(cv, held, (unsigned)args.kkeep, sh, et);
          tile_start = epi_compact(cv, ck, held, th, sh, et);
          if (et == 0) {
            sh->theta = fmaxf(sh->theta, th);
            atomicMax(args.g_theta, __float_as_uint(sh->theta));
          }
          epi_sync();
        }
        const float g_theta0 = g_theta_next;
        if (filter) g_theta_next = __uint_as_float(*((volatile unsigned int*)args.g_theta));
        // One decision per warp: the TMEM loads below are warp-collective.
        const bool ok =
            __all_sync(0xFFFFFFFFu, mbar_wait(&sh->acc_full[buf], (uint32_t)((it >> 1) & 1), abort_flag));
        const int64_t row = rb * TM + row_in_tile;
        const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(buf * BN + cq * kCols);
        const int64_t col_grp = cb * BN + cq * kCols;
        bool released = false;
        if (!filter) {
          // The diagnostic and pre-pass epilogues share named barriers, so
          // they leave together.
          if (!ok) atomicOr(&sh->epi_abort, 1);
          epi_sync();
          if (*((volatile int*)&sh->epi_abort)) {
            quit_all = true;
            break;
          }
          fence_after_sync();
        }
        if (args.dense_out) {
#pragma unroll 1
          for (int ch = 0; ch < kChunks; ++ch) {
            uint32_t r[64];
            tmem_ld32_nowait(taddr + (uint32_t)(ch * 64), r);
            tmem_ld32_nowait(taddr + (uint32_t)(ch * 64 + 32), r + 32);
            tmem_wait_ld();
            tmem_regs_ready<64>(r);
            const int64_t col0 = col_grp + ch * 64;
            if (row < args.m) {
#pragma unroll
              for (int q = 0; q < 64; ++q)
                if (col0 + q < args.n)
                  args.dense_out[(int64_t)args.perm_a[row] * args.n + args.perm_b[col0 + q]] =
                      __uint_as_float(r[q]);
            }
          }
        } else if (args.max_out) {
          // Threshold pre-pass: the largest |c~| of this thread's row segment.
          float hm = 0.0f;
#pragma unroll 1
          for (int ch = 0; ch < kChunks; ++ch) {
            uint32_t r[64];
            tmem_ld32_nowait(taddr + (uint32_t)(ch * 64), r);
            tmem_ld32_nowait(taddr + (uint32_t)(ch * 64 + 32), r + 32);
            tmem_wait_ld();
            tmem_regs_ready<64>(r);
            const int64_t rem = args.n - (col_grp + ch * 64);
            const int nvalid = rem >= 64 ? 64 : (rem > 0 ? (int)rem : 0);
            if (nvalid == 64) {
              hm = fmaxf(hm, abs_max64(r));
            } else {
#pragma unroll
              for (int q = 0; q < 64; ++q)
                hm = fmaxf(hm, q < nvalid ? fabsf(__uint_as_float(r[q])) : 0.0f);
            }
          }
          args.max_out[(u * args.unit_tiles + (cb - x.c0)) * kEpi + et] = row < args.m ? hm : 0.0f;
        } else {
          if (!ok) sh->epi_abort = 1;   // read by everyone after the barrier below
          // A row segment whose norm bound ||a~_i|| max_j ||b~_j|| is below
          // theta holds no candidate: a warp all of whose rows are below it
          // (about nine in ten) releases the accumulator without reading it.
          // Otherwise the largest |c~| of this thread's kCols values decides:
          // a warp none of whose values reaches theta releases the
          // accumulator at once; the others keep it and re-read their chunks
          // below.
          const float theta0 = fmaxf(sh->theta, g_theta0);
          const bool may = arow * args.bgmax[cb * (BN / kCols) + cq] >= theta0;
          bool hot = false;
          if (ok && __any_sync(0xFFFFFFFFu, may)) {
            fence_after_sync();
            uint32_t rr[kCols];
#pragma unroll
            for (int j = 0; j < kCols / 32; ++j)
              tmem_ld32_nowait(taddr + (uint32_t)(32 * j), rr + 32 * j);
            tmem_wait_ld();
            tmem_regs_ready<kCols>(rr);
            const int64_t rem = args.n - col_grp;
            const int nvalid = rem >= kCols ? kCols : (rem > 0 ? (int)rem : 0);
            float mx = 0.0f;
            if (nvalid == kCols) {
#pragma unroll
              for (int ch = 0; ch < kChunks; ++ch) mx = fmaxf(mx, abs_max64(rr + 64 * ch));
            } else {
#pragma unroll
              for (int q = 0; q < kCols; ++q)
                mx = fmaxf(mx, q < nvalid ? fabsf(__uint_as_float(rr[q])) : 0.0f);
            }
            hot = mx >= theta0 && row < args.m;
          }
          if (!__any_sync(0xFFFFFFFFu, hot)) {
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->acc_empty[buf]);
            released = true;   // and theta only rises: nothing of this warp passes below
          }
          bool stop = false;
          for (int round = 0; round < 8; ++round) {
            const float theta =
                fmaxf(sh->theta, round == 0 ? g_theta0
                                            : __uint_as_float(*((volatile unsigned int*)args.g_theta)));
            bool over = false;
            // Chunks of 64 columns, reloaded from TMEM on every pass (the
            // accumulator stays put until this warp releases it).
#pragma unroll 1
            for (int ch = 0; ch < kChunks && ok && !released; ++ch) {
              uint32_t r[64];
              tmem_ld32_nowait(taddr + (uint32_t)(ch * 64), r);
              tmem_ld32_nowait(taddr + (uint32_t)(ch * 64 + 32), r + 32);
              tmem_wait_ld();
              tmem_regs_ready<64>(r);
              const int64_t col0 = col_grp + ch * 64;
              const int64_t rem = args.n - col0;
              const int nvalid = rem >= 64 ? 64 : (rem > 0 ? (int)rem : 0);
              // Max first: the chunk is inspected element by element only when
              // its largest valid |c~| reaches theta.  nvalid is the same for
              // every lane of the warp, and all 64 columns are valid except in
              // the last column block.
              float mx = 0.0f;
              if (nvalid == 64) {
                mx = abs_max64(r);
              } else {
#pragma unroll
                for (int q = 0; q < 64; ++q)
                  mx = fmaxf(mx, q < nvalid ? fabsf(__uint_as_float(r[q])) : 0.0f);
              }
              unsigned cnt = 0;
              if (mx >= theta && row < args.m) {
#pragma unroll
                for (int q = 0; q < 64; ++q)
                  cnt += (q < nvalid && fabsf(__uint_as_float(r[q])) >= theta) ? 1u : 0u;
              }
              if (cnt) {
                // Reserve this thread's slots with one atomic, then write them.
                unsigned pos = atomicAdd(&sh->count, cnt);
                if (pos + cnt > cap) {
                  sh->overflow = 1;
                  over = true;
                }
#pragma unroll
                for (int q = 0; q < 64; ++q) {
                  const float a = fabsf(__uint_as_float(r[q]));
                  if (q < nvalid && a >= theta) {
                    if (pos < cap) {
                      cv[pos] = a;
                      ck[pos] = ((unsigned long long)args.perm_a[row] << 32) |
                                (unsigned long long)args.perm_b[col0 + q];
                    }
                    ++pos;
                  }
                }
              }
            }
            // One barrier: did any thread overflow the buffer or abort?
            if (!epi_any(over || !ok)) break;
            if (*((volatile int*)&sh->epi_abort)) {
              stop = true;
              break;
            }
            // Overflow: the buffer holds cap real entries, so its kkeep-th
            // largest is a valid lower bound.  Drop this tile's entries, tighten
            // the earlier ones and rescan the tile above it.
            const float th = epi_kth_largest(cv, cap, (unsigned)args.kkeep, sh, et);
            // The earlier tiles' survivors; the rescan appends after them.
            tile_start = epi_compact(cv, ck, tile_start, th, sh, et);
            if (et == 0) {
              sh->theta = fmaxf(sh->theta, th);
              sh->overflow = 0;
              atomicMax(args.g_theta, __float_as_uint(sh->theta));
            }
            epi_sync();
            if (round == 7 && et == 0) atomicOr(args.g_err, 2u);  // pathological ties
          }
          if (stop) {
            quit_all = true;
            break;
          }
        }
        if (!released) {
          fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&sh->acc_empty[buf]);
        }
      }
    }
    // Publish this CTA's survivors.
    epi_sync();
    if (!args.dense_out && !args.max_out) {
      const float theta =
          fmaxf(sh->theta, __uint_as_float(*((volatile unsigned int*)args.g_theta)));
      const unsigned n = min(sh->count, cap);
      for (unsigned x = et; x < n; x += kEpi) {
        if (cv[x] >= theta) {
          const unsigned long long pos = atomicAdd(args.cand_count, 1ull);
          if (pos < args.cand_cap) {
            args.cand_val[pos] = cv[x];
            args.cand_key[pos] = ck[x];
          }
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && sh->abort_flag) atomicOr(args.g_err, 1u);
  // Every MMA this CTA issued has completed: the epilogue consumed each
  // accumulator (or the CTA aborted, in which case wait for the MMA queue).
  const bool aborted = sh->abort_flag != 0;
  if (aborted && warp == kThreads / 32 - 1 && lane == 0) mma_commit(&sh->done);
  if (warp == 1) {
    if (aborted && lane == 0) {
      // Wait (bounded) for every MMA of both issuers still queued before
      // freeing TMEM.
      mma_commit(&sh->done);
      const long long t0 = clock64();
      while (!mbar_try_wait(&sh->done, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
    __syncwarp();
    fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512)
                 : "memory");
  }
}

// ---- casts: FP32/FP64 -> BF16, K padded with zeros ------------------------
// ---- norm order -------------------------------------------------------------
// Rows of A and columns of B enter the product grouped by their 2-norm,
// largest first (256 buckets of eighths of log2), so that the row segments
// and column groups the norm bound clears are whole warps and whole column
// groups, and the first row blocks and column tiles hold the largest
// products.  The order inside a bucket is the order of arrival; the
// products, and so the result, do not depend on it.
__device__ __forceinline__ int norm_bucket(float nrm) {
  if (!(nrm > 0.0f)) return 255;   // zero vectors last
  const int b = 127 - (int)floorf(log2f(nrm) * 8.0f);
  return min(max(b, 0), 254);
}

// One warp per row of A: its bucket, and the bucket counts.
template <typename T>
__global__ void __launch_bounds__(256)
k_row_buckets(const T* __restrict__ src, int64_t rows, int64_t cols, int64_t ld,
              uint8_t* __restrict__ bucket, unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[256];
  for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += warps) {
    float ss = 0.0f;
    for (int64_t c = lane; c < cols; c += 32) {
      const float v = (float)src[r * ld + c];
      ss = fmaf(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, off);
    if (lane == 0) {
      const int b = norm_bucket(sqrtf(ss));
      bucket[r] = (uint8_t)b;
      atomicAdd(&h[b], 1u);
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 256; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// One thread per column of B (d x n, row-major): its bucket and the counts.
template <typename T>
__global__ void __launch_bounds__(256)
k_col_buckets(const T* __restrict__ B, int64_t d, int64_t n, int64_t ldb,
              uint8_t* __restrict__ bucket, unsigned int* __restrict__ hist) {
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    float ss = 0.0f;
    for (int64_t k = 0; k < d; ++k) {
      const float v = (float)B[k * ldb + j];
      ss = fmaf(v, v, ss);
    }
    const int b = norm_bucket(sqrtf(ss));
    bucket[j] = (uint8_t)b;
    atomicAdd(&h[b], 1u);
  }
  __syncthreads();
  if (h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], h[threadIdx.x]);
}

// Exclusive scans of the two 256-bucket counts into cursors (one block).
__global__ void __launch_bounds__(256)
k_bucket_cursors(const unsigned int* __restrict__ hist_a, const unsigned int* __restrict__ hist_b,
                 unsigned int* __restrict__ cur_a, unsigned int* __restrict__ cur_b) {
  __shared__ unsigned int s[2][256];
  const int t = threadIdx.x;
  s[0][t] = hist_a[t];
  s[1][t] = hist_b[t];
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {
    const unsigned a = t >= off ? s[0][t - off] : 0u, b = t >= off ? s[1][t - off] : 0u;
    __syncthreads();
    s[0][t] += a;
    s[1][t] += b;
    __syncthreads();
  }
  cur_a[t] = s[0][t] - hist_a[t];
  cur_b[t] = s[1][t] - hist_b[t];
}

// Position of every column of B in the product, and the inverse map.  A
// block counts its 256 columns per bucket, takes a range of each bucket with
// one global atomic, and hands the places out in shared memory.
__global__ void __launch_bounds__(256)
k_claim_cols(const uint8_t* __restrict__ bucket, int64_t n, unsigned int* __restrict__ cur,
             uint32_t* __restrict__ pos, uint32_t* __restrict__ perm) {
  __shared__ unsigned int base[256];
  base[threadIdx.x] = 0;
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int b = j < n ? bucket[j] : -1;
  if (b >= 0) atomicAdd(&base[b], 1u);
  __syncthreads();
  if (base[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cur[threadIdx.x], base[threadIdx.x]);
  __syncthreads();
  if (b < 0) return;
  const uint32_t q = atomicAdd(&base[b], 1u);
  pos[j] = q;
  perm[q] = (uint32_t)j;
}

// One warp per row; the row goes to the next place of its bucket.  Lane L
// writes the BF16 pairs at columns 2L + 64j, and the warp the 2-norm of the
// rounded row.  The block first counts its rows per bucket and takes a range
// of each bucket with one global atomic; places are then handed out in
// shared memory.
template <typename T>
__global__ void __launch_bounds__(256)
k_cast_rows_bf16(const T* __restrict__ src, int64_t rows, int64_t cols, int64_t ld, int kp,
                 const uint8_t* __restrict__ bucket, unsigned int* __restrict__ cur,
                 __nv_bfloat16* __restrict__ dst, float* __restrict__ norm,
                 uint32_t* __restrict__ perm) {
  __shared__ unsigned int base[256];
  base[threadIdx.x] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5);
  // This block's rows are w0 + w + k * warps (w < 8): slot s = 8k + w.
  for (int64_t sl = threadIdx.x;; sl += blockDim.x) {
    const int64_t r = w0 + (sl & 7) + (sl >> 3) * warps;
    if (r >= rows) break;
    atomicAdd(&base[bucket[r]], 1u);
  }
  __syncthreads();
  if (base[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cur[threadIdx.x], base[threadIdx.x]);
  __syncthreads();
  for (int64_t r = w0 + (threadIdx.x >> 5); r < rows; r += warps) {
    uint32_t q = 0;
    if (lane == 0) {
      q = atomicAdd(&base[bucket[r]], 1u);
      perm[q] = (uint32_t)r;
    }
    q = __shfl_sync(0xFFFFFFFFu, q, 0);
    const T* a = src + r * ld;
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(dst + (int64_t)q * kp);
    float ss = 0.0f;
    for (int c = 2 * lane; c < kp; c += 64) {
      const float v0 = c < cols ? (float)a[c] : 0.0f;
      const float v1 = c + 1 < cols ? (float)a[c + 1] : 0.0f;
      const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
      o[c >> 1] = h;
      const float2 f = __bfloat1622float2(h);
      ss = fmaf(f.x, f.x, fmaf(f.y, f.y, ss));
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, off);
    if (lane == 0) norm[q] = sqrtf(ss);
  }
}

// Largest 2-norm of the BF16 columns of B in each group of `group` columns
// (rows of B^T, kp wide): one block per group, one thread per column.
__global__ void __launch_bounds__(128)
k_group_col_norms(const __nv_bfloat16* __restrict__ bt, int64_t n, int kp, int group,
                  float* __restrict__ gmax) {
  const int64_t j = (int64_t)blockIdx.x * group + threadIdx.x;
  float ss = 0.0f;
  if (threadIdx.x < group && j < n) {
    const __nv_bfloat162* row = reinterpret_cast<const __nv_bfloat162*>(bt + j * kp);
    for (int c = 0; c < kp / 2; ++c) {
      const float2 f = __bfloat1622float2(row[c]);
      ss = fmaf(f.x, f.x, fmaf(f.y, f.y, ss));
    }
  }
  float v = sqrtf(ss);
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xFFFFFFFFu, v, off));
  __shared__ float wmax[4];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0)
    gmax[blockIdx.x] = fmaxf(fmaxf(wmax[0], wmax[1]), fmaxf(wmax[2], wmax[3]));
}

// B (d x n) -> B^T (n x kp) in BF16.
template <typename T>
__global__ void k_cast_cols_bf16(const T* __restrict__ B, int64_t d, int64_t n, int64_t ldb, int kp,
                                 const uint32_t* __restrict__ pos, __nv_bfloat16* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t k = k0 + r, j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (k < d && j < n) ? (float)B[k * ldb + j] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, k = k0 + threadIdx.x;
    if (j < n && k < kp) dst[(int64_t)pos[j] * kp + k] = __float2bfloat16_rn(tile[threadIdx.x][r]);
  }
}

// Threshold from the pre-pass maxima: every maximum is a distinct entry of
// C~, so the kkeep-th largest maximum is at most the kkeep-th largest entry.
// A 4096-bucket histogram of the FP32 bits (exponent and 4 mantissa bits)
// gives the floor of the bucket where the count from the top reaches kkeep,
// a lower bound of that maximum, in one pass; the last block publishes it.
__global__ void __launch_bounds__(256)
k_max_floor(const float* __restrict__ v, unsigned long long n, unsigned kkeep,
            unsigned int* __restrict__ hist, unsigned int* ticket, unsigned int* g_theta) {
  __shared__ unsigned int h[4096];
  for (int b = threadIdx.x; b < 4096; b += blockDim.x) h[b] = 0;
  __syncthreads();
  constexpr int U = 4;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long rounds = (n + U * stride - 1) / (U * stride);
  for (unsigned long long r = 0; r < rounds; ++r) {
    float f[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const unsigned long long x = (r * U + q) * stride + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
      f[q] = x < n ? __ldcs(v + x) : -1.0f;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const unsigned bin = f[q] >= 0.0f ? (__float_as_uint(f[q]) >> 19) : 0x1000u;
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, bin);
      if (bin < 4096u && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&h[bin], __popc(peers));
    }
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 4096; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
  __threadfence();
  __shared__ unsigned int is_last;
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  unsigned long long total = 0;
  const int b = block_pick_from_top<4096>(hist, kkeep, &total);
  if (threadIdx.x == 0 && b >= 0) atomicMax(g_theta, (unsigned)b << 19);
}

// FP32 rescore of the selected candidates: lane L sums k = L mod 32 with
// fused multiply-add in FP32, then the partials fold in halves.
template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
k_rescore_fp32(const Item* __restrict__ sel, unsigned long long nsel, const TA* __restrict__ A,
               int64_t lda, const TB* __restrict__ B, int64_t ldb, int64_t d,
               float* __restrict__ cvals, Item* __restrict__ items) {
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned long long warps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long q = warp; q < nsel; q += warps) {
    const uint32_t i = (uint32_t)(sel[q].key >> 32), j = (uint32_t)sel[q].key;
    float acc = 0.0f;
    for (int64_t k = lane; k < d; k += 32)
      acc = __fmaf_rn((float)A[(int64_t)i * lda + k], (float)B[k * ldb + j], acc);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xFFFFFFFFu, acc, off));
    if (lane == 0) {
      cvals[q] = acc;
      Item it;
      it.p = (unsigned long long)__float_as_uint(fabsf(acc));
      it.key = sel[q].key;
      it.aux = q;
      items[q] = it;
    }
  }
}

__global__ void k_cand_items(const float* __restrict__ val, const unsigned long long* __restrict__ key,
                             unsigned long long n, Item* __restrict__ out) {
  const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  Item it;
  it.p = (unsigned long long)__float_as_uint(val[x]);
  it.key = key[x];
  it.aux = x;
  out[x] = it;
}

__global__ void k_fp32_pairs(const Item* __restrict__ items, unsigned long long n,
                             const float* __restrict__ cvals, mad_pair* __restrict__ out) {
  const unsigned long long x = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  mad_pair pr;
  pr.i = (uint32_t)(items[x].key >> 32);
  pr.j = (uint32_t)items[x].key;
  pr.x = 0;
  pr.c = (double)cvals[items[x].aux];
  out[x] = pr;
}

// ---- host side -----------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, uint64_t rows, int kp, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)KATOM, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct NormOrder {
  uint8_t* bkt_a;      // bucket of each row of A (m)
  uint8_t* bkt_b;      // bucket of each column of B (n)
  unsigned int* hist;  // 256 counts for A, then 256 for B
  unsigned int* cur;   // their exclusive scans, advanced as places are taken
  uint32_t* perm_a;    // original row at each row position
  uint32_t* perm_b;    // original column at each column position
  uint32_t* pos_b;     // position of each original column
};

// BF16 copies of A (rows) and B^T (columns of B as rows) in norm order,
// the 2-norms of the rounded rows of A and the column-group maxima of B.
template <typename T>
void launch_casts(const mad_matrix* A, const mad_matrix* B, int kp, const NormOrder& o,
                  __nv_bfloat16* Abf, __nv_bfloat16* Bbf, float* anorm, float* bgmax,
                  cudaStream_t st) {
  const int64_t m = A->rows, n = B->cols;
  const int64_t blocks = (m + 7) / 8;   // a warp per row
  const unsigned rgrid = (unsigned)(blocks < 152 * 16 ? blocks : 152 * 16);
  const unsigned cgrid = (unsigned)((n + 255) / 256);
  cudaMemsetAsync(o.hist, 0, 512 * sizeof(unsigned int), st);
  k_row_buckets<T><<<rgrid, 256, 0, st>>>((const T*)A->values, m, A->cols, A->ld, o.bkt_a, o.hist);
  k_col_buckets<T><<<cgrid, 256, 0, st>>>((const T*)B->values, B->rows, n, B->ld, o.bkt_b,
                                          o.hist + 256);
  k_bucket_cursors<<<1, 256, 0, st>>>(o.hist, o.hist + 256, o.cur, o.cur + 256);
  k_cast_rows_bf16<T><<<rgrid, 256, 0, st>>>((const T*)A->values, m, A->cols, A->ld, kp, o.bkt_a,
                                             o.cur, Abf, anorm, o.perm_a);
  k_claim_cols<<<cgrid, 256, 0, st>>>(o.bkt_b, n, o.cur + 256, o.pos_b, o.perm_b);
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((kp + 31) / 32));
  k_cast_cols_bf16<T><<<grid, dim3(32, 8), 0, st>>>((const T*)B->values, B->rows, n, B->ld, kp,
                                                    o.pos_b, Bbf);
  // Every group of every column tile, the ones past n included (norm 0).
  const int64_t groups = (B->cols + BN - 1) / BN * (BN / kCols);
  k_group_col_norms<<<(unsigned)groups, 128, 0, st>>>(Bbf, B->cols, kp, kCols, bgmax);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

// Shared by mad_dense_topt and the diagnostic full-product entry point.
mad_status dense_comparator(mad_ctx* ctx, const mad_matrix* A, const mad_matrix* B, uint32_t t,
                            uint32_t rescore, mad_pair* out, uint32_t* n_out, float* dense_out,
                            cudaStream_t st) {
  const int64_t m = A->rows, d = A->cols, n = B->cols;
  const int katoms = (int)((d + KATOM - 1) / KATOM);
  if (katoms > MAX_KATOMS) return MAD_ERR_UNSUPPORTED;
  const int kp = katoms * KATOM;
  // B stages: a whole tile each when K <= 128 (one barrier per tile), else
  // one K slice each; as many as the shared memory the A panel leaves holds
  // (at least two).
  const int spt = katoms <= 2 ? katoms : 1;
  const int nstage = std::min<int>(
      MAX_STAGES,
      (kSmemOptIn - kStaticSmem - 1024 - katoms * A_ATOM_BYTES) / (spt * B_ATOM_BYTES));
  if (nstage < 2) return MAD_ERR_UNSUPPORTED;
  const int smem_bytes = katoms * A_ATOM_BYTES + nstage * spt * B_ATOM_BYTES + 1024;
  const int64_t tiles_m = (m + TM - 1) / TM, tiles_n = (n + BN - 1) / BN;
  const int grid = (int)std::min<int64_t>(sm_count(), tiles_m * tiles_n);
  const uint32_t kkeep = dense_out ? 1u : std::max(t, rescore);
  if (!dense_out && kkeep > kKeepMax) return MAD_ERR_UNSUPPORTED;
  // Per-CTA buffer: four rescore budgets (at least 4096), compacted at half.
  const unsigned cta_cap = std::max<unsigned>(CAND_MIN, (4u * kkeep + 255u) & ~255u);
  const unsigned long long cand_cap = (unsigned long long)grid * cta_cap;
  auto al = [](size_t x) { return (x + 1023) & ~(size_t)1023; };
  const size_t a_bytes = al((size_t)m * kp * 2), b_bytes = al((size_t)n * kp * 2);
  const size_t cv_bytes = al(cand_cap * 4), ck_bytes = al(cand_cap * 8);
  const size_t ws_bytes = al(select_ws_bytes(cand_cap, kkeep));
  const size_t ws2_bytes = al(select_ws_bytes(kkeep, t ? t : 1));
  const size_t cvals_bytes = al((size_t)kkeep * 4);
  // Pre-pass: the corner of the largest norms, the first eighth of the row
  // blocks times the first eighth of the column tiles (a 64th of the tiles).
  const long long pre_rows = (tiles_m + 7) / 8, pre_cols = (tiles_n + 7) / 8;
  const long long pre_tiles = pre_rows * pre_cols;   // slots of the row-segment maxima
  const size_t pre_bytes = al((size_t)pre_tiles * kEpi * 4);
  const size_t hist_bytes = al(4097 * 4);
  const size_t anorm_bytes = al((size_t)m * 4);
  const size_t order_bytes = al((size_t)m) + al((size_t)n) + al(1024 * 4) + al((size_t)m * 4) +
                             2 * al((size_t)n * 4);
  const size_t bgmax_bytes = al((size_t)(tiles_n * (BN / kCols)) * 4);
  const size_t total = a_bytes + b_bytes + 2 * cv_bytes + 2 * ck_bytes + ws_bytes + ws2_bytes +
                       cvals_bytes + pre_bytes + hist_bytes + anorm_bytes + bgmax_bytes +
                       order_bytes + 1024;
  mad_status rs = ensure_scratch(ctx, total, st);
  if (rs != MAD_OK) return rs;
  char* p = (char*)ctx->scratch;
  __nv_bfloat16* Abf = (__nv_bfloat16*)p;             p += a_bytes;
  __nv_bfloat16* Bbf = (__nv_bfloat16*)p;             p += b_bytes;
  float* cand_val = (float*)p;                        p += cv_bytes;
  unsigned long long* cand_key = (unsigned long long*)p; p += ck_bytes;
  float* anorm = (float*)p;                           p += anorm_bytes;
  NormOrder ord;
  ord.bkt_a = (uint8_t*)p;                            p += al((size_t)m);
  ord.bkt_b = (uint8_t*)p;                            p += al((size_t)n);
  ord.hist = (unsigned int*)p;
  ord.cur = ord.hist + 512;                           p += al(1024 * 4);
  ord.perm_a = (uint32_t*)p;                          p += al((size_t)m * 4);
  ord.perm_b = (uint32_t*)p;                          p += al((size_t)n * 4);
  ord.pos_b = (uint32_t*)p;                           p += al((size_t)n * 4);
  float* bgmax = (float*)p;                           p += bgmax_bytes;
  float* cta_val = (float*)p;                         p += cv_bytes;
  unsigned long long* cta_key = (unsigned long long*)p; p += ck_bytes;
  char* wsb = p;                                      p += ws_bytes;
  char* ws2b = p;                                     p += ws2_bytes;
  float* cvals = (float*)p;                           p += cvals_bytes;
  float* pre_max = (float*)p;                         p += pre_bytes;
  unsigned int* pre_hist = (unsigned int*)p;          p += hist_bytes;
  unsigned int* g_theta = (unsigned int*)p;
  unsigned int* g_err = g_theta + 1;
  unsigned long long* cand_count = (unsigned long long*)(g_theta + 2);
  unsigned long long* next_pre = cand_count + 1;   // unit counters of the two passes
  unsigned long long* next_main = cand_count + 2;
  cudaMemsetAsync(g_theta, 0, 64, st);
  cudaMemsetAsync(pre_hist, 0, 4097 * 4, st);

  if (A->dt == MAD_F64) launch_casts<double>(A, B, kp, ord, Abf, Bbf, anorm, bgmax, st);
  else launch_casts<float>(A, B, kp, ord, Abf, Bbf, anorm, bgmax, st);
  count_launch(ctx, 7);

  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, Abf, (uint64_t)m, kp, BM) || !make_map(&tmB, Bbf, (uint64_t)n, kp, BN))
    return MAD_ERR_CUDA;
  static int attr_bytes = 0;
  if (smem_bytes > attr_bytes) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_topk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes);
    if (e != cudaSuccess) return cuda_status(e);
    attr_bytes = smem_bytes;
  }
  GemmArgs ga;
  ga.m = m;
  ga.n = n;
  ga.kp = kp;
  ga.katoms = katoms;
  ga.nstage = nstage;
  ga.spt = spt;
  ga.ksteps = (int)((d + 15) / 16);
  ga.tiles_m = tiles_m;
  ga.tiles_n = tiles_n;
  ga.kkeep = (int)kkeep;
  ga.g_theta = g_theta;
  ga.g_err = g_err;
  ga.perm_a = ord.perm_a;
  ga.perm_b = ord.perm_b;
  ga.anorm = anorm;
  ga.bgmax = bgmax;
  ga.cta_val = cta_val;
  ga.cta_key = cta_key;
  ga.cta_cap = cta_cap;
  ga.cta_trigger = cta_cap / 2;
  ga.cand_val = cand_val;
  ga.cand_key = cand_key;
  ga.cand_count = cand_count;
  ga.cand_cap = cand_cap;
  ga.dense_out = dense_out;
  // Units of about a 32nd of a CTA's share of tiles, cut evenly from a row
  // block's column tiles.
  {
    const long long share = tiles_m * tiles_n / ((long long)grid * 32);
    long long ut = std::max<long long>(1, std::min<long long>(tiles_n, share));
    const long long upr = (tiles_n + ut - 1) / ut;
    ut = (tiles_n + upr - 1) / upr;
    ga.unit_tiles = ut;
    ga.units_per_rb = upr;
    ga.total_units = tiles_m * upr;
  }
  ga.g_next = next_main;
  ga.max_out = nullptr;
  if (!dense_out) {
    // Threshold pre-pass over the corner of the largest norms, one unit
    // per row block: row-segment maxima.
    GemmArgs pre = ga;
    pre.max_out = pre_max;
    pre.unit_tiles = pre_cols;
    pre.units_per_rb = 1;
    pre.total_units = pre_rows;
    pre.g_next = next_pre;
    k_gemm_topk<<<(int)std::min<long long>(grid, pre_rows), kThreads, smem_bytes, st>>>(tmA, tmB,
                                                                                      pre);
    k_max_floor<<<152 * 2, 256, 0, st>>>(pre_max, (unsigned long long)pre_tiles * kEpi, kkeep,
                                         pre_hist, pre_hist + 4096, g_theta);
    count_launch(ctx, 2);
  }
  k_gemm_topk<<<grid, kThreads, smem_bytes, st>>>(tmA, tmB, ga);
  count_launch(ctx);
  if ((rs = cuda_status(cudaGetLastError())) != MAD_OK) return rs;

  unsigned int herr = 0;
  unsigned long long ncand = 0;
  cudaMemcpyAsync(&herr, g_err, sizeof(herr), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&ncand, cand_count, sizeof(ncand), cudaMemcpyDeviceToHost, st);
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  if (herr & 1u) return MAD_ERR_CUDA;      // a pipeline wait timed out
  if (dense_out) return MAD_OK;
  if (herr & 2u) return MAD_ERR_STATE;     // candidate buffer could not be tightened
  if (ncand > cand_cap) return MAD_ERR_STATE;

  // 8t largest |c~| of the merged candidates, then the FP32 rescore.
  const SelectWs ws = select_ws_carve(wsb, cand_cap, kkeep);
  if (ncand) {
    k_cand_items<<<(unsigned)((ncand + 255) / 256), 256, 0, st>>>(cand_val, cand_key, ncand, ws.l0);
    count_launch(ctx);
  }
  uint64_t nsel = 0;
  if ((rs = select_list(ctx, ws, ncand, kkeep, 4, &nsel, st)) != MAD_OK) return rs;
  const SelectWs ws2 = select_ws_carve(ws2b, kkeep, t ? t : 1);
  if (nsel) {
    const unsigned long long blocks = (nsel * 32 + 255) / 256;
    if (A->dt == MAD_F64 && B->dt == MAD_F64)
      k_rescore_fp32<double, double><<<(unsigned)blocks, 256, 0, st>>>(
          ws.out, nsel, (const double*)A->values, A->ld, (const double*)B->values, B->ld, d, cvals, ws2.l0);
    else if (A->dt == MAD_F64)
      k_rescore_fp32<double, float><<<(unsigned)blocks, 256, 0, st>>>(
          ws.out, nsel, (const double*)A->values, A->ld, (const float*)B->values, B->ld, d, cvals, ws2.l0);
    else if (B->dt == MAD_F64)
      k_rescore_fp32<float, double><<<(unsigned)blocks, 256, 0, st>>>(
          ws.out, nsel, (const float*)A->values, A->ld, (const double*)B->values, B->ld, d, cvals, ws2.l0);
    else
      k_rescore_fp32<float, float><<<(unsigned)blocks, 256, 0, st>>>(
          ws.out, nsel, (const float*)A->values, A->ld, (const float*)B->values, B->ld, d, cvals, ws2.l0);
    count_launch(ctx);
  }
  uint64_t nt = 0;
  if ((rs = select_list(ctx, ws2, nsel, t, 4, &nt, st)) != MAD_OK) return rs;
  if (nt) {
    k_fp32_pairs<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(ws2.out, nt, cvals, out);
    count_launch(ctx);
  }
  if ((rs = cuda_status(cudaStreamSynchronize(st))) != MAD_OK) return rs;
  *n_out = (uint32_t)nt;
  return MAD_OK;
}

}  // namespace mad
