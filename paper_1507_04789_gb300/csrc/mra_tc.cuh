// mra_tc.cuh -- 5th-generation tensor-core (tcgen05) tile product for the
// mixed-precision form: FP64 operands, 3xTF32 products, FP64 accumulation.
//
// C(128 x 64) += A(128 x K) B(64 x K)' with the operands read in FP64 (any
// strides, like tile_mma) and split as x = hi + lo, hi = tf32(x), lo =
// tf32(x - hi).  Each K-step of 8 issues three tcgen05.mma kind::tf32
// (hi*hi + hi*lo + lo*hi, the lo*lo term is dropped), accumulating in FP32 in
// tensor memory; every 64 columns of K the FP32 partial is read back with
// tcgen05.ld and added to FP64 registers, so the accumulation error does not
// grow with K.  This keeps the relative error of each product near 2^-22,
// which the M-RA prior chain, the leaf covariance and the leaf solve tolerate
// (|d loglik| / n about 5e-7 at n = 2^14 .. 2^18); the Gram products of the
// posterior pass do not, and stay in FP64.
//
// Operands are staged in shared memory in the canonical no-swizzle K-major
// layout: 8-row x 16-byte core matrices, 128 B each, adjacent K-cores 128 B
// apart (leading byte offset) and adjacent 8-row groups 8 x 128 B apart
// (stride byte offset).  One elected thread issues the MMAs and commits them
// to an mbarrier; every wait on it is bounded, and a timeout sets the CTA's
// error flag instead of hanging.
#pragma once
#include "mra_device.cuh"

namespace mra {

constexpr int TC_M = 128, TC_N = 64, TC_KC = 32;            // tile, staged K chunk (tf32)
constexpr int TC_KCORES = TC_KC / 4;                         // 16-byte core columns per chunk
constexpr int TC_A_WORDS = TC_M * TC_KC;                     // one of hi/lo for A
constexpr int TC_B_WORDS = TC_N * TC_KC;
constexpr int TC_STAGE_BYTES = 4 * 2 * (TC_A_WORDS + TC_B_WORDS);   // 48 KB
constexpr uint32_t TC_TMEM_COLS = 64;
constexpr long TC_WAIT_LIMIT = 1L << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
         ((uint64_t)(((TC_KCORES * 128u) >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M x N.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ int tc_cm(int row, int k) {   // word index in a staged operand
  return (((row >> 3) * TC_KCORES + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
  return u;
}

// Per-CTA tensor-core context: TMEM columns, mbarrier and its phase.
struct TcCtx {
  uint32_t* stage;      // TC_STAGE_BYTES of shared memory, 1 KB aligned
  uint64_t* mbar;       // shared
  uint32_t tmem;        // accumulator base address
  uint32_t phase;
  int* fail;            // shared flag: a wait timed out
};

// Output ownership: thread (warp w, lane l) holds row 32 (w % 4) + l and the
// 32 columns starting at 32 (w / 4) of the 128 x 64 tile.
struct TcAcc {
  double v[32];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = 0.0;
  }
  __device__ __forceinline__ int row() const { return (((threadIdx.x >> 5) & 3) << 5) | (threadIdx.x & 31); }
  __device__ __forceinline__ int col0() const { return (threadIdx.x >> 7) << 5; }
};

// Allocate TMEM (warp 0) and set up the mbarrier; all threads call it.
__device__ inline void tc_init(TcCtx& cx, uint32_t* tmem_slot) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(cx.mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    *cx.fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  cx.tmem = *tmem_slot;
  cx.phase = 0;
}

// Release TMEM (warp 0); all threads call it, after their last tcgen05.ld.
__device__ inline void tc_release(TcCtx& cx) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cx.tmem), "r"(TC_TMEM_COLS));
}

// Stage rows [0, nx) x k [k0, k0 + kn) of X (FP64, element (i, k) at
// X[i * sxi + k * sxk]) as tf32 hi/lo pairs; zero outside.
__device__ __forceinline__ void tc_stage(uint32_t* hi, uint32_t* lo, int rows, const double* X, long sxi, long sxk,
                                         int nx, int k0, int kn) {
  const int total = rows * TC_KC;
  if (sxk == 1) {
    for (int t = threadIdx.x; t < total; t += NT) {
      int i = t / TC_KC, k = t - i * TC_KC;
      float f = (i < nx && k < kn) ? (float)X[i * sxi + (long)(k0 + k)] : 0.f;
      uint32_t h = to_tf32(f);
      int w = tc_cm(i, k);
      hi[w] = h;
      lo[w] = to_tf32(f - __uint_as_float(h));
    }
  } else {
    for (int t = threadIdx.x; t < total; t += NT) {
      int k = t / rows, i = t - k * rows;
      float f = (i < nx && k < kn) ? (float)X[(long)(k0 + k) * sxk + i * sxi] : 0.f;
      uint32_t h = to_tf32(f);
      int w = tc_cm(i, k);
      hi[w] = h;
      lo[w] = to_tf32(f - __uint_as_float(h));
    }
  }
}

__device__ __forceinline__ void tc_issue(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(TC_IDESC), "r"(accumulate));
}

// Wait (bounded) for the MMAs committed to an mbarrier; flips the phase once
// they completed.  Returns false on timeout (phase unchanged).
__device__ __forceinline__ bool tc_wait_phase(uint64_t* mbar, uint32_t& phase) {
  uint32_t done = 0;
  for (long it = 0; it < TC_WAIT_LIMIT && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(phase));
  }
  if (done) phase ^= 1;
  return done != 0;
}

// After a timed-out wait: flag the failure and give the MMAs still in flight
// one more bounded wait before the caller frees tensor memory.
__device__ __forceinline__ void tc_abandon(uint64_t* mbar, uint32_t& phase, int* fail) {
  if (threadIdx.x == 0) *fail = 1;
  tc_wait_phase(mbar, phase);
  __syncthreads();
}

__device__ __forceinline__ bool tc_wait(TcCtx& cx) { return tc_wait_phase(cx.mbar, cx.phase); }

// Add the FP32 accumulator to the FP64 registers of this thread.
__device__ __forceinline__ void tc_drain(TcCtx& cx, TcAcc& acc) {
  uint32_t r[32];
  const uint32_t taddr = cx.tmem + ((uint32_t)((threadIdx.x >> 5) & 3) << 21) + (uint32_t)acc.col0();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int c = 0; c < 32; ++c) acc.v[c] += (double)__uint_as_float(r[c]);
}

// acc(i, j) += sum_k A(i, k) B(j, k), i < na <= 128, j < nb <= 64.
// Returns false (uniformly) if a tensor-core wait timed out.
__device__ inline bool tc_mma(TcCtx& cx, TcAcc& acc, const double* A, long sai, long sak, int na, const double* B,
                              long sbj, long sbk, int nb, int K) {
  uint32_t* aH = cx.stage;
  uint32_t* aL = aH + TC_A_WORDS;
  uint32_t* bH = aL + TC_A_WORDS;
  uint32_t* bL = bH + TC_B_WORDS;
  bool ok = true;
  for (int k0 = 0; k0 < K; k0 += TC_KC) {
    const int kn = min(TC_KC, K - k0);
    tc_stage(aH, aL, TC_M, A, sai, sak, na, k0, kn);
    tc_stage(bH, bL, TC_N, B, sbj, sbk, nb, k0, kn);
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool first = (k0 & 63) == 0;            // a new 64-column accumulation group
    if (threadIdx.x == 0) {
      for (int j = 0; j < TC_KC / 8; ++j) {
        const uint32_t off = (uint32_t)j * 256u;   // two 16-byte core columns per K-step
        const uint64_t ah = tc_desc(smem_addr(aH) + off), al = tc_desc(smem_addr(aL) + off);
        const uint64_t bh = tc_desc(smem_addr(bH) + off), bl = tc_desc(smem_addr(bL) + off);
        tc_issue(cx.tmem, ah, bh, (first && j == 0) ? 0u : 1u);
        tc_issue(cx.tmem, ah, bl, 1u);
        tc_issue(cx.tmem, al, bh, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(cx.mbar)));
    }
    const bool done = tc_wait(cx);
    if (__syncthreads_or(!done)) {            // uniform: every thread leaves the loop
      tc_abandon(cx.mbar, cx.phase, cx.fail);
      ok = false;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    const bool group_end = ((k0 + TC_KC) & 63) == 0 || k0 + TC_KC >= K;
    if (group_end) tc_drain(cx, acc);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();                          // staging and TMEM are free for the next chunk
  }
  return ok;
}

}  // namespace mra
