// mra_emu.cuh -- FP64-grade tile product on the tcgen05 tensor cores.
//
// GB300 retires 2 FP64 FMA per clock per SM, so FP64 contractions are emulated
// with the error-free splitting of Ozaki et al. (2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications"), written here for bf16 tensor cores:
//
//  * every row of A and of B is scaled, per group of 64 K-columns, by a power of
//    two 2^e with |x| < 2^e over the group, and its 49 leading bits are cut into
//    S = 7 slices of 7 bits: x = sum_p a_p 2^(e - 7p), a_p integer, |a_p| < 128,
//    exact in bf16;
//  * a_p b_q products are exact (< 2^14) and the FP32 sums of every pair with
//    the same weight t = p + q over a group stay below 64 * 7 * 127^2 < 2^24, so
//    the tensor-memory accumulation is exact too; the 28 pairs with t <= S + 1
//    go to 7 accumulators (one per t, 64 TMEM columns each);
//  * every group is drained: accumulator t is scaled by 2^(e_i + f_j - 7t)
//    (exact) and added to a double-float (hi + lo FP32 pair, TwoSum) register
//    accumulator, converted to FP64 once at the end.
//
// The only rounding is the truncation of each operand to 49 bits below its
// group's largest element and the double-float sum (about 2^-48 relative), so
// a product matches FP64 to about 1e-14 relative to sum |a b| while running on
// the tensor cores; the FP64 pipe only does the final conversion.
#pragma once
#include "mra_tc.cuh"

namespace mra {

constexpr int EM_S = 7;                       // slices per operand
constexpr int EM_BITS = EM_S * 7;             // 49 leading bits
constexpr int EM_KC = 32;                     // staged K chunk (bf16 elements)
constexpr int EM_KG = 64;                     // K group sharing one scale per row (drain period)
constexpr int EM_NACC = EM_S;                 // accumulators, t = 2 .. S + 1
constexpr int EM_KCORES = EM_KC / 8;          // 16-byte core columns (8 bf16) per chunk
constexpr int EM_A_HALFS = TC_M * EM_KC;      // bf16 per slice plane of A
constexpr int EM_B_HALFS = TC_N * EM_KC;
constexpr int EM_STAGE_BYTES = 2 * EM_S * (EM_A_HALFS + EM_B_HALFS);   // 86016
constexpr uint32_t EM_TMEM_COLS = 512;
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, 128 x 64.
constexpr uint32_t EM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

__device__ __forceinline__ uint64_t em_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
         ((uint64_t)(((EM_KCORES * 128u) >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ int em_cm(int row, int k) {   // bf16 index in a staged plane
  return (((row >> 3) * EM_KCORES + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// Binary exponent e with |x| < 2^e (x != 0, normal); -2000 for zero.
__device__ __forceinline__ int em_exp(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7FF);
  return be == 0 ? -2000 : be - 1022;
}

struct EmCtx {
  uint16_t* stage;   // EM_STAGE_BYTES of shared memory: 7 A planes, then 7 B planes
  int* rexp;         // TC_M row scales of A (shared)
  int* cexp;         // TC_N row scales of B (shared)
  uint64_t* mbar;
  uint32_t tmem;
  uint32_t phase;
  int* fail;
};

__device__ inline void em_init(EmCtx& cx, uint32_t* tmem_slot) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(EM_TMEM_COLS));
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

__device__ inline void em_release(EmCtx& cx) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(cx.tmem), "r"(EM_TMEM_COLS));
}

// Row scales over K columns [k0, k0 + kn <= 64) of rows [0, nx): one warp per
// row for row-major operands (coalesced along K), one thread per row otherwise.
__device__ __forceinline__ void em_scales(int* ex, int rows, const double* X, long sxi, long sxk, int nx, int k0,
                                          int kn) {
  if (sxk == 1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < rows; i += NT / 32) {
      int e = -2000;
      if (i < nx)
        for (int k = lane; k < kn; k += 32) e = max(e, em_exp(X[i * sxi + (long)(k0 + k)]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
      if (lane == 0) ex[i] = e;
    }
  } else {
    for (int i = threadIdx.x; i < rows; i += NT) {
      int e = -2000;
      if (i < nx)
        for (int k = 0; k < kn; ++k) e = max(e, em_exp(X[(long)(k0 + k) * sxk + i * sxi]));
      ex[i] = e;
    }
  }
  __syncthreads();
}

// 7 bf16 slices of x relative to scale e (|x| < 2^e) into planes[p * pstride + w].
__device__ __forceinline__ void em_split(double x, int e, uint16_t* planes, int pstride, int w) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (be != 0) {
    const int E = be - 1023;
    const unsigned long long m = (u & ((1ull << 52) - 1)) | (1ull << 52);   // x = m 2^(E - 52)
    const int sh = (52 - EM_BITS) + e - E;                                   // >= 4
    X = sh < 64 ? (m >> sh) : 0ull;                                          // x 2^(49 - e), truncated
  }
  const uint16_t sgn = (uint16_t)((u >> 48) & 0x8000u);
#pragma unroll
  for (int p = 1; p <= EM_S; ++p) {
    const unsigned a = (unsigned)((X >> (EM_BITS - 7 * p)) & 127ull);
    const uint16_t h = (uint16_t)(__float_as_uint((float)a) >> 16);          // exact: a < 128
    planes[(p - 1) * pstride + w] = (uint16_t)(h | sgn);
  }
}

__device__ __forceinline__ void em_stage(uint16_t* planes, int pstride, const int* ex, int rows, const double* X,
                                         long sxi, long sxk, int nx, int k0, int kn) {
  const int total = rows * EM_KC;
  if (sxk == 1) {
    for (int t = threadIdx.x; t < total; t += NT) {
      const int i = t / EM_KC, k = t - i * EM_KC;
      const double x = (i < nx && k < kn) ? X[i * sxi + (long)(k0 + k)] : 0.0;
      em_split(x, ex[i], planes, pstride, em_cm(i, k));
    }
  } else {
    for (int t = threadIdx.x; t < total; t += NT) {
      const int k = t / rows, i = t - k * rows;
      const double x = (i < nx && k < kn) ? X[(long)(k0 + k) * sxk + i * sxi] : 0.0;
      em_split(x, ex[i], planes, pstride, em_cm(i, k));
    }
  }
}

__device__ __forceinline__ void em_issue(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(da), "l"(db), "r"(EM_IDESC), "r"(accumulate));
}

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (v - bb);
  hi = s;
  lo += err;
}

// acc(i, j) += sum_k A(i, k) B(j, k) with FP64-grade accuracy, i < na <= 128,
// j < nb <= 64.  Returns false (uniformly) if a tensor-core wait timed out.
__device__ inline bool em_mma(EmCtx& cx, TcAcc& acc, const double* A, long sai, long sak, int na, const double* B,
                              long sbj, long sbk, int nb, int K) {
  uint16_t* aP = cx.stage;
  uint16_t* bP = cx.stage + EM_S * EM_A_HALFS;
  const int row = acc.row(), c0 = acc.col0();
  float hi[32], lo[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
  bool ok = true;
  for (int g0 = 0; g0 < K && ok; g0 += EM_KG) {
    const int gn = min(EM_KG, K - g0);
    em_scales(cx.rexp, TC_M, A, sai, sak, na, g0, gn);
    em_scales(cx.cexp, TC_N, B, sbj, sbk, nb, g0, gn);
    for (int k0 = g0; k0 < g0 + gn; k0 += EM_KC) {
      const int kn = min(EM_KC, g0 + gn - k0);
      em_stage(aP, EM_A_HALFS, cx.rexp, TC_M, A, sai, sak, na, k0, kn);
      em_stage(bP, EM_B_HALFS, cx.cexp, TC_N, B, sbj, sbk, nb, k0, kn);
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (threadIdx.x == 0) {
        for (int j = 0; j < EM_KC / 16; ++j) {
          const uint32_t off = (uint32_t)j * 256u;           // K-step of 16 bf16 = two core columns
          for (int t = 2; t <= EM_S + 1; ++t) {
            const uint32_t dt = cx.tmem + (uint32_t)(t - 2) * TC_N;
            bool first = (k0 == g0) && (j == 0);
            for (int p = max(1, t - EM_S); p <= min(EM_S, t - 1); ++p) {
              const int q = t - p;
              const uint64_t da = em_desc(smem_addr(aP + (p - 1) * EM_A_HALFS) + off);
              const uint64_t db = em_desc(smem_addr(bP + (q - 1) * EM_B_HALFS) + off);
              em_issue(dt, da, db, first ? 0u : 1u);
              first = false;
            }
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(cx.mbar)));
      }
      const bool done = tc_wait_phase(cx.mbar, cx.phase);
      if (__syncthreads_or(!done)) {
        tc_abandon(cx.mbar, cx.phase, cx.fail);
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
    if (!ok) break;
    // drain the group: accumulator t weighs 2^(e_i + f_j - 7t)
    const uint32_t lane_off = (uint32_t)((threadIdx.x >> 5) & 3) << 21;
    const int ei = cx.rexp[row];
    for (int t = 2; t <= EM_S + 1; ++t) {
      uint32_t r[32];
      const uint32_t taddr = cx.tmem + lane_off + (uint32_t)((t - 2) * TC_N + c0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int e = ei + cx.cexp[c0 + c] - 7 * t;
        const float v = __uint_as_float(r[c]);
        if (v != 0.f && e >= -126 && e <= 127) two_sum_add(hi[c], lo[c], v * __int_as_float((e + 127) << 23));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();   // scales and TMEM are reused by the next group
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) acc.v[c] += (double)hi[c] + (double)lo[c];
  return ok;
}

}  // namespace mra
