// mra_emu.cuh -- FP64-grade tile product on the tcgen05 tensor cores.
//
// GB300 retires 2 FP64 FMA per clock per SM, so FP64 contractions are emulated
// with the error-free splitting of Ozaki et al. (2012, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications"), written here for bf16 tensor cores:
//
//  * every row of A and of B is scaled, per group of 128 K-columns, by a power
//    of two 2^e with |x| < 2^e over the group, and its 49 leading bits are cut
//    into S = 7 slices of 7 bits: x = sum_p a_p 2^(e - 7p), a_p integer,
//    |a_p| < 128, exact in bf16;
//  * a_p b_q products are exact (< 2^14) and the FP32 sums of every pair with
//    the same weight t = p + q over a group stay below 128 * 7 * 127^2 < 2^24,
//    so the tensor-memory accumulation is exact too; the 28 pairs with
//    t <= S + 1 go to 7 accumulators (one per t, 64 TMEM columns each);
//  * every group is drained: the 7 accumulators of a column are combined in
//    units of the leading weight (double-float, TwoSum for the three largest
//    corrections), scaled by 2^(e_i + f_j - 14) (exact) and added to a
//    double-float register accumulator, converted to FP64 once at the end.
//
// The only rounding is the truncation of each operand to 49 bits below its
// group's largest element and the double-float sums (about 2^-48 relative), so
// a product matches FP64 to about 1e-14 relative to sum |a b| while running on
// the tensor cores; the FP64 pipe only does the final conversion.  Range: the
// running sums are FP32 pairs, so |results| < 2^127, and a group whose scale
// product 2^(e_i + f_j) is below 2^-88 is dropped (its contribution is below
// 2^-80 in absolute value).
//
// Pipeline: the K range is staged in chunks of 16 (one MMA K-step) into two
// shared-memory buffers; while the MMAs of one chunk run, the CTA splits the
// next chunk into the other buffer.  Row scales of up to four groups are found
// in one pass before the chunks that use them.
#pragma once
#include "mra_tc.cuh"

namespace mra {

constexpr int EM_S = 7;                       // slices per operand
constexpr int EM_BITS = EM_S * 7;             // 49 leading bits
constexpr int EM_KC = 16;                     // staged K chunk (bf16 elements) = one MMA K-step
constexpr int EM_KG = 128;                    // K group sharing one scale per row (drain period)
constexpr int EM_MAXG = 4;                    // groups whose scales one pass finds
constexpr int EM_CC = EM_KC / 8;              // 16-byte core columns (8 bf16) per chunk
constexpr int EM_A_HALFS = TC_M * EM_KC;      // bf16 per slice plane of A (4 KB)
constexpr int EM_B_HALFS = TC_N * EM_KC;      // (2 KB)
constexpr int EM_BUF_HALFS = EM_S * (EM_A_HALFS + EM_B_HALFS);
constexpr int EM_STAGE_BYTES = 2 * 2 * EM_BUF_HALFS;                    // two buffers: 86016
constexpr int EM_REXP = EM_MAXG * TC_M;       // ints of row scales of A (shared)
constexpr int EM_CEXP = EM_MAXG * TC_N;       // ints of row scales of B (shared)
constexpr uint32_t EM_TMEM_COLS = 512;
// The engine takes all 512 TMEM columns of an SM; its kernels ask for more than
// half of the SM's shared memory so that a second CTA is never resident (it
// would only wait in tcgen05.alloc).
constexpr size_t EM_SOLO_SMEM = 116 * 1024;
static_assert(EM_KG * EM_S * 127 * 127 < (1 << 24), "group sums must stay exact in FP32");
static_assert(EM_S * TC_N <= (int)EM_TMEM_COLS, "accumulators exceed the tensor-memory allocation");
// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, 128 x 64.
constexpr uint32_t EM_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) |
                              ((uint32_t)(TC_M >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle, K-major core matrices of 8 rows x
// 16 bytes: 128 B between K-adjacent cores, EM_CC * 128 B between 8-row groups.
__device__ __forceinline__ uint64_t em_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((128u >> 4) & 0x3FFF) << 16) |
         ((uint64_t)(((EM_CC * 128u) >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ int em_cm(int row, int k) {   // bf16 index in a staged plane
  return (((row >> 3) * EM_CC + (k >> 3)) << 6) + ((row & 7) << 3) + (k & 7);
}

// Binary exponent e with |x| < 2^e (x != 0, normal); -2000 for zero.
__device__ __forceinline__ int em_exp(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((u >> 52) & 0x7FF);
  return be == 0 ? -2000 : be - 1022;
}

struct EmCtx {
  uint16_t* stage;   // EM_STAGE_BYTES of shared memory: two buffers of 7 A planes, then 7 B planes
  int* rexp;         // EM_REXP row scales of A, [group][row], when the scale pass forms them
  int* cexp;         // EM_CEXP row scales of B
  const int* ra;     // row scales of A in use: ra[g * rs + i] (rexp or a producer's table)
  const int* cb;     // row scales of B in use: cb[g * cs + j]
  int rs, cs;
  uint64_t* mbar;    // two mbarriers, one per staging buffer
  uint32_t tmem;
  uint32_t phase;    // bit b: parity of the next completion of mbar[b] (tracked by warp 0)
  int* fail;
};

__device__ inline void em_init(EmCtx& cx, uint32_t* tmem_slot) {
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                 "r"(EM_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(cx.mbar + b)), "r"(1));
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

// Wait (bounded) for the MMAs committed to buffer b; flips b's phase once they
// completed.  Called by warp 0 only, which alone tracks the phases.
__device__ __forceinline__ bool em_poll(EmCtx& cx, int b) {
  uint32_t ph = (cx.phase >> b) & 1u;
  const bool done = tc_wait_phase(cx.mbar + b, ph);
  if (done) cx.phase ^= 1u << b;
  return done;
}

// Row scales of the groups of K columns [K0, K0 + KS), KS <= EM_MAXG * EM_KG:
// rexp[g * TC_M + i] = max exponent of row i < na of A over group g (cexp for
// B, rows < nb).  The high words of the doubles (sign, exponent, top of the
// mantissa) are brought into the idle staging buffers with asynchronous
// copies, a slab of 64 K columns of every kept row at a time, so that one
// memory latency covers a slab; one thread per row then scans its words.
constexpr int EM_SLAB = 64;                    // K columns per slab (a divisor of EM_KG)
constexpr int EM_SLAB_LD = EM_SLAB + 1;        // padded words per row in shared memory
static_assert((TC_M + TC_N) * EM_SLAB_LD * 4 <= EM_STAGE_BYTES, "slab exceeds the staging buffers");

__device__ __forceinline__ void em_cp4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ inline void em_scales(EmCtx& cx, const double* A, long sai, long sak, int na, const double* B, long sbj,
                                 long sbk, int nb, int K0, int KS) {
  uint32_t* words = reinterpret_cast<uint32_t*>(cx.stage);   // [row][EM_SLAB_LD]; rows of A, then of B
  const uint32_t wbase = smem_addr(words);
  const int rows = na + nb;                  // na (nb) = 0: that operand's scales come from its producer
  if (rows == 0) {
    __syncthreads();
    return;
  }
  for (int s0 = 0; s0 < KS; s0 += EM_SLAB) {
    const int sn = min(EM_SLAB, KS - s0);
    __syncthreads();                         // scratch (and, on the first slab, earlier scales) no longer read
    if (s0 == 0) {
      const int ng = (KS + EM_KG - 1) / EM_KG;
      for (int t = threadIdx.x; t < ng * (TC_M + TC_N); t += NT) {
        if (t < ng * TC_M) cx.rexp[t] = -2000;
        else cx.cexp[t - ng * TC_M] = -2000;
      }
    }
    // copies: along K for row-major operands, along rows otherwise (coalesced
    // either way); an operand that already lives in shared memory is read
    // directly (the asynchronous copy takes global sources only)
    for (int q = 0; q < 2; ++q) {
      const double* X = q == 0 ? A : B;
      const long si = q == 0 ? sai : sbj, sk = q == 0 ? sak : sbk;
      const int n = q == 0 ? na : nb, r0 = q == 0 ? 0 : na;
      const bool in_smem = __isShared(X);
      const int cnt = n * sn;
      for (int t = threadIdx.x; t < cnt; t += NT) {
        int i, k;
        if (sk == 1) { i = t / sn; k = t - i * sn; }
        else { k = t / n; i = t - k * n; }
        const unsigned* src = reinterpret_cast<const unsigned*>(X + (long)i * si + (long)(K0 + s0 + k) * sk) + 1;
        if (in_smem) words[(r0 + i) * EM_SLAB_LD + k] = *src;
        else em_cp4(wbase + 4u * (uint32_t)((r0 + i) * EM_SLAB_LD + k), src);
      }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int g = s0 / EM_KG;
    for (int i = threadIdx.x; i < rows; i += NT) {   // (the scanned rows are the kept ones)
      const uint32_t* wr = words + i * EM_SLAB_LD;
      int be = 0;
      for (int k = 0; k < sn; ++k) be = max(be, (int)((wr[k] >> 20) & 0x7FFu));
      if (be) {
        int* slot = i < na ? cx.rexp + g * TC_M + i : cx.cexp + g * TC_N + (i - na);
        *slot = max(*slot, be - 1022);       // one thread per row: no race
      }
    }
  }
  __syncthreads();
}

// The 49-bit magnitude window of x relative to scale e (|x| < 2^e):
// X = floor(|x| 2^(49 - e)) as h (top 17 bits) and l (low 32 bits); 0 for zero.
__device__ __forceinline__ void em_window(double x, int e, uint32_t& h, uint32_t& l) {
  const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
  const int be = (int)((hw >> 20) & 0x7FFu);
  const uint32_t mh = (hw & 0xFFFFFu) | 0x100000u;                   // mantissa = mh : lw (53 bits)
  const int sh = min(e + 1026 - be, 63);                              // >= 4 when |x| < 2^e
  const uint32_t l_lo = __funnelshift_r(lw, mh, (uint32_t)sh);        // used when sh < 32
  const uint32_t l_hi = sh < 53 ? mh >> (sh - 32 < 0 ? 0 : sh - 32) : 0u;
  l = be == 0 ? 0u : (sh < 32 ? l_lo : l_hi);
  h = (be == 0 || sh >= 32) ? 0u : mh >> sh;
}

// bf16x2 fused multiply-add: exact here (small integers).
__device__ __forceinline__ uint32_t em_hfma2(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// The 7 slice planes of a pair of elements (x0 low half, x1 high half) as
// bf16x2 words: slice p of X is the 7-bit field at bits 49 - 7 (p + 1); the two
// fields go to bits 0-6 and 16-22 of a word biased to bf16 (128 + a), and one
// bf16x2 FMA gives sg (128 + a) - 128 sg = sg a exactly.
__device__ __forceinline__ void em_split_pair(double x0, double x1, int e, uint32_t* w) {
  uint32_t h0, l0, h1, l1;
  em_window(x0, e, h0, l0);
  em_window(x1, e, h1, l1);
  const uint32_t sgn = (((uint32_t)__double2hiint(x0) >> 16) & 0x8000u) | ((uint32_t)__double2hiint(x1) & 0x80000000u);
  const uint32_t sg = 0x3F803F80u | sgn;              // (+-1, +-1) in bf16
  const uint32_t nb = 0xC300C300u ^ sgn;              // -128 sg
  const uint32_t bias = 0x43004300u;
  const uint32_t M0 = 0x7Fu, M1 = 0x7F0000u;
  // field of element 0 in bits 0-6 (t0), of element 1 in bits 16-22 (t1)
  uint32_t t0, t1;
  t0 = h0 >> 10;                        t1 = h1 << 6;                        w[0] = em_hfma2(t0 | (t1 & M1) | bias, sg, nb);
  t0 = h0 >> 3;                         t1 = h1 << 13;                       w[1] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
  t0 = __funnelshift_r(l0, h0, 28);     t1 = __funnelshift_r(l1, h1, 12);    w[2] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
  t0 = l0 >> 21;                        t1 = l1 >> 5;                        w[3] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
  t0 = l0 >> 14;                        t1 = l1 << 2;                        w[4] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
  t0 = l0 >> 7;                         t1 = l1 << 9;                        w[5] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
  t0 = l0;                              t1 = l1 << 16;                       w[6] = em_hfma2((t0 & M0) | (t1 & M1) | bias, sg, nb);
}

// The 7 slice planes of 4 consecutive K of row i, as bf16 pairs, into planes.
__device__ __forceinline__ void em_split_store(uint16_t* planes, int pstride, int e, const double* x, int i, int k4) {
  uint32_t w0[EM_S], w1[EM_S];
  em_split_pair(x[0], x[1], e, w0);
  em_split_pair(x[2], x[3], e, w1);
  const int off = em_cm(i, 4 * k4);
#pragma unroll
  for (int s = 0; s < EM_S; ++s) *reinterpret_cast<uint2*>(planes + s * pstride + off) = make_uint2(w0[s], w1[s]);
}

constexpr int EM_MAX_ITEMS = (4 * (TC_M + TC_N) + NT - 32 - 1) / (NT - 32);   // per staging thread

// Split K columns [k0, k0 + kn) (kn <= EM_KC) of rows i < na of A and j < nb of
// B into buffer b.  Rows beyond na (nb) are left as they are: they only reach
// output rows (columns) that the caller discards.  Item = half a 16-byte core
// row (4 K) of one row; the 32 lanes of a warp cover 8 rows x 2 core columns
// x 2 halves, i.e. 256 contiguous bytes per plane.  Warp 0 issues the MMAs of
// the previous chunk meanwhile, so the items go to warps 1..7.
__device__ inline void em_stage(EmCtx& cx, int b, int g, const double* A, long sai, long sak, int na,
                                const double* B, long sbj, long sbk, int nb, int k0, int kn) {
  if (threadIdx.x < 32) return;
  uint16_t* base = cx.stage + b * EM_BUF_HALFS;
  const int ia = 4 * ((na + 7) & ~7), items = ia + 4 * ((nb + 7) & ~7);
  // every load of this thread's items first, so that one memory latency
  // covers the chunk; then the splits
  double x[EM_MAX_ITEMS][4];
#pragma unroll
  for (int u = 0; u < EM_MAX_ITEMS; ++u) {
    const int it = threadIdx.x - 32 + u * (NT - 32);
    const bool isA = it < ia;
    const int jt = isA ? it : it - ia;
    const int i = ((jt >> 1) & 7) | ((jt >> 5) << 3), k4 = ((jt >> 4) & 1) * 2 + (jt & 1);
    const double* X = isA ? A : B;
    const long si = isA ? sai : sbj, sk = isA ? sak : sbk;
    const bool ok = it < items && i < (isA ? na : nb);
    const double* p = X + (long)i * si + (long)(k0 + 4 * k4) * sk;
#pragma unroll
    for (int j = 0; j < 4; ++j) x[u][j] = (ok && 4 * k4 + j < kn) ? p[(long)j * sk] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < EM_MAX_ITEMS; ++u) {
    const int it = threadIdx.x - 32 + u * (NT - 32);
    if (it >= items) break;
    const bool isA = it < ia;
    const int jt = isA ? it : it - ia;
    const int i = ((jt >> 1) & 7) | ((jt >> 5) << 3), k4 = ((jt >> 4) & 1) * 2 + (jt & 1);
    if (isA) em_split_store(base, EM_A_HALFS, cx.ra[g * cx.rs + i], x[u], i, k4);
    else em_split_store(base + EM_S * EM_A_HALFS, EM_B_HALFS, cx.cb[g * cx.cs + i], x[u], i, k4);
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

__device__ __forceinline__ void em_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// Drain the group with row scale ei and column scales cexp[c0 + c] into the
// running double-float sums (hi, lo) of this thread's 32 columns.
__device__ inline void em_drain(EmCtx& cx, const int* cexp, int ei, int c0, int na, int nb, float* hi, float* lo) {
  const int wq = (threadIdx.x >> 5) & 3;
  if (wq * 32 >= na) return;                         // warp-uniform: every row of this warp is discarded
  const uint32_t lane_off = (uint32_t)wq << 21;
#pragma unroll
  for (int cb = 0; cb < 32; cb += 8) {
    if (c0 + cb >= nb) break;                        // warp-uniform
    uint32_t v[EM_S][8];
#pragma unroll
    for (int t = 0; t < EM_S; ++t) em_ld8(cx.tmem + lane_off + (uint32_t)(t * TC_N + c0 + cb), v[t]);
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      // group value in units of 2^(e_i + f_j - 14): sum_t v_t 2^(-7 (t - 2))
      float gh = __uint_as_float(v[0][c]), gl = 0.0f;
      two_sum_add(gh, gl, __uint_as_float(v[1][c]) * 0x1p-7f);
      two_sum_add(gh, gl, __uint_as_float(v[2][c]) * 0x1p-14f);
      two_sum_add(gh, gl, __uint_as_float(v[3][c]) * 0x1p-21f);
      gl = fmaf(__uint_as_float(v[4][c]), 0x1p-28f, gl);
      gl = fmaf(__uint_as_float(v[5][c]), 0x1p-35f, gl);
      gl = fmaf(__uint_as_float(v[6][c]), 0x1p-42f, gl);
      const int e = ei + cexp[c0 + cb + c] - 14;
      if (e >= -102 && e <= 127) {
        const float s = __int_as_float((e + 127) << 23);
        two_sum_add(hi[cb + c], lo[cb + c], gh * s);
        lo[cb + c] = fmaf(gl, s, lo[cb + c]);
      }
    }
  }
}

// Issue the 28 slice-pair MMAs of one staged chunk (lane 0 of warp 0).
__device__ __forceinline__ void em_issue_chunk(const EmCtx& cx, int b, bool gfirst) {
  // plane descriptors differ only in the start-address field (addr >> 4, 14 bits; shared memory
  // addresses stay below 2^18, so the offsets below never carry out of the field)
  const uint16_t* aP = cx.stage + b * EM_BUF_HALFS;
  const uint64_t da0 = em_desc(smem_addr(aP)), db0 = em_desc(smem_addr(aP + EM_S * EM_A_HALFS));
#pragma unroll
  for (int t = 2; t <= EM_S + 1; ++t) {
    const uint32_t dt = cx.tmem + (uint32_t)(t - 2) * TC_N;
#pragma unroll
    for (int p = 1; p < t; ++p) {                 // q = t - p in [1, 7] since t <= 8
      const uint64_t da = da0 + (uint64_t)(((p - 1) * EM_A_HALFS * 2) >> 4);
      const uint64_t db = db0 + (uint64_t)(((t - p - 1) * EM_B_HALFS * 2) >> 4);
      em_issue(dt, da, db, (gfirst && p == 1) ? 0u : 1u);
    }
  }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_addr(cx.mbar + b)));
}

// Exact float -> double by bit moves (subnormal floats, below 2^-126, become 0).
__device__ __forceinline__ double em_widen(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  const uint32_t de = e == 0xFFu ? 0x7FFu : e + 896u;          // 1023 - 127
  const uint32_t hi = (u & 0x80000000u) | (de << 20) | ((u >> 3) & 0xFFFFFu);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// acc(i, j) = sum_k A(i, k) B(j, k) with FP64-grade accuracy, i < na <= 128,
// j < nb <= 64 (acc is overwritten).  Returns false (uniformly) if a
// tensor-core wait timed out.
//
// Software pipeline over the 16-column chunks of each scale pass: in step c,
// warps 1..7 split chunk c into buffer c & 1 while warp 0 issues the MMAs of
// chunk c - 1 (buffer (c - 1) & 1) and waits for them; the barrier that ends
// the step therefore leaves buffer c & 1 staged and buffer (c - 1) & 1 free.
//
// pa / pb, when not null, hold the operands' row scales from their producers:
// pa[g * pas + i] = the exponent e with |A(i, k)| < 2^e over K group g (any
// upper bound a producer can form cheaply, e.g. a maximum over a superset of
// the group's columns); the scale pass then skips that operand.
__device__ inline bool em_mma(EmCtx& cx, TcAcc& acc, const double* A, long sai, long sak, int na, const double* B,
                              long sbj, long sbk, int nb, int K, const int* pa = nullptr, int pas = 0,
                              const int* pb = nullptr, int pbs = 0) {
  const int row = acc.row(), c0 = acc.col0();
  float hi[32], lo[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) hi[c] = lo[c] = 0.f;
  for (int K0 = 0; K0 < K; K0 += EM_MAXG * EM_KG) {
    const int KS = min(EM_MAXG * EM_KG, K - K0);
    const int g0 = K0 / EM_KG;
    cx.ra = pa ? pa + g0 * pas : cx.rexp;
    cx.rs = pa ? pas : TC_M;
    cx.cb = pb ? pb + g0 * pbs : cx.cexp;
    cx.cs = pb ? pbs : TC_N;
    em_scales(cx, A, sai, sak, pa ? 0 : na, B, sbj, sbk, pb ? 0 : nb, K0, KS);
    const int nch = (KS + EM_KC - 1) / EM_KC;
    for (int c = 0; c <= nch; ++c) {
      bool done = true;
      if (threadIdx.x < 32) {
        if (c > 0) {
          if (threadIdx.x == 0) em_issue_chunk(cx, (c - 1) & 1, ((c - 1) * EM_KC) % EM_KG == 0);
          __syncwarp();
          done = em_poll(cx, (c - 1) & 1);
          asm volatile("tcgen05.fence::before_thread_sync;");
        }
      } else if (c < nch) {
        em_stage(cx, c & 1, (c * EM_KC) / EM_KG, A, sai, sak, na, B, sbj, sbk, nb, K0 + c * EM_KC,
                 min(EM_KC, KS - c * EM_KC));
        asm volatile("fence.proxy.async.shared::cta;");
      }
      if (__syncthreads_or(!done)) {                     // uniform: every thread leaves
        if (threadIdx.x == 0) *cx.fail = 1;
        if (threadIdx.x < 32) em_poll(cx, (c - 1) & 1);  // one more bounded wait for the MMAs in flight
        __syncthreads();
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int last = (c - 1) * EM_KC;                   // first column of the chunk whose MMAs completed
      if (c > 0 && ((last + EM_KC) % EM_KG == 0 || last + EM_KC >= KS)) {   // its group is complete
        const int g = last / EM_KG;
        em_drain(cx, cx.cb + g * cx.cs, row < na ? cx.ra[g * cx.rs + row] : -2000, c0, na, nb, hi, lo);
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();                                  // accumulators are read before the next group's MMAs
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
    }
  }
  // hi + lo to FP64 with one DADD: the float-to-double widening is done on the
  // integer pipe (exact bit moves), not as a conversion on the narrow FP64 pipe
  // (for every row and column: skipping the discarded ones was measured slower)
#pragma unroll
  for (int c = 0; c < 32; ++c) acc.v[c] = em_widen(hi[c]) + em_widen(lo[c]);
  return true;
}

// Row blocks of r rows stacked into one 128-row tile.
__host__ __device__ inline int em_stack(int r) { return r > 64 ? 1 : TC_M / r; }

// Tiles of the packed lower blocks (l, k), k <= l < M, stacked S high along l:
// per column block k, the diagonal tile (l = k) alone, then l = k+1.. in
// stacks of S (the leaf and prior partial sums, whose diagonal tiles take
// another operand).
__host__ __device__ inline int partial_tiles(int M, int S) {
  int n = 0;
  for (int k = 0; k < M; ++k) n += 1 + (M - 1 - k + S - 1) / S;
  return n;
}
__device__ inline bool partial_tile(int t, int M, int S, int& k, int& l0, int& nl) {
  for (k = 0; k < M; ++k) {
    const int nt = 1 + (M - 1 - k + S - 1) / S;
    if (t < nt) {
      l0 = t == 0 ? k : k + 1 + (t - 1) * S;
      nl = t == 0 ? 1 : min(S, M - l0);
      return true;
    }
    t -= nt;
  }
  return false;
}

}  // namespace mra
