// mra_grad.cu -- reverse-mode adjoint of the M-RA log-likelihood.
//
// The gradient d loglik / d(sigma2, kappa, tau2) is not in the paper (it
// serves the likelihood-based inference of Sec. 3.3 and the maximum-likelihood
// fit of Sec. 4.3).  It is the exact reverse of the whitened forward pass of
// mra_loglik.cu, with symmetric adjoints S (d loglik = <S, dA> over the full
// symmetric matrix) for every symmetric quantity and these rules:
//   Cholesky  L = chol(A):    Abar = sym(L^{-T} Phi(L' Lbar) L^{-1}),
//             Phi = lower triangle with the diagonal halved (Murray 2016);
//   inverse   Li = L^{-1}:    Lbar = lower(-Li' Libar Li');
//   products  Y = X Li':      Xbar = Ybar Li,  Libar += lower(Ybar' X);
//   Gram      Ahat = H' H:    Hbar = 2 H S.
// The kernels run in the reverse order of the forward pass:
//   post_adjoint   m = 0..M-1  Ahat-adjoint row m and omegahat-adjoint of every
//                              region (the rows of coarser levels are owned by
//                              the ancestors, which are shared by all children)
//   leaf_adjoint   level M     Hbar, Vbar_F, the Sigma_F adjoint (C0 and tau2
//                              terms), the chain adjoint Xbar_F
//   leaf_partial   level M-1   contributions of the leaves to the adjoints of
//                              every ancestor's V and L^{-1}, summed per parent
//   prior_adjoint  m = M-1..0  a region's own V / L^{-1} adjoints from the
//                              partial sums of its children, its Cholesky
//                              adjoint, its chain adjoint, and the partial sums
//                              it passes up
//   grad_reduce                the per-CTA sums of Cbar * dC0/dtheta
// Every C0 evaluation whose adjoint Cbar is formed contributes
// sum Cbar_ij dC0_ij/dtheta, with dC0/dsigma2 = C0 / sigma2 and dC0/dkappa in
// closed form for both families.  Sums over children and rows are in a fixed
// order: the gradient is deterministic.
#include <algorithm>

#include "mra_emu.cuh"
#include "mra_launch.h"

namespace mra {

template <int TILE>
__device__ __forceinline__ void store_tile(const TileAcc<TILE>& acc, double* dst, long ld, int nr, int nc,
                                           double scale) {
#pragma unroll
  for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
    for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
      int row = acc.row(p), col = acc.col(q);
      if (row < nr && col < nc) dst[(long)row * ld + col] = scale * acc.v[p][q];
    }
}

// Phi(Y): lower triangle, halved diagonal, zero above (in place, square n).
__device__ __forceinline__ void phi_inplace(double* Y, int n, long ld) {
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int i = t / n, j = t - i * n;
    if (j > i) Y[i * ld + j] = 0.0;
    else if (j == i) Y[i * ld + j] *= 0.5;
  }
  __syncthreads();
}

__device__ __forceinline__ void lower_inplace(double* Y, int n, long ld) {
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int i = t / n, j = t - i * n;
    if (j > i) Y[i * ld + j] = 0.0;
  }
  __syncthreads();
}

// Cholesky-factor adjoint chain shared by every level:
//   given Ybar (adjoint of Li = L^{-1}, lower) in B0, L and Li (row-major n x n,
//   global or shared), diag term dlog (adjoint of each log L_ii, 0 if none):
//   Lbar = lower(-Li' Ybar Li') + dlog / L_ii;  S = sym(Li' Phi(L' Lbar) Li)
// Result S in B2 (full, symmetric).  B0, B1, B2: n x ld shared buffers.
template <int TILE>
__device__ void chol_inverse_adjoint(double* B0, double* B1, double* B2, long ld, int n, const double* L, long ldl,
                                     const double* Li, long ldi, double dlog, double* stg) {
  TileAcc<TILE> acc;
  const int nt = (n + TILE - 1) / TILE;
  // B1 = Ybar Li'
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = 0; bj < nt; ++bj) {
      acc.zero();
      tile_mma<TILE>(acc, B0 + bi * TILE * ld, ld, 1, min(TILE, n - bi * TILE), Li + bj * TILE * ldi, ldi, 1,
                     min(TILE, n - bj * TILE), n, stg);
      store_tile<TILE>(acc, B1 + bi * TILE * ld + bj * TILE, ld, min(TILE, n - bi * TILE), min(TILE, n - bj * TILE), 1.0);
    }
  __syncthreads();
  // B2 = lower(-Li' B1) + dlog / L_ii
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = 0; bj < nt; ++bj) {
      acc.zero();
      tile_mma<TILE>(acc, Li + bi * TILE, 1, ldi, min(TILE, n - bi * TILE), B1 + bj * TILE, 1, ld,
                     min(TILE, n - bj * TILE), n, stg);
      store_tile<TILE>(acc, B2 + bi * TILE * ld + bj * TILE, ld, min(TILE, n - bi * TILE), min(TILE, n - bj * TILE), -1.0);
    }
  __syncthreads();
  lower_inplace(B2, n, ld);
  if (dlog != 0.0)
    for (int t = threadIdx.x; t < n; t += NT) B2[t * ld + t] += dlog / L[t * ldl + t];
  __syncthreads();
  // B0 = Phi(L' B2)
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = 0; bj < nt; ++bj) {
      acc.zero();
      tile_mma<TILE>(acc, L + bi * TILE, 1, ldl, min(TILE, n - bi * TILE), B2 + bj * TILE, 1, ld,
                     min(TILE, n - bj * TILE), n, stg);
      store_tile<TILE>(acc, B0 + bi * TILE * ld + bj * TILE, ld, min(TILE, n - bi * TILE), min(TILE, n - bj * TILE), 1.0);
    }
  __syncthreads();
  phi_inplace(B0, n, ld);
  // B1 = B0 Li
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = 0; bj < nt; ++bj) {
      acc.zero();
      tile_mma<TILE>(acc, B0 + bi * TILE * ld, ld, 1, min(TILE, n - bi * TILE), Li + bj * TILE, 1, ldi,
                     min(TILE, n - bj * TILE), n, stg);
      store_tile<TILE>(acc, B1 + bi * TILE * ld + bj * TILE, ld, min(TILE, n - bi * TILE), min(TILE, n - bj * TILE), 1.0);
    }
  __syncthreads();
  // B2 = Li' B1, then symmetrise in place
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = 0; bj < nt; ++bj) {
      acc.zero();
      tile_mma<TILE>(acc, Li + bi * TILE, 1, ldi, min(TILE, n - bi * TILE), B1 + bj * TILE, 1, ld,
                     min(TILE, n - bj * TILE), n, stg);
      store_tile<TILE>(acc, B2 + bi * TILE * ld + bj * TILE, ld, min(TILE, n - bi * TILE), min(TILE, n - bj * TILE), 1.0);
    }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int i = t / n, j = t - i * n;
    if (j < i) {
      double v = 0.5 * (B2[i * ld + j] + B2[j * ld + i]);
      B2[i * ld + j] = v;
      B2[j * ld + i] = v;
    }
  }
  __syncthreads();
}

// The same chain with its five n x n products on the emulation engine (n <=
// 128; B0..B2 may live in global or shared memory).  Returns false (uniformly)
// if a tensor-core wait timed out; the buffers are then incomplete.
// (pa, pb: the operands' row scales from their producers, one group since n <= 128, or null)
__device__ inline bool em_store_product(EmCtx& cx, const double* A, long sai, long sak, const double* B, long sbj,
                                        long sbk, int n, double* C, long ldc, double scale,
                                        const int* pa = nullptr, const int* pb = nullptr) {
  TcAcc acc;
  const int row = acc.row(), c0 = acc.col0();
  for (int j0 = 0; j0 < n; j0 += TC_N) {
    const int nb = min(TC_N, n - j0);
    if (!em_mma(cx, acc, A, sai, sak, n, B + (long)j0 * sbj, sbj, sbk, nb, n, pa, 0, pb ? pb + j0 : nullptr, 0))
      return false;
    if (row < n) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < nb) C[(long)row * ldc + j0 + c0 + c] = scale * acc.v[c];
    }
  }
  __syncthreads();
  return true;
}

// Optional scale tables (exponents over the n rows or columns, or null): y_r
// rows of Ybar, li_r / li_c rows / columns of Li, l_c columns of L.
__device__ inline bool chol_inverse_adjoint_em(EmCtx& cx, double* B0, double* B1, double* B2, long ld, int n,
                                               const double* L, long ldl, const double* Li, long ldi, double dlog,
                                               const int* y_r = nullptr, const int* li_r = nullptr,
                                               const int* li_c = nullptr, const int* l_c = nullptr) {
  // B1 = Ybar Li'
  if (!em_store_product(cx, B0, ld, 1, Li, ldi, 1, n, B1, ld, 1.0, y_r, li_r)) return false;
  // B2 = lower(-Li' B1) + dlog / L_ii
  if (!em_store_product(cx, Li, 1, ldi, B1, 1, ld, n, B2, ld, -1.0, li_c)) return false;
  lower_inplace(B2, n, ld);
  if (dlog != 0.0)
    for (int t = threadIdx.x; t < n; t += NT) B2[t * ld + t] += dlog / L[t * ldl + t];
  __syncthreads();
  // B0 = Phi(L' B2)
  if (!em_store_product(cx, L, 1, ldl, B2, 1, ld, n, B0, ld, 1.0, l_c)) return false;
  phi_inplace(B0, n, ld);
  // B1 = B0 Li
  if (!em_store_product(cx, B0, ld, 1, Li, 1, ldi, n, B1, ld, 1.0, nullptr, li_c)) return false;
  // B2 = Li' B1, then symmetrise in place
  if (!em_store_product(cx, Li, 1, ldi, B1, 1, ld, n, B2, ld, 1.0, li_c)) return false;
  for (int t = threadIdx.x; t < n * n; t += NT) {
    int i = t / n, j = t - i * n;
    if (j < i) {
      double v = 0.5 * (B2[i * ld + j] + B2[j * ld + i]);
      B2[i * ld + j] = v;
      B2[j * ld + i] = v;
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Posterior adjoint, level m (top-down).
// ---------------------------------------------------------------------------
// EMU (launched only with gb_ready): Ltbar, the Cholesky/inverse adjoint of
// I + Ahat^{m,m} and S^{m,l} = Lti' Gbar^l / 2 on the emulation engine; a
// timeout sets status.
template <int TILE, bool EMU>
__global__ void __launch_bounds__(NT) post_adjoint_kernel(int m, const Desc* __restrict__ D, GradState gs,
                                                          int gb_ready, int* status) {
  extern __shared__ __align__(1024) double smem_all[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EMU ? EM_REXP : 1], cexp[EMU ? EM_CEXP : 1];
  double* smem = smem_all + (EMU ? EM_STAGE_BYTES / sizeof(double) : 0);
  EmCtx cx;
  bool ok = true;
  if (EMU) {
    cx.stage = reinterpret_cast<uint16_t*>(smem_all);
    cx.rexp = rexp;
    cx.cexp = cexp;
    cx.mbar = mbar;
    cx.fail = &fail;
    em_init(cx, &tmem_slot);
  }
  TcAcc ea;
  const int erow = ea.row(), ec0 = ea.col0();
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const long i = gs.rbase + blockIdx.x;
  const long ld = r + 1;
  double* wbar = smem;                       // m r: omega~ adjoint (from ancestors)
  double* gbar = wbar + MAXL * MAX_R_DEV;    // r
  double* B0 = gbar + MAX_R_DEV;
  double* B1 = B0 + MAX_R_DEV * (MAX_R_DEV + 1);
  double* B2 = B1 + MAX_R_DEV * (MAX_R_DEV + 1);
  double* stg = B2 + MAX_R_DEV * (MAX_R_DEV + 1);
  long anc[MAXL];
  for (int l = 0; l <= m; ++l) anc[l] = ancestor(st, m, i, l);
  for (int t = threadIdx.x; t < mr; t += NT) {
    int k = t / r;
    wbar[t] = gs.Obar[k][anc[k] * r + (t - k * r)];
  }
  __syncthreads();
  const double* G = st.G[m] + i * (long)r * mr;
  const double* g = st.gv[m] + i * r;
  const int T = (m + 1) * (m + 2) / 2;
  const double* A = st.Acc[m] + i * (long)T * r * r;
  // gbar = g - G omega~bar
  for (int q = threadIdx.x; q < r; q += NT) {
    double s = g[q];
    for (int c = 0; c < mr; ++c) s = fma(-G[(long)q * mr + c], wbar[c], s);
    gbar[q] = s;
  }
  // Gbar^l = -2 sum_k G^k S^{k,l} - g omega~bar^l'   -> gs.GB
  double* GB = gs.GB[m] + i * (long)r * mr;
  TileAcc<TILE> acc;
  for (int l = 0; l < m && !gb_ready; ++l) {   // (gb_ready: formed by gbar_kernel_em)
    acc.zero();
    for (int k = 0; k < m; ++k) {
      SRef b = sblock(gs, anc, r, k, l);
      tile_mma<TILE>(acc, G + k * r, mr, 1, r, b.p, b.sj, b.sk, r, r, stg);
    }
#pragma unroll
    for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
      for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < r && col < r) GB[(long)row * mr + l * r + col] = -2.0 * acc.v[p][q] - g[row] * wbar[l * r + col];
      }
  }
  __syncthreads();
  // Ltbar = sum_l Gbar^l (Ahat^{m,l})' + gbar omegahat^m'   -> B0 (lower)
  const double* om = st.Om[m] + (i * (m + 1) + m) * (long)r;
  if (EMU) {   // one product per l, summed in B0 (each thread owns its entries)
    for (int t = threadIdx.x; t < r * r; t += NT) B0[(t / r) * ld + t % r] = 0.0;
    for (int l = 0; l < m && ok; ++l) {
      ok = em_mma(cx, ea, GB + l * r, mr, 1, r, A + (long)tri_index(m, l) * r * r, r, 1, r, r);
      if (ok && erow < r) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (ec0 + c < r) B0[erow * ld + ec0 + c] += ea.v[c];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < r * r; t += NT) {
      const int row = t / r, col = t % r;
      B0[row * ld + col] = row >= col ? B0[row * ld + col] + gbar[row] * om[col] : 0.0;
    }
  } else {
    acc.zero();
    for (int l = 0; l < m; ++l)
      tile_mma<TILE>(acc, GB + l * r, mr, 1, r, A + (long)tri_index(m, l) * r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
      for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < r && col < r) B0[row * ld + col] = row >= col ? acc.v[p][q] + gbar[row] * om[col] : 0.0;
      }
  }
  __syncthreads();
  const double* Ltf = st.Ltf[m] + i * (long)r * r;   // Cholesky factor of I + Ahat^{m,m}
  const double* Lti = st.Lt[m] + i * (long)r * r;    // its inverse
  // S^{m,m} = sym(Lti' Phi(Ltf' Lbar) Lti), Lbar = lower(-Lti' Ltbar Lti') - 1 / Ltf_ii
  if (EMU) {
    if (ok) ok = chol_inverse_adjoint_em(cx, B0, B1, B2, ld, r, Ltf, r, Lti, r, -1.0);
  } else {
    chol_inverse_adjoint<TILE>(B0, B1, B2, ld, r, Ltf, r, Lti, r, -1.0, stg);
  }
  double* Ab = gs.Abar[m] + i * (long)r * (mr + r);
  for (int t = threadIdx.x; t < r * r; t += NT) {
    int a = t / r, b = t - a * r;
    Ab[(long)a * (mr + r) + mr + b] = B2[a * ld + b];
  }
  // S^{m,l} = 1/2 Lti' Gbar^l (EMU: transposed, 128/r blocks l per product)
  if (EMU) {
    const int S = em_stack(r);
    for (int l0 = 0; l0 < m && ok; l0 += S) {
      ok = em_mma(cx, ea, GB + l0 * r, 1, mr, min(S, m - l0) * r, Lti, 1, r, r, r);
      if (ok && erow < min(S, m - l0) * r) {
        const int l = l0 + erow / r, jj = erow % r;
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (ec0 + c < r) Ab[(long)(ec0 + c) * (mr + r) + l * r + jj] = 0.5 * ea.v[c];
      }
    }
  } else {
    for (int l = 0; l < m; ++l) {
      acc.zero();
      tile_mma<TILE>(acc, Lti, 1, r, r, GB + l * r, 1, mr, r, r, stg);
      store_tile<TILE>(acc, Ab + l * r, mr + r, r, r, 0.5);
    }
  }
  // omegahat^m bar = Lti' gbar
  for (int q = threadIdx.x; q < r; q += NT) {
    double s = 0.0;
    for (int c = q; c < r; ++c) s = fma(Lti[(long)c * r + q], gbar[c], s);
    gs.Obar[m][i * r + q] = s;
  }
  if (EMU) {
    em_release(cx);
    if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, m, i);
  }
}

// ---------------------------------------------------------------------------
// Leaf adjoint: one CTA per leaf.
// ---------------------------------------------------------------------------
// em_parts: bit 0, Hbar is already in HB; bit 1, the chain adjoint runs in
// chain_adjoint_kernel_em (both on the emulation engine).  EMU: the products
// LSi' Hbar, Hbar V_F' and Sigmabar V_F run on the emulation engine (its
// staging buffers open the dynamic shared memory); a timeout sets status.
template <int TILE, bool EMU>
__global__ void __launch_bounds__(NT) leaf_adjoint_kernel(const Desc* __restrict__ D, GradState gs, long slot0,
                                                           int em_parts, int* status) {
  extern __shared__ __align__(1024) double smem_all[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EMU ? EM_REXP : 1], cexp[EMU ? EM_CEXP : 1];
  // EMU: operand scales formed once per leaf (exponents, |x| < 2^e): rows of Hbar and of V_F per
  // 128-column group, their columns over the leaf's rows, the rows and columns of L_Sigma^{-1}, the
  // columns of L_Sigma, the rows of LSibar and of Sigmabar
  constexpr int ET = EMU ? 1 : 0;
  constexpr int NGMAX = (MAXL * MAX_R_DEV + EM_KG - 1) / EM_KG;   // 128-column groups of an M r row
  __shared__ int hb_r[ET ? NGMAX * TC_M : 1], vf_r[ET ? NGMAX * TC_M : 1];
  __shared__ int hb_c[ET ? MAXL * MAX_R_DEV : 1], vf_c[ET ? MAXL * MAX_R_DEV : 1];
  __shared__ int li_r[ET ? TC_M : 1], li_c[ET ? TC_M : 1], l_c[ET ? TC_M : 1], t1_r[ET ? TC_M : 1],
      t3_r[ET ? TC_M : 1];
  double* smem = smem_all + (EMU ? EM_STAGE_BYTES / sizeof(double) : 0);
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long F = gs.rbase + blockIdx.x;         // compact leaf id
  const long Fm = st.mort[M][F];
  const long o0 = lf.off[Fm];
  const int nF = (int)(lf.off[Fm + 1] - o0);
  double* wbar = smem;                      // M r
  double* zb = wbar + MAXL * MAX_R_DEV;     // nF (<= MAX_LEAF)
  double* sx = zb + 128;
  double* sy = sx + 128;
  double* ax = sy + 128;
  double* ay = ax + MAX_R_DEV;
  double* red = ay + MAX_R_DEV;
  double* stg = red + 32;
  double g_s2 = 0.0, g_k = 0.0, g_t = 0.0, g_nu = 0.0;
  EmCtx cx;
  bool ok = true;
  if (EMU) {
    cx.stage = reinterpret_cast<uint16_t*>(smem_all);
    cx.rexp = rexp;
    cx.cexp = cexp;
    cx.mbar = mbar;
    cx.fail = &fail;
    em_init(cx, &tmem_slot);
  }
  TcAcc ea;                                  // EMU: the engine's accumulator
  const int erow = ea.row(), ec0 = ea.col0();
  if (nF > 0) {
    long anc[MAXL];
    for (int l = 0; l < M; ++l) anc[l] = ancestor(st, M, F, l);
    for (int t = threadIdx.x; t < Mr; t += NT) {
      int k = t / r;
      wbar[t] = gs.Obar[k][anc[k] * r + (t - k * r)];
    }
    for (int t = threadIdx.x; t < nF; t += NT) {
      sx[t] = lf.xs[o0 + t];
      sy[t] = lf.ys[o0 + t];
    }
    __syncthreads();
    const double* H = lf.H + o0 * Mr;
    const double* VF = lf.VF + o0 * Mr;
    const double* z = lf.z + o0;
    const double* yv = lf.yv + o0;
    double* HB = gs.HB + o0 * Mr;
    double* VB = gs.VBF + o0 * Mr;
    double* XB = gs.XBF + o0 * Mr;
    const double* LSi = lf.LS + lf.sq_off[Fm];
    const double* LSf = lf.LSf + lf.sq_off[Fm];
    double* T1 = gs.T + 3 * lf.sq_off[Fm];     // three nF x nF scratch blocks per leaf
    double* T2 = T1 + (long)nF * nF;
    double* T3 = T2 + (long)nF * nF;
    const int nrt = (nF + TILE - 1) / TILE;
    TileAcc<TILE> acc;
    // Hbar = 2 H S_p + z omegabar' (already in HB when the emulated form formed it); a leaf
    // of at most 16 observations in one 16-row tile (sparse leaves: no FMA lanes on empty rows)
    if (!(em_parts & 1) && TILE > 16 && nF <= 16) {
      TileAccR<16, TILE> a16;
      for (int l = 0; l < M; ++l) {
        a16.zero();
        for (int k = 0; k < M; ++k) {
          SRef b = sblock(gs, anc, r, k, l);
          tile_mma_r<16, TILE>(a16, H + k * r, Mr, 1, nF, b.p, b.sj, b.sk, r, r, stg);
        }
#pragma unroll
        for (int p = 0; p < TileAccR<16, TILE>::RR; ++p)
#pragma unroll
          for (int q = 0; q < TileAccR<16, TILE>::RC; ++q) {
            const int row = a16.row(p), col = a16.col(q);
            if (row < nF && col < r) HB[(long)row * Mr + l * r + col] = 2.0 * a16.v[p][q] + z[row] * wbar[l * r + col];
          }
      }
    }
    for (int rt = 0; rt < nrt && !(em_parts & 1) && !(TILE > 16 && nF <= 16); ++rt) {
      const int nrow = min(TILE, nF - rt * TILE);
      for (int l = 0; l < M; ++l) {
        acc.zero();
        for (int k = 0; k < M; ++k) {
          SRef b = sblock(gs, anc, r, k, l);
          tile_mma<TILE>(acc, H + (long)rt * TILE * Mr + k * r, Mr, 1, nrow, b.p, b.sj, b.sk, r, r, stg);
        }
#pragma unroll
        for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
          for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
            int row = acc.row(p), col = acc.col(q);
            if (row < nrow && col < r) {
              int o = rt * TILE + row;
              HB[(long)o * Mr + l * r + col] = 2.0 * acc.v[p][q] + z[o] * wbar[l * r + col];
            }
          }
      }
    }
    // zbar = H omegabar - z
    for (int t = threadIdx.x; t < nF; t += NT) {
      double s = -z[t];
      for (int c = 0; c < Mr; ++c) s = fma(H[(long)t * Mr + c], wbar[c], s);
      zb[t] = s;
    }
    __syncthreads();
    if (EMU) {   // the operand scales, one pass over Hbar, V_F, L_Sigma^{-1} and L_Sigma
      const int ng = (Mr + EM_KG - 1) / EM_KG;
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int t = threadIdx.x; t < TC_M; t += NT) t1_r[t] = -2000;
      for (int o = warp; o < TC_M; o += NT / 32)   // rows per group: a warp per row
        for (int g = 0; g < ng; ++g) {
          int eh = -2000, ev = -2000;
          if (o < nF)
            for (int c = g * EM_KG + lane; c < min(Mr, (g + 1) * EM_KG); c += 32) {
              eh = max(eh, xexp_of(HB[(long)o * Mr + c]));
              ev = max(ev, xexp_of(VF[(long)o * Mr + c]));
            }
          eh = __reduce_max_sync(0xffffffffu, eh);
          ev = __reduce_max_sync(0xffffffffu, ev);
          if (lane == 0) {
            hb_r[g * TC_M + o] = eh;
            vf_r[g * TC_M + o] = ev;
          }
        }
      for (int c = threadIdx.x; c < Mr; c += NT) {   // columns over the leaf's rows: a thread per column
        int eh = -2000, ev = -2000;
        for (int o = 0; o < nF; ++o) {
          eh = max(eh, xexp_of(HB[(long)o * Mr + c]));
          ev = max(ev, xexp_of(VF[(long)o * Mr + c]));
        }
        hb_c[c] = eh;
        vf_c[c] = ev;
      }
      for (int j = threadIdx.x; j < nF; j += NT) {   // L_Sigma^{-1} (lower) and L_Sigma
        int er = -2000, ec = -2000, el = -2000;
        for (int q = 0; q < nF; ++q) {
          er = max(er, xexp_of(LSi[(long)j * nF + q]));
          ec = max(ec, xexp_of(LSi[(long)q * nF + j]));
          el = max(el, xexp_of(LSf[(long)q * nF + j]));
        }
        li_r[j] = er;
        li_c[j] = ec;
        l_c[j] = el;
      }
      __syncthreads();
    }
    // Vbar_F = LSi' Hbar
    for (int l = 0; l < M && EMU && ok; ++l) {
      ok = em_mma(cx, ea, LSi, 1, nF, nF, HB + l * r, 1, Mr, r, nF, li_c, 0, hb_c + l * r, 0);
      if (ok && erow < nF) {
        double* out = VB + (long)erow * Mr + l * r;
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (ec0 + c < r) out[ec0 + c] = ea.v[c];
      }
    }
    for (int l = 0; l < M && !EMU; ++l)
      for (int rt = 0; rt < nrt; ++rt) {
        const int nrow = min(TILE, nF - rt * TILE);
        acc.zero();
        tile_mma<TILE>(acc, LSi + rt * TILE, 1, nF, nrow, HB + l * r, 1, Mr, r, nF, stg);
        store_tile<TILE>(acc, VB + (long)rt * TILE * Mr + l * r, Mr, nrow, r, 1.0);
      }
    // LSibar = lower(Hbar V_F' + zbar y')  -> T1
    for (int j0 = 0; j0 < nF && EMU && ok; j0 += TC_N) {
      const int nb = min(TC_N, nF - j0);
      ok = em_mma(cx, ea, HB, Mr, 1, nF, VF + (long)j0 * Mr, Mr, 1, nb, Mr, hb_r, TC_M, vf_r + j0, TC_M);
      if (ok && erow < nF) {
        int e = -2000;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int j = j0 + ec0 + c;
          if (ec0 + c < nb) {
            const double v = erow >= j ? ea.v[c] + zb[erow] * yv[j] : 0.0;
            T1[(long)erow * nF + j] = v;
            e = max(e, xexp_of(v));
          }
        }
        atomicMax(t1_r + erow, e);   // rows of LSibar, the Cholesky adjoint's first operand
      }
    }
    for (int bi = 0; bi < nrt && !EMU; ++bi)
      for (int bj = 0; bj <= bi; ++bj) {
        const int ni = min(TILE, nF - bi * TILE), nj = min(TILE, nF - bj * TILE);
        acc.zero();
        tile_mma<TILE>(acc, HB + (long)bi * TILE * Mr, Mr, 1, ni, VF + (long)bj * TILE * Mr, Mr, 1, nj, Mr, stg);
#pragma unroll
        for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
          for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
            int row = acc.row(p), col = acc.col(q);
            if (row < ni && col < nj) {
              int oi = bi * TILE + row, oj = bj * TILE + col;
              T1[(long)oi * nF + oj] = oi >= oj ? acc.v[p][q] + zb[oi] * yv[oj] : 0.0;
            }
          }
        if (bj < bi) {   // zero the mirrored upper block
          for (int t = threadIdx.x; t < nj * ni; t += NT) {
            int a = t / ni, b = t - a * ni;
            T1[(long)(bj * TILE + a) * nF + bi * TILE + b] = 0.0;
          }
        }
      }
    __syncthreads();
    // Cholesky/inverse adjoint of Sigma_F in the leaf's global scratch: T3 = Sigmabar
    if (EMU) {
      if (ok) ok = chol_inverse_adjoint_em(cx, T1, T2, T3, nF, nF, LSf, nF, LSi, nF, -1.0, t1_r, li_r, li_c, l_c);
      if (ok) {   // rows of Sigmabar for the product below
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int o = warp; o < TC_M; o += NT / 32) {
          int e = -2000;
          if (o < nF)
            for (int c = lane; c < nF; c += 32) e = max(e, xexp_of(T3[(long)o * nF + c]));
          e = __reduce_max_sync(0xffffffffu, e);
          if (lane == 0) t3_r[o] = e;
        }
      }
    } else {
      chol_inverse_adjoint<TILE>(T1, T2, T3, nF, nF, LSf, nF, LSi, nF, -1.0, stg);
    }
    // T3 = Sigmabar (symmetric): C0 and tau2 terms
    for (int t = threadIdx.x; t < nF * nF; t += NT) {
      int a = t / nF, b = t - a * nF;
      double sb = T3[t];
      double d1, d2, d3;
      dcov0(cv, sx[a], sy[a], sx[b], sy[b], d1, d2, d3);
      g_s2 = fma(sb, d1, g_s2);
      g_k = fma(sb, d2, g_k);
      g_nu = fma(sb, d3, g_nu);
      if (a == b) g_t += sb;
    }
    // Vbar_F -= 2 Sigmabar V_F
    for (int l = 0; l < M && EMU && ok; ++l) {
      ok = em_mma(cx, ea, T3, nF, 1, nF, VF + l * r, 1, Mr, r, nF, t3_r, 0, vf_c + l * r, 0);
      if (ok && erow < nF) {
        double* out = VB + (long)erow * Mr + l * r;
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (ec0 + c < r) out[ec0 + c] -= 2.0 * ea.v[c];
      }
    }
    for (int l = 0; l < M && !EMU; ++l)
      for (int rt = 0; rt < nrt; ++rt) {
        const int nrow = min(TILE, nF - rt * TILE);
        acc.zero();
        tile_mma<TILE>(acc, T3 + (long)rt * TILE * nF, nF, 1, nrow, VF + l * r, 1, Mr, r, nF, stg);
#pragma unroll
        for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
          for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
            int row = acc.row(p), col = acc.col(q);
            if (row < nrow && col < r) VB[(long)(rt * TILE + row) * Mr + l * r + col] -= 2.0 * acc.v[p][q];
          }
      }
    __syncthreads();
    // chain adjoint, l = M-1..0: Xbar^l = Vbar^l Li_a ; Vbar^k -= Xbar^l V^k_a (k < l)
    for (int l = M - 1; l >= 0 && !(em_parts & 2); --l) {
      const long a = anc[l];
      const double* Lia = st.Li[l] + a * (long)r * r;
      const double* Va = st.V[l] + a * (long)r * (l * r);
      __syncthreads();
      load_knots(sh, l, st.mort[l][a], ax, ay);
      __syncthreads();
      for (int rt = 0; rt < nrt; ++rt) {
        const int nrow = min(TILE, nF - rt * TILE);
        acc.zero();
        tile_mma<TILE>(acc, VB + (long)rt * TILE * Mr + l * r, Mr, 1, nrow, Lia, 1, r, r, r, stg);
#pragma unroll
        for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
          for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
            int row = acc.row(p), col = acc.col(q);
            if (row < nrow && col < r) {
              int o = rt * TILE + row;
              double xb = acc.v[p][q];
              XB[(long)o * Mr + l * r + col] = xb;
              double d1, d2, d3;
              dcov0(cv, sx[o], sy[o], ax[col], ay[col], d1, d2, d3);
              g_s2 = fma(xb, d1, g_s2);
              g_k = fma(xb, d2, g_k);
              g_nu = fma(xb, d3, g_nu);
            }
          }
      }
      __syncthreads();
      for (int k = 0; k < l; ++k)
        for (int rt = 0; rt < nrt; ++rt) {
          const int nrow = min(TILE, nF - rt * TILE);
          acc.zero();
          tile_mma<TILE>(acc, XB + (long)rt * TILE * Mr + l * r, Mr, 1, nrow, Va + k * r, 1, l * r, r, r, stg);
#pragma unroll
          for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
            for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
              int row = acc.row(p), col = acc.col(q);
              if (row < nrow && col < r) VB[(long)(rt * TILE + row) * Mr + k * r + col] -= acc.v[p][q];
            }
        }
    }
  }
  if (EMU) em_release(cx);
  g_s2 = block_sum(g_s2, red);
  g_k = block_sum(g_k, red);
  g_t = block_sum(g_t, red);
  g_nu = block_sum(g_nu, red);
  if (EMU && !ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M, F);
  if (threadIdx.x == 0) {
    gs.gpart[GP * (slot0 + F) + 0] = g_s2;
    gs.gpart[GP * (slot0 + F) + 1] = g_k;
    gs.gpart[GP * (slot0 + F) + 2] = g_t;
    gs.gpart[GP * (slot0 + F) + 3] = g_nu;
  }
}

// ---------------------------------------------------------------------------
// Leaf partials: parent p (level M-1), packed tile t = (l, k), k <= l <= M-1:
//   k < l : -sum_rows Xbar^l' V^k      (adjoint of V^k of the level-l ancestor)
//   k = l :  sum_rows Vbar^l' V^l      (times L_l' at the ancestor: adjoint of L_l^{-1})
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(NT) leaf_partial_kernel(const Desc* __restrict__ D, GradState gs) {
  extern __shared__ double smem[];
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long p = gs.rbase + blockIdx.x;         // compact id at level M-1
  const long pm = ds.st.mort[M - 1][p];
  const int t = blockIdx.y;
  int l = 0;
  while (tri_index(l + 1, 0) <= t) ++l;
  const int k = t - tri_index(l, 0);
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const int K = (int)(row1 - row0);
  const double* Ab = (k < l ? gs.XBF : gs.VBF) + row0 * Mr + l * r;
  const double* Bb = lf.VF + row0 * Mr + k * r;
  TileAcc<TILE> acc;
  acc.zero();
  tile_mma<TILE>(acc, Ab, 1, Mr, r, Bb, 1, Mr, r, K, smem);
  const int T = M * (M + 1) / 2;
  store_tile<TILE>(acc, gs.PartLeaf + (p * T + t) * (long)r * r, r, r, r, k < l ? -1.0 : 1.0);
}

// ---------------------------------------------------------------------------
// Prior adjoint, level m (bottom-up): one CTA per region.
// ---------------------------------------------------------------------------
// EMU: every r x r x r product (and the Cholesky/inverse adjoint) runs on the
// emulation engine, whose staging buffers open the dynamic shared memory; a
// timeout sets status.
template <int TILE, bool EMU>
__global__ void __launch_bounds__(NT) prior_adjoint_kernel(int m, const Desc* __restrict__ D, GradState gs,
                                                           long slot0, int* status) {
  extern __shared__ __align__(1024) double smem_all[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EMU ? EM_REXP : 1], cexp[EMU ? EM_CEXP : 1];
  double* smem = smem_all + (EMU ? EM_STAGE_BYTES / sizeof(double) : 0);
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const long i = gs.rbase + blockIdx.x;
  const long ld = r + 1;
  double* qx = smem;
  double* qy = qx + MAX_R_DEV;
  double* ax = qy + MAX_R_DEV;
  double* ay = ax + MAX_R_DEV;
  double* red = ay + MAX_R_DEV;
  double* B0 = red + 32;
  double* B1 = B0 + MAX_R_DEV * (MAX_R_DEV + 1);
  double* B2 = B1 + MAX_R_DEV * (MAX_R_DEV + 1);
  double* stg = B2 + MAX_R_DEV * (MAX_R_DEV + 1);
  const bool from_leaves = (m + 1 == sh.M);
  const int Tin = (m + 1) * (m + 2) / 2;   // incoming tiles, l <= m
  const long cf = from_leaves ? 0 : st.cfirst[m][i], cc = from_leaves ? 0 : st.ccnt[m][i];
  // incoming tile (l, k): sum over the active children (fixed order)
  auto incoming = [&](int l, int k, int a, int b) -> double {
    const long t = tri_index(l, k);
    if (from_leaves) return gs.PartLeaf[(i * Tin + t) * (long)r * r + a * r + b];
    double s = 0.0;
    for (long c = cf; c < cf + cc; ++c) s += gs.Up[m + 1][(c * Tin + t) * (long)r * r + a * r + b];
    return s;
  };
  EmCtx cx;
  bool ok = true;
  if (EMU) {
    cx.stage = reinterpret_cast<uint16_t*>(smem_all);
    cx.rexp = rexp;
    cx.cexp = cexp;
    cx.mbar = mbar;
    cx.fail = &fail;
    em_init(cx, &tmem_slot);
  }
  TileAcc<TILE> acc;
  TcAcc ea;
  // f(i, j, P(i, j)) for the r x r product P(i, j) = sum_{c < kk} A(i, c) B(j, c)
  auto product = [&](const double* A, long sai, long sak, const double* B, long sbj, long sbk, int kk, auto&& f) {
    if constexpr (EMU) {
      if (ok) ok = em_mma(cx, ea, A, sai, sak, r, B, sbj, sbk, r, kk);
      const int row = ea.row(), c0 = ea.col0();
      if (ok && row < r) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c0 + c < r) f(row, c0 + c, ea.v[c]);
      }
    } else {
      acc.zero();
      tile_mma<TILE>(acc, A, sai, sak, r, B, sbj, sbk, r, kk, stg);
#pragma unroll
      for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
        for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
          const int row = acc.row(p), col = acc.col(q);
          if (row < r && col < r) f(row, col, acc.v[p][q]);
        }
    }
  };
  // EMU: f(i, j, P(i, j)) for P(i, j) = sum_{c < kk} A(i, c) B(j, c), i < na <= 128 (stacked
  // row blocks), j < r
  // (pa, pb: the operands' row scales from their producers, one group since kk = r, or null)
  auto product_n = [&](const double* A, long sai, long sak, int na, const double* B, long sbj, long sbk, int kk,
                       const int* pa, const int* pb, auto&& f) {
    if (ok) ok = em_mma(cx, ea, A, sai, sak, na, B, sbj, sbk, r, kk, pa, 0, pb, 0);
    const int row = ea.row(), c0 = ea.col0();
    if (ok && row < na) {
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < r) f(row, c0 + c, ea.v[c]);
    }
  };
  const int S = em_stack(r);
  double g_s2 = 0.0, g_k = 0.0, g_nu = 0.0;
  load_knots(sh, m, st.mort[m][i], qx, qy);
  const double* L = st.L[m] + i * (long)r * r;
  const double* Li = st.Li[m] + i * (long)r * r;
  const double* V = st.V[m] + i * (long)r * mr;
  // Libar = lower(incoming(m, m) L')  -> B0   (the adjoint of L^{-1} gathered from the subtree)
  for (int t = threadIdx.x; t < r * r; t += NT) {
    int a = t / r, b = t - a * r;
    B1[a * ld + b] = incoming(m, m, a, b);
  }
  __syncthreads();
  product(B1, ld, 1, L, r, 1, r, [&](int row, int col, double v) { B0[row * ld + col] = row >= col ? v : 0.0; });
  __syncthreads();
  if (EMU) {
    if (ok) ok = chol_inverse_adjoint_em(cx, B0, B1, B2, ld, r, L, r, Li, r, 0.0);   // B2 = Wbar
  } else {
    chol_inverse_adjoint<TILE>(B0, B1, B2, ld, r, L, r, Li, r, 0.0, stg);
  }
  for (int t = threadIdx.x; t < r * r; t += NT) {
    int a = t / r, b = t - a * r;
    double d1, d2, d3;
    dcov0(cv, qx[a], qy[a], qx[b], qy[b], d1, d2, d3);
    g_s2 = fma(B2[a * ld + b], d1, g_s2);
    g_k = fma(B2[a * ld + b], d2, g_k);
    g_nu = fma(B2[a * ld + b], d3, g_nu);
  }
  double* VB = gs.VB[m] + i * (long)r * mr;
  double* XB = gs.XB[m] + i * (long)r * mr;
  // Vbar^k = incoming(m, k) - 2 Wbar V^k (EMU: transposed, S blocks k per product: the
  // columns of V are contiguous across its blocks)
  if (EMU) {
    for (int k0 = 0; k0 < m; k0 += S)
      product_n(V + k0 * r, 1, mr, min(S, m - k0) * r, B2, ld, 1, r,
                st.vcol[m] ? st.vcol[m] + i * (long)mr + k0 * r : nullptr, nullptr, [&](int ii, int row, double v) {
        const int k = k0 + ii / r, col = ii % r;
        VB[(long)row * mr + k * r + col] = incoming(m, k, row, col) - 2.0 * v;
      });
  } else {
    for (int k = 0; k < m; ++k)
      product(B2, ld, 1, V + k * r, 1, mr, r, [&](int row, int col, double v) {
        VB[(long)row * mr + k * r + col] = incoming(m, k, row, col) - 2.0 * v;
      });
  }
  // chain adjoint
  for (int l = m - 1; l >= 0; --l) {
    const long a = ancestor(st, m, i, l);
    const double* Lia = st.Li[l] + a * (long)r * r;
    const double* Va = st.V[l] + a * (long)r * (l * r);
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    __syncthreads();
    auto xbar_epi = [&](int row, int col, double xb) {
      XB[(long)row * mr + l * r + col] = xb;
      double d1, d2, d3;
      dcov0(cv, qx[row], qy[row], ax[col], ay[col], d1, d2, d3);
      g_s2 = fma(xb, d1, g_s2);
      g_k = fma(xb, d2, g_k);
      g_nu = fma(xb, d3, g_nu);
    };
    if (EMU)
      product_n(VB + l * r, mr, 1, r, Lia, 1, r, r, nullptr, st.licol[l] ? st.licol[l] + a * r : nullptr, xbar_epi);
    else
      product(VB + l * r, mr, 1, Lia, 1, r, r, xbar_epi);
    __syncthreads();
    if (EMU) {   // Vbar^k -= Xbar^l V^k_a, transposed, S blocks k per product
      for (int k0 = 0; k0 < l; k0 += S)
        product_n(Va + k0 * r, 1, l * r, min(S, l - k0) * r, XB + l * r, mr, 1, r,
                  st.vcol[l] ? st.vcol[l] + a * (long)(l * r) + k0 * r : nullptr, nullptr,
                  [&](int ii, int row, double v) {
          VB[(long)row * mr + (k0 + ii / r) * r + ii % r] -= v;
        });
    } else {
      for (int k = 0; k < l; ++k)
        product(XB + l * r, mr, 1, Va + k * r, 1, l * r, r,
                [&](int row, int col, double v) { VB[(long)row * mr + k * r + col] -= v; });
    }
  }
  __syncthreads();
  // partial sums passed up: tiles (l, k), k <= l < m
  if (m > 0) {
    const int Tup = m * (m + 1) / 2;
    double* Up = gs.Up[m] + i * (long)Tup * r * r;
    if (EMU) {   // tiles (l0.., k) stacked S high (diagonal tiles alone: their operand is Vbar)
      for (int t = 0; t < partial_tiles(m, S); ++t) {
        int k, l0, nl;
        partial_tile(t, m, S, k, l0, nl);
        const double* Ab = (l0 == k ? VB : XB) + l0 * r;
        const double sgn = l0 == k ? 1.0 : -1.0;
        product_n(Ab, 1, mr, nl * r, V + k * r, 1, mr, r, nullptr,
                  st.vcol[m] ? st.vcol[m] + i * (long)mr + k * r : nullptr, [&](int ii, int col, double v) {
          const int l = l0 + ii / r, row = ii % r;
          Up[(long)tri_index(l, k) * r * r + row * r + col] = incoming(l, k, row, col) + sgn * v;
        });
      }
    }
    for (int l = 0; l < m && !EMU; ++l)
      for (int k = 0; k <= l; ++k) {
        const double* Ab = (k < l ? XB : VB) + l * r;
        double* out = Up + (long)tri_index(l, k) * r * r;
        const double sgn = k < l ? -1.0 : 1.0;
        product(Ab, 1, mr, V + k * r, 1, mr, r,
                [&](int row, int col, double v) { out[row * r + col] = incoming(l, k, row, col) + sgn * v; });
      }
  }
  if (EMU) em_release(cx);
  g_s2 = block_sum(g_s2, red);
  g_k = block_sum(g_k, red);
  g_nu = block_sum(g_nu, red);
  if (threadIdx.x == 0) {
    gs.gpart[GP * (slot0 + i) + 0] = g_s2;
    gs.gpart[GP * (slot0 + i) + 1] = g_k;
    gs.gpart[GP * (slot0 + i) + 2] = 0.0;
    gs.gpart[GP * (slot0 + i) + 3] = g_nu;
    if (EMU && !ok) flag_error(status, ST_TIMEOUT, m, i);
  }
}

// Emulated form: column exponents of every region's L^{-1} and V at level m
// (the right operands of the chain adjoints), one CTA per region.
__global__ void __launch_bounds__(NT) col_scales_kernel(int m, const Desc* __restrict__ D, long rbase) {
  const Desc& ds = D[0];
  const LevelState& st = ds.st;
  const int r = ds.sh.r, mr = m * r;
  const long i = rbase + blockIdx.x;
  const double* Li = st.Li[m] + i * (long)r * r;
  const double* V = st.V[m] + i * (long)r * mr;
  for (int c = threadIdx.x; c < r + mr; c += NT) {
    int e = -2000;
    if (c < r)
      for (int a = 0; a < r; ++a) e = max(e, xexp_of(Li[(long)a * r + c]));
    else
      for (int a = 0; a < r; ++a) e = max(e, xexp_of(V[(long)a * mr + c - r]));
    if (c < r) st.licol[m][i * r + c] = e;
    else st.vcol[m][i * (long)mr + c - r] = e;
  }
}

// Sum of the per-CTA partial gradients (fixed assignment: deterministic).
__global__ void __launch_bounds__(NT) grad_reduce_kernel(const double* gpart, long nslots, double* out) {
  __shared__ double red[32];
  for (int c = 0; c < GP; ++c) {
    double s = 0.0;
    for (long t = threadIdx.x; t < nslots; t += NT) s += gpart[GP * t + c];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[c] = s;
  }
}

// ---------------------------------------------------------------------------
static int tile_of(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

#define MRA_GRAD_LAUNCH(tile, KERNEL, grid, smem, stream, ...)                                          \
  do {                                                                                                  \
    if ((tile) == 16) {                                                                                 \
      if ((e = cudaFuncSetAttribute(KERNEL<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem)))) return e; \
      KERNEL<16><<<grid, NT, smem, stream>>>(__VA_ARGS__);                                              \
    } else if ((tile) == 32) {                                                                          \
      if ((e = cudaFuncSetAttribute(KERNEL<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem)))) return e; \
      KERNEL<32><<<grid, NT, smem, stream>>>(__VA_ARGS__);                                              \
    } else {                                                                                            \
      if ((e = cudaFuncSetAttribute(KERNEL<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem)))) return e; \
      KERNEL<64><<<grid, NT, smem, stream>>>(__VA_ARGS__);                                              \
    }                                                                                                   \
  } while (0)

template <bool EMU>
static cudaError_t launch_leaf_adjoint(int tile, int nleaves, size_t sm, cudaStream_t s, const Desc* d_desc,
                                       const GradState& gs, long slot0, int em_parts, int* status) {
  cudaError_t e;
#define MRA_LEAF_ADJ(T)                                                                                       \
  if ((e = cudaFuncSetAttribute(leaf_adjoint_kernel<T, EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                (int)sm)))                                                                    \
    return e;                                                                                                 \
  leaf_adjoint_kernel<T, EMU><<<nleaves, NT, sm, s>>>(d_desc, gs, slot0, em_parts, status);
  if constexpr (EMU) {   // the emulated instances use 64-wide FP64 tiles only (fewer instantiations)
    MRA_LEAF_ADJ(64)
  } else {
    if (tile == 64) {
      MRA_LEAF_ADJ(64)
    } else if (tile == 32) {
      MRA_LEAF_ADJ(32)
    } else {
      MRA_LEAF_ADJ(16)
    }
  }
#undef MRA_LEAF_ADJ
  return cudaGetLastError();
}

template <bool EMU>
static cudaError_t launch_post_adjoint(int tile, int m, int nregions, size_t sm, cudaStream_t s, const Desc* d_desc,
                                       const GradState& gs, int gb_ready, int* status) {
  cudaError_t e;
#define MRA_POST_ADJ(T)                                                                                       \
  if ((e = cudaFuncSetAttribute(post_adjoint_kernel<T, EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                (int)sm)))                                                                    \
    return e;                                                                                                 \
  post_adjoint_kernel<T, EMU><<<nregions, NT, sm, s>>>(m, d_desc, gs, gb_ready, status);
  if constexpr (EMU) {   // the emulated instances use 64-wide FP64 tiles only (fewer instantiations)
    MRA_POST_ADJ(64)
  } else {
    if (tile == 64) {
      MRA_POST_ADJ(64)
    } else if (tile == 32) {
      MRA_POST_ADJ(32)
    } else {
      MRA_POST_ADJ(16)
    }
  }
#undef MRA_POST_ADJ
  return cudaGetLastError();
}

template <bool EMU>
static cudaError_t launch_prior_adjoint(int tile, int m, int nregions, size_t sm, cudaStream_t s,
                                        const Desc* d_desc, const GradState& gs, long slot0, int* status) {
  cudaError_t e;
#define MRA_PRIOR_ADJ(T)                                                                                      \
  if ((e = cudaFuncSetAttribute(prior_adjoint_kernel<T, EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                (int)sm)))                                                                    \
    return e;                                                                                                 \
  prior_adjoint_kernel<T, EMU><<<nregions, NT, sm, s>>>(m, d_desc, gs, slot0, status);
  if constexpr (EMU) {   // the emulated instances use 64-wide FP64 tiles only (fewer instantiations)
    MRA_PRIOR_ADJ(64)
  } else {
    if (tile == 64) {
      MRA_PRIOR_ADJ(64)
    } else if (tile == 32) {
      MRA_PRIOR_ADJ(32)
    } else {
      MRA_PRIOR_ADJ(16)
    }
  }
#undef MRA_PRIOR_ADJ
  return cudaGetLastError();
}

// Slots of the per-CTA gradient partials: the prior-adjoint CTAs of levels
// 0..M-1, then the leaves, then one per level-(M-1) region for the emulated
// chain adjoint.
static long slot_of_level(const LevelState& st, int m) {
  long s = 0;
  for (int l = 0; l < m; ++l) s += st.nreg[l];
  return s;
}

// The per-parent S buffer seen from the parents [base, ...) of a range whose S
// rows are (w x w) blocks, w = (parent level + 1) r: the range's first parent
// lands at the buffer's start.
static void local_s(GradState& g, long base, long w) {
  const long ng = (w + EM_KG - 1) / EM_KG;
  g.SF = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(g.SF) - (uintptr_t)(base * w * w * (long)sizeof(double)));
  g.SFexp = reinterpret_cast<int32_t*>(reinterpret_cast<uintptr_t>(g.SFexp) -
                                       (uintptr_t)(base * ng * w * (long)sizeof(int32_t)));
}

cudaError_t launch_grad_range(const Desc& hd, const Desc* d_desc, GradState gs, const GradRange& R, int* status,
                              cudaStream_t s, int64_t* launches) {
  const int tile = tile_of(hd.sh.r);
  const int M = hd.sh.M;
  const LevelState& st = hd.st;
  cudaError_t e;
  const size_t stg = sizeof(double) * 2 * KC * (tile + 2);
  const size_t sq = sizeof(double) * 3 * MAX_R_DEV * (MAX_R_DEV + 1);
  const int post_hi = R.post_hi < 0 ? M : R.post_hi, prior_hi = R.prior_hi < 0 ? M : R.prior_hi;
  auto base = [&](int m) { return R.count[m] < 0 ? 0L : R.base[m]; };
  auto count = [&](int m) { return R.count[m] < 0 ? (long)st.nreg[m] : R.count[m]; };
  const long slot_leaf = slot_of_level(st, M);
  const bool emu = hd.sh.mixed == 2 && M > 0;
  if (emu && st.licol[0]) {   // column scales of L^{-1} and V for the emulated chain adjoints
    const int cs_lo = R.cs_lo < 0 ? R.prior_lo : R.cs_lo;
    const int cs_hi = R.cs_lo < 0 ? prior_hi : (R.cs_hi < 0 ? M : R.cs_hi);
    for (int m = cs_lo; m < cs_hi; ++m) {
      if (count(m) == 0) continue;
      col_scales_kernel<<<(unsigned)count(m), NT, 0, s>>>(m, d_desc, base(m));
      ++*launches;
    }
    if ((e = cudaGetLastError())) return e;
  }
  for (int m = R.post_lo; m < post_hi; ++m) {
    if (count(m) == 0) continue;
    gs.rbase = base(m);
    // emulated form with the per-region S buffer: Gbar on the tensor cores first
    const int gb_ready = emu && gs.SF != nullptr && m > 0;
    if (gb_ready) {   // (over the level-(m-1) parents)
      GradState gp = gs;
      gp.rbase = base(m - 1);
      if (R.local_sf) local_s(gp, base(m - 1), (long)m * hd.sh.r);
      if ((e = launch_gbar_em(m, hd, d_desc, gp, status, s, launches, count(m - 1)))) return e;
    }
    const size_t sm = sizeof(double) * (MAXL * MAX_R_DEV + MAX_R_DEV) + sq;
    if (gb_ready) e = launch_post_adjoint<true>(tile, m, (int)count(m), std::max(sm + EM_STAGE_BYTES, EM_SOLO_SMEM), s,
                                                d_desc, gs, gb_ready, status);
    else e = launch_post_adjoint<false>(tile, m, (int)count(m), sm + stg, s, d_desc, gs, gb_ready, status);
    if (e) return e;
    ++*launches;
  }
  const int em_parts = (emu && gs.SF != nullptr ? 1 : 0) | (emu ? 2 : 0);
  if (R.leaves) {
    // emulated form: Hbar on the tensor cores (when its per-parent S was allocated)
    gs.rbase = M > 0 ? base(M - 1) : 0;
    if (em_parts & 1) {
      GradState gh = gs;
      if (R.local_sf) local_s(gh, base(M - 1), (long)M * hd.sh.r);
      if ((e = launch_hbar_em(hd, d_desc, gh, status, s, launches, count(M - 1)))) return e;
    }
    gs.rbase = base(M);
    size_t sm = sizeof(double) * (MAXL * MAX_R_DEV + 3 * 128 + 2 * MAX_R_DEV + 32) + stg;
    if (emu) {   // (the emulated instance's FP64 tiles are 64 wide: its staging sized for them)
      sm += EM_STAGE_BYTES + sizeof(double) * 2 * KC * (64 + 2) - stg;
      if (sm < EM_SOLO_SMEM) sm = EM_SOLO_SMEM;
      e = launch_leaf_adjoint<true>(tile, (int)count(M), sm, s, d_desc, gs, slot_leaf, em_parts, status);
    } else {
      e = launch_leaf_adjoint<false>(tile, (int)count(M), sm, s, d_desc, gs, slot_leaf, em_parts, status);
    }
    if (e) return e;
    ++*launches;
    // slots after the leaves': the emulated chain adjoint's, one per level-(M-1) region
    const long slot_chain = slot_leaf + st.nreg[M];
    gs.rbase = M > 0 ? base(M - 1) : 0;
    if (em_parts & 2) {
      if ((e = launch_chain_adjoint_em(hd, d_desc, gs, slot_chain, status, s, count(M - 1)))) return e;
      ++*launches;
    }
    if (M > 0 && hd.sh.mixed == 2) {
      if ((e = launch_leaf_partial_em(hd, d_desc, gs, status, s, count(M - 1)))) return e;
      ++*launches;
    } else if (M > 0) {
      dim3 grid((unsigned)count(M - 1), M * (M + 1) / 2);
      MRA_GRAD_LAUNCH(tile, leaf_partial_kernel, grid, stg, s, d_desc, gs);
      ++*launches;
    }
  }
  for (int m = prior_hi - 1; m >= R.prior_lo; --m) {
    if (count(m) == 0) continue;
    gs.rbase = base(m);
    const long slot = slot_of_level(st, m);
    const size_t sm = sizeof(double) * (4 * MAX_R_DEV + 32) + sq;
    if (emu) e = launch_prior_adjoint<true>(tile, m, (int)count(m), std::max(sm + EM_STAGE_BYTES, EM_SOLO_SMEM), s,
                                            d_desc, gs, slot, status);
    else e = launch_prior_adjoint<false>(tile, m, (int)count(m), sm + stg, s, d_desc, gs, slot, status);
    if (e) return e;
    ++*launches;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const Desc& hd, const GradState& gs, double* grad_out_dev, cudaStream_t s,
                               int64_t* launches) {
  const int M = hd.sh.M;
  const bool emu = hd.sh.mixed == 2 && M > 0;
  const long nslots = slot_of_level(hd.st, M) + hd.st.nreg[M] + (emu ? hd.st.nreg[M - 1] : 0);
  grad_reduce_kernel<<<1, NT, 0, s>>>(gs.gpart, nslots, grad_out_dev);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_grad(const Desc& hd, const Desc* d_desc, const GradState& gs, double* grad_out_dev, int* status,
                        cudaStream_t s, int64_t* launches, Timer* tm) {
  GradRange all;
  tm->start(6, s);
  cudaError_t e = launch_grad_range(hd, d_desc, gs, all, status, s, launches);
  if (!e) e = launch_grad_reduce(hd, gs, grad_out_dev, s, launches);
  tm->stop(s);
  return e;
}

}  // namespace mra
