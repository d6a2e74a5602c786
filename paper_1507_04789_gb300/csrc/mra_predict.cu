// mra_predict.cu -- posterior predictive mean and variance (Sec. 3.4, Prop. 2).
//
// One CTA per (leaf F, chunk of up to TILE prediction points in F).  In the
// whitened coordinates of the log-likelihood pass (xi_l = L_l' eta_l):
//   Uhat^l = (C0(S^P, Q_l) - sum_{k<l} Uhat^k V^k_{R_l}') L_l^{-T}    (U^l of Sec. 3.4, whitened)
//   v^P    = C0(s, s) - sum_{l<M} |Uhat^l row|^2                      (diag V^P, reading R4)
//   P      = L^M L_Sigma^{-T} = C0(S^P, S_F) L_Sigma^{-T} - Uhat H_F'  (L^M = v_M(S^P, S_F))
//   mean   = P z_F,  var = v^P - |P row|^2                           (the delta~ term of Prop. 2)
//   Bhat^{M,k} = Uhat^k - P H^k_F                                    (Eq. bfrecursion, definition at l = M)
//   for l = M-1..0:  Y_l = Bhat^{l+1,l} Lt_l^{-T}
//       mean += Y_l g_l,  var += |Y_l row|^2                          (the eta~ terms of Prop. 2)
//       Bhat^{l,k} -= Y_l G^k_l  for k < l                            (Eq. bfrecursion, recursion)
// since K~_l = L_l^{-T} Lt_l^{-T} Lt_l^{-1} L_l^{-1}, K~_l omega^l = L_l^{-T} Lt_l^{-T} g_l
// and K~_l A^{l,k} L_k^{-T} = L_l^{-T} Lt_l^{-T} G^k_l.
//
// The joint posterior predictive distribution of Prop. 2 (y(S^P_F) = sum_m
// B~^{m+1,m}_F eta~_m + delta~_F, eta~ shared by the leaves under a region)
// follows from the same quantities: with F_l = L_l^{-T} Lt_l^{-T} (F_l F_l' =
// K~_l), B~^{l+1,l} F_l = Y_l, so
//   Cov(s1, s2) = sum_{l: common level-l region} Y_l(s1) Y_l(s2)' + 1[same leaf] D(s1, s2),
//   D = V^P - L^M Sigma^{-1} L^M' = C0(S^P, S^P) - Uhat Uhat' - P P',
// and a draw is mean + sum_l Y_l xi_{R_l} + chol(D) zeta.  The joint modes of
// predict_kernel keep the Y_l in place of the Bhat blocks and store D (or its
// Cholesky factor) per leaf; joint_cov_kernel and simulate_kernel use them.
#include <algorithm>

#include "mra_launch.h"

namespace mra {

// MODE 0: marginal mean and variance; 1: also D and the Y_l (joint
// covariance); 2: also chol(D) and the Y_l (simulation).  In the joint modes
// one CTA holds all points of its leaf (at most TILE).  TP: the points of one
// CTA (TILE, or 16 in mode 0 where leaves hold few points): the products are
// TP x TILE tiles, the TILE columns covering the r knots of a block.
template <int TP, int TILE, int MODE>
__global__ void __launch_bounds__(NT) predict_kernel(const Desc* __restrict__ D, PredState ps, int* status) {
  static_assert(MODE == 0 || TP == TILE, "the joint modes take whole leaves in square tiles");
  extern __shared__ double smem[];
  const Desc& ds = D[ps.desc];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const int nlmax = ds.nlmax;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long F = ps.leaf0 + blockIdx.x;          // Morton id of the leaf
  const long p0 = ps.off[F] + (long)blockIdx.y * TP;
  const long p1 = min(ps.off[F + 1], p0 + TP);
  if (p0 >= p1) return;
  const int nP = (int)(p1 - p0);
  long anc[MAXL];                                // compact ids of the ancestors
  const int dM = lvl_depth(sh.hx, sh.hy, M);
  for (int l = 0; l < M; ++l) {
    anc[l] = st.cid[l][F >> (dM - lvl_depth(sh.hx, sh.hy, l))];
    if (anc[l] < 0) {                            // pruned tree: no data above this point
      if (threadIdx.x == 0) flag_error(status, ST_ARG, l, F);
      return;
    }
  }
  const long o0 = lf.off[F];
  const int nF = (int)(lf.off[F + 1] - o0);
  const int ldp = nlmax + 1, ldy = r + 1;
  const int ldc = MODE ? (nlmax > TILE ? nlmax : TILE) + 1 : ldp;   // Cs later holds D (joint modes)
  double* px = smem;
  double* py = px + TP;
  double* mu = py + TP;
  double* va = mu + TP;
  double* ax = va + TP;
  double* ay = ax + MAX_R_DEV;
  double* Cs = ay + MAX_R_DEV;                  // TP x ldc: C0(S^P, S_F), then D
  double* Ps = Cs + (long)TP * ldc;             // TP x (nlmax + 1): P
  double* Ys = Ps + (long)TP * ldp;             // TP x (r + 1)
  double* stg = Ys + (long)TP * ldy;
  for (int t = threadIdx.x; t < nP; t += NT) {
    px[t] = ps.xs[p0 + t];
    py[t] = ps.ys[p0 + t];
  }
  __syncthreads();
  double* U = ps.U + p0 * Mr;                   // nP x (M r), row-major
  TileAccR<TP, TILE> acc;
  constexpr int RR = TileAccR<TP, TILE>::RR, RC = TileAccR<TP, TILE>::RC;
  // ---- Uhat chain (same recursion as the leaf basis) --------------------------
  for (int l = 0; l < M; ++l) {
    const long a = anc[l];
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    __syncthreads();
    acc.zero();
    if (l > 0) tile_mma_r<TP, TILE>(acc, U, Mr, 1, nP, st.V[l] + a * (long)r * (l * r), l * r, 1, r, l * r, stg);
#pragma unroll
    for (int p = 0; p < RR; ++p)
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < nP && col < r) U[(long)row * Mr + l * r + col] = cov0(cv, px[row], py[row], ax[col], ay[col]) - acc.v[p][q];
      }
    __syncthreads();
    acc.zero();
    tile_mma_r<TP, TILE>(acc, U + l * r, Mr, 1, nP, st.Li[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < RR; ++p)
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < nP && col < r) U[(long)row * Mr + l * r + col] = acc.v[p][q];
      }
  }
  __syncthreads();
  // ---- prior variance v^P = C0(s, s) - |Uhat row|^2 --------------------------
  for (int t = threadIdx.x; t < nP; t += NT) {
    double s = cov0(cv, px[t], py[t], px[t], py[t]);
    for (int c = 0; c < Mr; ++c) s = fma(-U[(long)t * Mr + c], U[(long)t * Mr + c], s);
    va[t] = s;
    mu[t] = 0.0;
  }
  // ---- leaf term: P = C0(S^P, S_F) L_Sigma^{-T} - Uhat H_F' -------------------
  if (nF > 0) {
    const double* LS = lf.LS + lf.sq_off[F];
    const double* HF = lf.H + o0 * Mr;
    for (int t = threadIdx.x; t < nP * nF; t += NT) {
      int i = t / nF, k = t - i * nF;
      Cs[i * ldc + k] = cov0(cv, px[i], py[i], lf.xs[o0 + k], lf.ys[o0 + k]);
    }
    __syncthreads();
    const int nct = (nF + TILE - 1) / TILE;
    for (int ct = 0; ct < nct; ++ct) {
      const int ncol = min(TILE, nF - ct * TILE);
      acc.zero();
      tile_mma_r<TP, TILE>(acc, Cs, ldc, 1, nP, LS + (long)ct * TILE * nF, nF, 1, ncol, nF, stg);
      if (M > 0) {
        TileAccR<TP, TILE> sub;
        sub.zero();
        tile_mma_r<TP, TILE>(sub, U, Mr, 1, nP, HF + (long)ct * TILE * Mr, Mr, 1, ncol, Mr, stg);
#pragma unroll
        for (int p = 0; p < RR; ++p)
#pragma unroll
          for (int q = 0; q < RC; ++q) acc.v[p][q] -= sub.v[p][q];
      }
#pragma unroll
      for (int p = 0; p < RR; ++p)
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nP && col < ncol) Ps[row * ldp + ct * TILE + col] = acc.v[p][q];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nP; t += NT) {
      double m = 0.0, q2 = 0.0;
      for (int k = 0; k < nF; ++k) {
        double pv = Ps[t * ldp + k];
        m = fma(pv, lf.z[o0 + k], m);
        q2 = fma(pv, pv, q2);
      }
      mu[t] += m;
      va[t] -= q2;
    }
  }
  if (MODE) {
    // D = C0(S^P, S^P) - Uhat Uhat' - P P' over the leaf's points (Cs is free)
    __syncthreads();
    acc.zero();
    if (M > 0) tile_mma_r<TP, TILE>(acc, U, Mr, 1, nP, U, Mr, 1, nP, Mr, stg);
    if (nF > 0) tile_mma_r<TP, TILE>(acc, Ps, ldp, 1, nP, Ps, ldp, 1, nP, nF, stg);
#pragma unroll
    for (int p = 0; p < RR; ++p)
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < nP && col < nP) Cs[row * ldc + col] = cov0(cv, px[row], py[row], px[col], py[col]) - acc.v[p][q];
      }
    __shared__ int bad;
    if (MODE == 2) {
      if (threadIdx.x == 0) bad = 0;
      chol_smem(Cs, nP, ldc, &bad);
      if (threadIdx.x == 0 && bad) flag_error(status, ST_NOT_PD, M + 1, F);
    }
    __syncthreads();
    double* Dg = ps.D + ps.sq_off[F];
    for (int t = threadIdx.x; t < nP * nP; t += NT) {
      const int i = t / nP, j = t - i * nP;
      Dg[t] = (MODE == 2 && j > i) ? 0.0 : Cs[i * ldc + j];
    }
    for (int t = threadIdx.x; t < nP; t += NT) ps.leaf[p0 + t] = (int32_t)F;
  }
  if (nF > 0) {
    const double* HF = lf.H + o0 * Mr;
    __syncthreads();
    // Bhat^{M,k} = Uhat^k - P H^k_F  (in place in U)
    for (int k = 0; k < M; ++k) {
      acc.zero();
      tile_mma_r<TP, TILE>(acc, Ps, ldp, 1, nP, HF + k * r, 1, Mr, r, nF, stg);
#pragma unroll
      for (int p = 0; p < RR; ++p)
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nP && col < r) U[(long)row * Mr + k * r + col] -= acc.v[p][q];
        }
    }
  }
  // ---- posterior basis recursion, l = M-1..0 -----------------------------------
  for (int l = M - 1; l >= 0; --l) {
    const long a = anc[l];
    __syncthreads();
    acc.zero();
    tile_mma_r<TP, TILE>(acc, U + l * r, Mr, 1, nP, st.Lt[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < RR; ++p)
#pragma unroll
      for (int q = 0; q < RC; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < nP && col < r) Ys[row * ldy + col] = acc.v[p][q];
      }
    __syncthreads();
    const double* g = st.gv[l] + a * r;
    for (int t = threadIdx.x; t < nP; t += NT) {
      double m = 0.0, q2 = 0.0;
      for (int c = 0; c < r; ++c) {
        double yv = Ys[t * ldy + c];
        m = fma(yv, g[c], m);
        q2 = fma(yv, yv, q2);
      }
      mu[t] += m;
      va[t] += q2;
    }
    if (MODE)                                    // keep Y_l in place of block l (no longer read)
      for (int t = threadIdx.x; t < nP * r; t += NT) {
        const int i = t / r, c = t - i * r;
        U[(long)i * Mr + l * r + c] = Ys[i * ldy + c];
      }
    const double* Gl = st.G[l] + a * (long)r * (l * r);
    for (int k = 0; k < l; ++k) {
      acc.zero();
      tile_mma_r<TP, TILE>(acc, Ys, ldy, 1, nP, Gl + k * r, 1, l * r, r, r, stg);
#pragma unroll
      for (int p = 0; p < RR; ++p)
#pragma unroll
        for (int q = 0; q < RC; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nP && col < r) U[(long)row * Mr + k * r + col] -= acc.v[p][q];
        }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nP; t += NT) {
    const long orig = ps.perm[p0 + t];
    ps.mean[orig] = mu[t];
    ps.var[orig] = va[t];
  }
}

static int tile_of(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

static size_t predict_smem_tp(int tp, int r, int nlmax) {
  const int tile = tile_of(r);
  return sizeof(double) * (4 * (size_t)tp + 2 * MAX_R_DEV + 2 * (size_t)tp * (nlmax + 1) +
                           (size_t)tp * (r + 1) + KC * (tp + 2) + KC * (tile + 2));
}
size_t predict_smem_bytes(int r, int nlmax) { return predict_smem_tp(tile_of(r), r, nlmax); }

// Joint modes: one 64-point tile per leaf; Cs wide enough to hold D.
size_t joint_smem_bytes(int r, int nlmax) {
  const size_t tile = JOINT_TILE, ldc = (size_t)(nlmax > JOINT_TILE ? nlmax : JOINT_TILE) + 1;
  return sizeof(double) * (4 * tile + 2 * MAX_R_DEV + tile * ldc + tile * (nlmax + 1) + tile * (r + 1) +
                           2 * KC * (tile + 2));
}

cudaError_t launch_predict(const Desc* d_desc, int M, int r, int nlmax, const PredState& ps, int max_per_leaf,
                           int* status, cudaStream_t s, int64_t* launches, Timer* tm, long nleaf) {
  const int tile = tile_of(r);
  // points per CTA: a 16-row tile where the leaves hold few points (one TILE-wide column tile still
  // covers a block's r knots)
  const int tp = max_per_leaf <= 16 ? 16 : tile;
  const size_t sm = predict_smem_tp(tp, r, nlmax);
  dim3 grid(nleaf > 0 ? (unsigned)nleaf : (unsigned)ps.nleaves, (unsigned)((max_per_leaf + tp - 1) / tp));
  if (grid.y == 0) return cudaSuccess;
  cudaError_t e;
  tm->start(5, s);
#define MRA_PRED_LAUNCH(P, T)                                                                                 \
  {                                                                                                           \
    e = cudaFuncSetAttribute(predict_kernel<P, T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);  \
    if (e) return e;                                                                                          \
    predict_kernel<P, T, 0><<<grid, NT, sm, s>>>(d_desc, ps, status);                                         \
  }
  if (tile == 16) MRA_PRED_LAUNCH(16, 16)
  else if (tile == 32 && tp == 16) MRA_PRED_LAUNCH(16, 32)
  else if (tile == 32) MRA_PRED_LAUNCH(32, 32)
  else if (tp == 16) MRA_PRED_LAUNCH(16, 64)
  else MRA_PRED_LAUNCH(64, 64)
#undef MRA_PRED_LAUNCH
  tm->stop(s);
  ++*launches;
  return cudaGetLastError();
}

// ---- joint posterior predictive covariance ------------------------------------
// cov[perm i][perm j] = sum_{l < M: i, j share their level-l region} Y_l(i) Y_l(j)'
//                       + 1[same leaf] D(i, j), over 64 x 64 tiles of sorted points.
__global__ void __launch_bounds__(NT) joint_cov_kernel(const Desc* __restrict__ D, PredState ps, int64_t np,
                                                       double* cov) {
  __shared__ double Ya[64][MAX_R_DEV + 1], Yb[64][MAX_R_DEV + 1];
  __shared__ int32_t fa[64], fb[64];
  const Desc& ds = D[0];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r;
  const long i0 = (long)blockIdx.y * 64, j0 = (long)blockIdx.x * 64;
  const int ni = (int)min((int64_t)64, np - i0), nj = (int)min((int64_t)64, np - j0);
  for (int t = threadIdx.x; t < 64; t += NT) {
    fa[t] = t < ni ? ps.leaf[i0 + t] : -1;
    fb[t] = t < nj ? ps.leaf[j0 + t] : -2;
  }
  __syncthreads();                               // (read below even when M = 0)
  const int ti = (threadIdx.x >> 4) * 4, tj = (threadIdx.x & 15) * 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int l = 0; l < M; ++l) {
    __syncthreads();
    for (int t = threadIdx.x; t < 64 * r; t += NT) {
      const int p = t / r, c = t - p * r;
      Ya[p][c] = p < ni ? ps.U[(i0 + p) * Mr + l * r + c] : 0.0;
      Yb[p][c] = p < nj ? ps.U[(j0 + p) * Mr + l * r + c] : 0.0;
    }
    __syncthreads();
    const int sh = lvl_depth(ds.sh.hx, ds.sh.hy, M) - lvl_depth(ds.sh.hx, ds.sh.hy, l);
    bool any = false;
    bool same[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        same[a][b] = fa[ti + a] >= 0 && fb[tj + b] >= 0 && (fa[ti + a] >> sh) == (fb[tj + b] >> sh);
        any |= same[a][b];
      }
    if (!any) continue;
    for (int c = 0; c < r; ++c) {
      double xa[4], xb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xa[a] = Ya[ti + a][c];
#pragma unroll
      for (int b = 0; b < 4; ++b) xb[b] = Yb[tj + b][c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
          if (same[a][b]) acc[a][b] = fma(xa[a], xb[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = ti + a, j = tj + b;
      if (i >= ni || j >= nj) continue;
      double v = acc[a][b];
      const int32_t F = fa[i];
      if (F == fb[j]) {
        const long o = ps.off[F];
        const long nP = ps.off[F + 1] - o;
        v += ps.D[ps.sq_off[F] + (i0 + i - o) * nP + (j0 + j - o)];
      }
      cov[ps.perm[i0 + i] * np + ps.perm[j0 + j]] = v;
    }
}

// ---- conditional simulation ------------------------------------------------------
// draw[s][perm p] = mean[perm p] + sum_l Y_l(p) xi[s][(o_l + R_l) r ..] + sum_{q <= p in the leaf}
// chol(D)(p, q) zeta[s][perm q]; o_l = the regions of the complete tree's levels < l
// ((4^l - 1) / 3 for the quadtree).  One CTA
// per (leaf, chunk of 4 draws), one thread per (point, draw).
__global__ void __launch_bounds__(NT) simulate_kernel(const Desc* __restrict__ D, PredState ps, int64_t np,
                                                      int64_t nsim, int64_t nxi, const double* __restrict__ xi,
                                                      const double* __restrict__ zeta, double* draws) {
  __shared__ double xs[4][MAXL * MAX_R_DEV];
  __shared__ double zs[4][JOINT_TILE];
  const Desc& ds = D[0];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r;
  const long F = blockIdx.x;
  const long p0 = ps.off[F];
  __shared__ long o_reg[MAXL];                   // regions before level l, and the shift to the level-l id
  __shared__ int d_reg[MAXL];
  if (threadIdx.x == 0) {
    const int dM = lvl_depth(ds.sh.hx, ds.sh.hy, M);
    long o = 0;
    for (int l = 0; l < M; ++l) {
      o_reg[l] = o;
      d_reg[l] = dM - lvl_depth(ds.sh.hx, ds.sh.hy, l);
      o += 1L << lvl_depth(ds.sh.hx, ds.sh.hy, l);
    }
  }
  __syncthreads();
  const int nP = (int)(ps.off[F + 1] - p0);
  if (nP == 0) return;
  const double* Lc = ps.D + ps.sq_off[F];
  for (long s0 = (long)blockIdx.y * 4; s0 < nsim; s0 += 4L * gridDim.y) {
    __syncthreads();
    for (int t = threadIdx.x; t < 4 * Mr; t += NT) {
      const int d = t / Mr, c = t - d * Mr, l = c / r;
      const long s = s0 + d;
      const long reg = o_reg[l] + (F >> d_reg[l]);
      xs[d][c] = s < nsim ? xi[s * nxi + reg * r + (c - l * r)] : 0.0;
    }
    for (int t = threadIdx.x; t < 4 * nP; t += NT) {
      const int d = t / nP, q = t - d * nP;
      const long s = s0 + d;
      zs[d][q] = s < nsim ? zeta[s * np + ps.perm[p0 + q]] : 0.0;
    }
    __syncthreads();
    const int d = threadIdx.x / JOINT_TILE, p = threadIdx.x - d * JOINT_TILE;
    const long s = s0 + d;
    if (p < nP && s < nsim) {
      const long orig = ps.perm[p0 + p];
      double v = ps.mean[orig];
      const double* Yp = ps.U + (p0 + p) * Mr;
      for (int c = 0; c < Mr; ++c) v = fma(Yp[c], xs[d][c], v);
      for (int q = 0; q <= p; ++q) v = fma(Lc[p * nP + q], zs[d][q], v);
      draws[s * np + orig] = v;
    }
  }
}

cudaError_t launch_predict_joint(const Desc* d_desc, int M, int r, int nlmax, const PredState& ps, int mode,
                                 int* status, cudaStream_t s, int64_t* launches, Timer* tm) {
  const size_t sm = joint_smem_bytes(r, nlmax);
  dim3 grid((unsigned)ps.nleaves, 1);
  cudaError_t e;
  tm->start(5, s);
  if (mode == 1) {
    if ((e = cudaFuncSetAttribute(predict_kernel<JOINT_TILE, JOINT_TILE, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    predict_kernel<JOINT_TILE, JOINT_TILE, 1><<<grid, NT, sm, s>>>(d_desc, ps, status);
  } else {
    if ((e = cudaFuncSetAttribute(predict_kernel<JOINT_TILE, JOINT_TILE, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm)))
      return e;
    predict_kernel<JOINT_TILE, JOINT_TILE, 2><<<grid, NT, sm, s>>>(d_desc, ps, status);
  }
  tm->stop(s);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_joint_cov(const Desc* d_desc, const PredState& ps, int64_t np, double* cov, cudaStream_t s,
                             int64_t* launches) {
  const unsigned nb = (unsigned)((np + 63) / 64);
  joint_cov_kernel<<<dim3(nb, nb), NT, 0, s>>>(d_desc, ps, np, cov);
  ++*launches;
  return cudaGetLastError();
}

cudaError_t launch_simulate(const Desc* d_desc, int M, const PredState& ps, int64_t np, int64_t nsim, int64_t nxi,
                            const double* xi, const double* zeta, double* draws, cudaStream_t s, int64_t* launches) {
  const unsigned gy = (unsigned)std::min<int64_t>((nsim + 3) / 4, 64);
  simulate_kernel<<<dim3((unsigned)ps.nleaves, gy), NT, 0, s>>>(d_desc, ps, np, nsim, nxi, xi, zeta, draws);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace mra
