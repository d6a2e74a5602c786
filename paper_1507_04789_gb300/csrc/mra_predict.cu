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
#include "mra_launch.h"

namespace mra {

template <int TILE>
__global__ void __launch_bounds__(NT) predict_kernel(const Desc* __restrict__ D, PredState ps, int* status) {
  extern __shared__ double smem[];
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const int nlmax = ds.nlmax;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long F = blockIdx.x;                     // Morton id of the leaf
  const long p0 = ps.off[F] + (long)blockIdx.y * TILE;
  const long p1 = min(ps.off[F + 1], p0 + TILE);
  if (p0 >= p1) return;
  const int nP = (int)(p1 - p0);
  long anc[MAXL];                                // compact ids of the ancestors
  for (int l = 0; l < M; ++l) {
    anc[l] = st.cid[l][F >> (2 * (M - l))];
    if (anc[l] < 0) {                            // pruned tree: no data above this point
      if (threadIdx.x == 0) flag_error(status, ST_ARG, l, F);
      return;
    }
  }
  const long o0 = lf.off[F];
  const int nF = (int)(lf.off[F + 1] - o0);
  const int ldp = nlmax + 1, ldy = r + 1;
  double* px = smem;
  double* py = px + TILE;
  double* mu = py + TILE;
  double* va = mu + TILE;
  double* ax = va + TILE;
  double* ay = ax + MAX_R_DEV;
  double* Cs = ay + MAX_R_DEV;                  // TILE x (nlmax + 1): C0(S^P, S_F)
  double* Ps = Cs + (long)TILE * ldp;           // TILE x (nlmax + 1): P
  double* Ys = Ps + (long)TILE * ldp;           // TILE x (r + 1)
  double* stg = Ys + (long)TILE * ldy;
  for (int t = threadIdx.x; t < nP; t += NT) {
    px[t] = ps.xs[p0 + t];
    py[t] = ps.ys[p0 + t];
  }
  __syncthreads();
  double* U = ps.U + p0 * Mr;                   // nP x (M r), row-major
  TileAcc<TILE> acc;
  constexpr int RM = TileAcc<TILE>::RM;
  // ---- Uhat chain (same recursion as the leaf basis) --------------------------
  for (int l = 0; l < M; ++l) {
    const long a = anc[l];
    __syncthreads();
    load_knots(sh.bbox, l, st.mort[l][a], sh.gx, sh.gy, ax, ay);
    __syncthreads();
    acc.zero();
    if (l > 0) tile_mma<TILE>(acc, U, Mr, 1, nP, st.V[l] + a * (long)r * (l * r), l * r, 1, r, l * r, stg);
#pragma unroll
    for (int p = 0; p < RM; ++p)
#pragma unroll
      for (int q = 0; q < RM; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < nP && col < r) U[(long)row * Mr + l * r + col] = cov0(cv, px[row], py[row], ax[col], ay[col]) - acc.v[p][q];
      }
    __syncthreads();
    acc.zero();
    tile_mma<TILE>(acc, U + l * r, Mr, 1, nP, st.Li[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < RM; ++p)
#pragma unroll
      for (int q = 0; q < RM; ++q) {
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
      Cs[i * ldp + k] = cov0(cv, px[i], py[i], lf.xs[o0 + k], lf.ys[o0 + k]);
    }
    __syncthreads();
    const int nct = (nF + TILE - 1) / TILE;
    for (int ct = 0; ct < nct; ++ct) {
      const int ncol = min(TILE, nF - ct * TILE);
      acc.zero();
      tile_mma<TILE>(acc, Cs, ldp, 1, nP, LS + (long)ct * TILE * nF, nF, 1, ncol, nF, stg);
      if (M > 0) {
        TileAcc<TILE> sub;
        sub.zero();
        tile_mma<TILE>(sub, U, Mr, 1, nP, HF + (long)ct * TILE * Mr, Mr, 1, ncol, Mr, stg);
#pragma unroll
        for (int p = 0; p < RM; ++p)
#pragma unroll
          for (int q = 0; q < RM; ++q) acc.v[p][q] -= sub.v[p][q];
      }
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
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
    // Bhat^{M,k} = Uhat^k - P H^k_F  (in place in U)
    for (int k = 0; k < M; ++k) {
      acc.zero();
      tile_mma<TILE>(acc, Ps, ldp, 1, nP, HF + k * r, 1, Mr, r, nF, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
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
    tile_mma<TILE>(acc, U + l * r, Mr, 1, nP, st.Lt[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < RM; ++p)
#pragma unroll
      for (int q = 0; q < RM; ++q) {
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
    const double* Gl = st.G[l] + a * (long)r * (l * r);
    for (int k = 0; k < l; ++k) {
      acc.zero();
      tile_mma<TILE>(acc, Ys, ldy, 1, nP, Gl + k * r, 1, l * r, r, r, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
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

size_t predict_smem_bytes(int r, int nlmax) {
  const int tile = tile_of(r);
  return sizeof(double) * (4 * (size_t)tile + 2 * MAX_R_DEV + 2 * (size_t)tile * (nlmax + 1) +
                           (size_t)tile * (r + 1) + 2 * KC * (tile + 2));
}

cudaError_t launch_predict(const Desc* d_desc, int M, int r, int nlmax, const PredState& ps, int max_per_leaf,
                           int* status, cudaStream_t s, int64_t* launches, Timer* tm) {
  const int tile = tile_of(r);
  const size_t sm = predict_smem_bytes(r, nlmax);
  dim3 grid(1u << (2 * M), (unsigned)((max_per_leaf + tile - 1) / tile));
  if (grid.y == 0) return cudaSuccess;
  cudaError_t e;
  tm->start(5, s);
#define MRA_PRED_LAUNCH(T)                                                                              \
  {                                                                                                     \
    e = cudaFuncSetAttribute(predict_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);  \
    if (e) return e;                                                                                    \
    predict_kernel<T><<<grid, NT, sm, s>>>(d_desc, ps, status);                                         \
  }
  if (tile == 16) MRA_PRED_LAUNCH(16)
  else if (tile == 32) MRA_PRED_LAUNCH(32)
  else MRA_PRED_LAUNCH(64)
#undef MRA_PRED_LAUNCH
  tm->stop(s);
  ++*launches;
  return cudaGetLastError();
}

}  // namespace mra
