// mra_loglik.cu -- prior pass, leaf pass and posterior pass of the M-RA
// log-likelihood (Sec. 3.1-3.3) in FP64, one CTA per region per level.
//
// Level kernels, in launch order for one evaluation:
//   prior_level  m = 0..M-1  Eq. (priorw) in block-Cholesky form: V^l_R, L_R^{-1}
//   leaf         (level M)   B^l, Sigma_F + tau2 I (Sec. 4.3), its Cholesky factor,
//                            H = L_Sigma^{-1} V_F, z = L_Sigma^{-1} y, d_F, u_F
//   leaf_syrk    (level M-1) Ahat = sum_children H' H, omegahat = sum H' z
//                            (Eq. helpquantities from the definition at m = M,
//                            summed over children as in Eq. mainquantities)
//   post_level   m = M-1..0  Cholesky of I + Ahat^{m,m}, G, g, d_R, u_R (Sec. 3.3)
//   aggregate    m = M-1..1  Atilde = Ahat - G' G summed into the parent (Eqs.
//                            mainquantities, helpquantities), omega likewise
#include "mra_emu.cuh"
#include "mra_kernels.cuh"
#include "mra_launch.h"

namespace mra {

// ---------------------------------------------------------------------------
// Prior pass, level m: region i computes its block row of the chain factor.
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(NT) prior_level_kernel(int m, const Desc* __restrict__ D,
                                                         const int2* __restrict__ work, int* status) {
  extern __shared__ double smem[];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const long i = it.i;
  double* qx = smem;                 // own knots
  double* qy = qx + MAX_R_DEV;
  double* ax = qy + MAX_R_DEV;       // ancestor knots
  double* ay = ax + MAX_R_DEV;
  double* tmp = ay + MAX_R_DEV;
  double* red = tmp + MAX_R_DEV;
  double* W = red + 32;              // r x (r + 1)
  double* stg = W + MAX_R_DEV * (MAX_R_DEV + 1);
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  load_knots(sh, m, st.mort[m][i], qx, qy);
  double* Vrow = st.V[m] + i * (long)r * mr;
  TileAcc<TILE> acc;
  for (int l = 0; l < m; ++l) {
    const long a = ancestor(st, m, i, l);
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    acc.zero();
    if (l > 0) tile_mma<TILE>(acc, Vrow, mr, 1, r, Vanc, l * r, 1, r, l * r, stg);
    __syncthreads();
#pragma unroll
    for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
      for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < r && col < r)
          Vrow[(long)row * mr + l * r + col] = cov0(cv, qx[row], qy[row], ax[col], ay[col]) - acc.v[p][q];
      }
    __syncthreads();
    acc.zero();
    tile_mma<TILE>(acc, Vrow + l * r, mr, 1, r, st.Li[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
    for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
      for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
        int row = acc.row(p), col = acc.col(q);
        if (row < r && col < r) Vrow[(long)row * mr + l * r + col] = acc.v[p][q];
      }
  }
  __syncthreads();
  acc.zero();
  if (m > 0) tile_mma<TILE>(acc, Vrow, mr, 1, r, Vrow, mr, 1, r, mr, stg);
  const int ldw = r + 1;
#pragma unroll
  for (int p = 0; p < TileAcc<TILE>::RM; ++p)
#pragma unroll
    for (int q = 0; q < TileAcc<TILE>::RM; ++q) {
      int row = acc.row(p), col = acc.col(q);
      if (row < r && col < r) W[row * ldw + col] = cov0(cv, qx[row], qy[row], qx[col], qy[col]) - acc.v[p][q];
    }
  chol_smem(W, r, ldw, &bad);
  if (st.L[m]) {
    double* Lr = st.L[m] + i * (long)r * r;
    for (int t = threadIdx.x; t < r * r; t += NT) Lr[t] = W[(t / r) * ldw + (t % r)];
    __syncthreads();
  }
  trinv_smem(W, r, ldw, tmp);
  double* Li = st.Li[m] + i * (long)r * r;
  for (int t = threadIdx.x; t < r * r; t += NT) Li[t] = W[(t / r) * ldw + (t % r)];
  if (threadIdx.x == 0 && bad) flag_error(status, ST_NOT_PD, m, i);
}

// ---------------------------------------------------------------------------
// Leaf pass: one CTA per leaf F (Sec. 3.1 leaf quantities, Sec. 3.2-3.3 leaf
// terms from the definition, Sec. 4.3 nugget).
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(NT) leaf_kernel(const Desc* __restrict__ D, const int2* __restrict__ work,
                                                  int* status) {
  extern __shared__ double smem[];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const double tau2 = ds.tau2;
  const int nlmax = ds.nlmax;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long F = it.i;                           // compact leaf id
  const long Fm = st.mort[M][F];                 // its Morton id
  const long o0 = lf.off[Fm];
  const int nF = (int)(lf.off[Fm + 1] - o0);
  if (nF == 0) {
    if (threadIdx.x == 0) { lf.d[F] = 0.0; lf.u[F] = 0.0; }
    return;
  }
  const int lds = nlmax + 1;
  double* sx = smem;
  double* sy = sx + nlmax;
  double* sv = sy + nlmax;
  double* tmp = sv + nlmax;
  double* ax = tmp + nlmax;
  double* ay = ax + MAX_R_DEV;
  double* red = ay + MAX_R_DEV;
  double* S = red + 32;                       // nlmax x (nlmax + 1)
  double* stg = S + (long)nlmax * lds;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int t = threadIdx.x; t < nF; t += NT) {
    sx[t] = lf.xs[o0 + t];
    sy[t] = lf.ys[o0 + t];
    sv[t] = lf.yv[o0 + t];
  }
  double* Hrow = lf.H + o0 * Mr;
  const int nrt = (nF + TILE - 1) / TILE;
  TileAcc<TILE> acc;
  constexpr int RM = TileAcc<TILE>::RM;
  // chain: V^l_F = (C0(S_F, Q_l) - sum_{k<l} V^k_F V^k_{R_l}') L_l^{-T}
  for (int l = 0; l < M; ++l) {
    const long a = ancestor(st, M, F, l);
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    __syncthreads();
    for (int rt = 0; rt < nrt; ++rt) {
      const int nrow = min(TILE, nF - rt * TILE);
      acc.zero();
      if (l > 0) tile_mma<TILE>(acc, Hrow + (long)rt * TILE * Mr, Mr, 1, nrow, Vanc, l * r, 1, r, l * r, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nrow && col < r) {
            int o = rt * TILE + row;
            Hrow[(long)o * Mr + l * r + col] = cov0(cv, sx[o], sy[o], ax[col], ay[col]) - acc.v[p][q];
          }
        }
    }
    __syncthreads();
    for (int rt = 0; rt < nrt; ++rt) {
      const int nrow = min(TILE, nF - rt * TILE);
      acc.zero();
      tile_mma<TILE>(acc, Hrow + (long)rt * TILE * Mr + l * r, Mr, 1, nrow, st.Li[l] + a * (long)r * r, r, 1, r, r, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nrow && col < r) Hrow[(long)(rt * TILE + row) * Mr + l * r + col] = acc.v[p][q];
        }
    }
  }
  __syncthreads();
  // Sigma_F = C0(S_F, S_F) - V_F V_F' + tau2 I  (lower blocks)
  for (int bi = 0; bi < nrt; ++bi)
    for (int bj = 0; bj <= bi; ++bj) {
      const int ni = min(TILE, nF - bi * TILE), nj = min(TILE, nF - bj * TILE);
      acc.zero();
      if (M > 0) tile_mma<TILE>(acc, Hrow + (long)bi * TILE * Mr, Mr, 1, ni, Hrow + (long)bj * TILE * Mr, Mr, 1, nj, Mr, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < ni && col < nj) {
            int oi = bi * TILE + row, oj = bj * TILE + col;
            double v = cov0(cv, sx[oi], sy[oi], sx[oj], sy[oj]) - acc.v[p][q];
            if (oi == oj) v += tau2;
            S[oi * lds + oj] = v;
          }
        }
    }
  chol_smem(S, nF, lds, &bad);
  double ld = 0.0;
  for (int t = threadIdx.x; t < nF; t += NT) ld += log(S[t * lds + t]);
  ld = 2.0 * block_sum(ld, red);
  if (lf.LSf) {
    double* Lf = lf.LSf + lf.sq_off[Fm];
    for (int t = threadIdx.x; t < nF * nF; t += NT) Lf[t] = S[(t / nF) * lds + (t % nF)];
  }
  if (lf.VF) {
    for (long t = threadIdx.x; t < (long)nF * Mr; t += NT) lf.VF[o0 * Mr + t] = Hrow[t];
  }
  trinv_smem(S, nF, lds, tmp);
  double* LS = lf.LS + lf.sq_off[Fm];
  for (int t = threadIdx.x; t < nF * nF; t += NT) LS[t] = S[(t / nF) * lds + (t % nF)];
  // z = L_Sigma^{-1} y
  double zz = 0.0;
  for (int t = threadIdx.x; t < nF; t += NT) {
    double s = 0.0;
    for (int k = 0; k <= t; ++k) s = fma(S[t * lds + k], sv[k], s);
    lf.z[o0 + t] = s;
    zz = fma(s, s, zz);
  }
  zz = block_sum(zz, red);
  if (threadIdx.x == 0) {
    lf.d[F] = ld;
    lf.u[F] = zz;
    if (bad) flag_error(status, ST_NOT_PD, M, F);
  }
  // H^l = L_Sigma^{-1} V^l_F, in place: row tiles from the last, since row
  // tile t only reads rows below its end (L_Sigma^{-1} is lower triangular).
  for (int l = 0; l < M; ++l)
    for (int rt = nrt - 1; rt >= 0; --rt) {
      const int nrow = min(TILE, nF - rt * TILE);
      const int kend = rt * TILE + nrow;
      acc.zero();
      tile_mma<TILE>(acc, S + rt * TILE * lds, lds, 1, nrow, Hrow + l * r, 1, Mr, r, kend, stg);
#pragma unroll
      for (int p = 0; p < RM; ++p)
#pragma unroll
        for (int q = 0; q < RM; ++q) {
          int row = acc.row(p), col = acc.col(q);
          if (row < nrow && col < r) Hrow[(long)(rt * TILE + row) * Mr + l * r + col] = acc.v[p][q];
        }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Leaf SYRK: parent p of level M-1, packed block t = (k, l), k >= l:
//   Ahat_p^{k,l} = sum over the observations of p's children of H^k' H^l.
// The children of p are leaves 4p..4p+3, whose rows are contiguous.
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(NT) leaf_syrk_kernel(const Desc* __restrict__ D, const int2* __restrict__ work) {
  extern __shared__ double smem[];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long p = it.i;                           // compact id at level M-1
  const int t = blockIdx.y;
  if (t >= M * (M + 1) / 2) return;              // fewer blocks in a shallower dataset
  const long pm = st.mort[M - 1][p];
  int k = 0;
  while (tri_index(k + 1, 0) <= t) ++k;
  const int l = t - tri_index(k, 0);
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const int K = (int)(row1 - row0);
  const double* Hb = lf.H + row0 * Mr;
  TileAcc<TILE> acc;
  acc.zero();
  tile_mma<TILE>(acc, Hb + k * r, 1, Mr, r, Hb + l * r, 1, Mr, r, K, smem);
  const int m = M - 1;
  const int T = (m + 1) * (m + 2) / 2;
  double* out = st.Acc[m] + (p * T + t) * (long)r * r;
#pragma unroll
  for (int a = 0; a < TileAcc<TILE>::RM; ++a)
#pragma unroll
    for (int b = 0; b < TileAcc<TILE>::RM; ++b) {
      int row = acc.row(a), col = acc.col(b);
      if (row < r && col < r) out[row * r + col] = acc.v[a][b];
    }
  if (k == l) {
    double* om = st.Om[m] + (p * (m + 1) + k) * (long)r;
    for (int a = threadIdx.x; a < r; a += NT) {
      double s = 0.0;
      for (long o = 0; o < K; ++o) s = fma(Hb[o * Mr + k * r + a], lf.z[row0 + o], s);
      om[a] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Posterior pass, level m: Lt Lt' = I + Ahat^{m,m}; G^l = Lt^{-1} Ahat^{m,l};
// g = Lt^{-1} omegahat^m; d_R = sum_children d + 2 sum log diag Lt;
// u_R = sum_children u - g'g  (Sec. 3.3 in whitened form).
// ---------------------------------------------------------------------------
// EMU: the products G^l = Lt^{-1} Ahat^{m,l} on the emulation engine (its
// staging buffers open the dynamic shared memory).
template <int TILE, bool EMU>
__global__ void __launch_bounds__(NT) post_level_kernel(int m, const Desc* __restrict__ D,
                                                        const int2* __restrict__ work, int* status) {
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
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int r = sh.r, mr = m * r;
  const long i = it.i;
  const int T = (m + 1) * (m + 2) / 2;
  const int ldw = r + 1;
  double* tmp = smem;
  double* red = tmp + MAX_R_DEV;
  double* gs = red + 32;
  double* W = gs + MAX_R_DEV;
  double* stg = W + MAX_R_DEV * (MAX_R_DEV + 1);
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  const double* A = st.Acc[m] + i * (long)T * r * r;
  const double* Amm = A + (long)tri_index(m, m) * r * r;
  for (int t = threadIdx.x; t < r * r; t += NT) {
    int a = t / r, b = t % r;
    W[a * ldw + b] = Amm[t] + (a == b ? 1.0 : 0.0);
  }
  chol_smem(W, r, ldw, &bad);
  double ld = 0.0;
  for (int t = threadIdx.x; t < r; t += NT) ld += log(W[t * ldw + t]);
  ld = 2.0 * block_sum(ld, red);
  if (st.Ltf[m]) {
    double* Lf = st.Ltf[m] + i * (long)r * r;
    for (int t = threadIdx.x; t < r * r; t += NT) Lf[t] = W[(t / r) * ldw + (t % r)];
    __syncthreads();
  }
  trinv_smem(W, r, ldw, tmp);
  double* Lt = st.Lt[m] + i * (long)r * r;
  for (int t = threadIdx.x; t < r * r; t += NT) Lt[t] = W[(t / r) * ldw + (t % r)];
  // g = Lt^{-1} omegahat^m
  const double* om = st.Om[m] + (i * (m + 1) + m) * (long)r;
  double gg = 0.0;
  for (int a = threadIdx.x; a < r; a += NT) {
    double s = 0.0;
    for (int b = 0; b <= a; ++b) s = fma(W[a * ldw + b], om[b], s);
    gs[a] = s;
    st.gv[m][i * r + a] = s;
    gg = fma(s, s, gg);
  }
  gg = block_sum(gg, red);
  // G^l = Lt^{-1} Ahat^{m,l}, l < m.  Ahat^{m,l}(a, b) is stored row-major.
  double* Gr = st.G[m] + i * (long)r * mr;
  if constexpr (EMU) {
    TcAcc ea;
    const int row = ea.row(), c0 = ea.col0();
    for (int l = 0; l < m && ok; ++l) {
      const double* Aml = A + (long)tri_index(m, l) * r * r;
      ok = em_mma(cx, ea, W, ldw, 1, r, Aml, 1, r, r, r);
      if (ok && row < r) {
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c0 + c < r) Gr[(long)row * mr + l * r + c0 + c] = ea.v[c];
      }
    }
  } else {
    TileAcc<TILE> acc;
    for (int l = 0; l < m; ++l) {
      const double* Aml = A + (long)tri_index(m, l) * r * r;
      acc.zero();
      tile_mma<TILE>(acc, W, ldw, 1, r, Aml, 1, r, r, r, stg);
#pragma unroll
      for (int a = 0; a < TileAcc<TILE>::RM; ++a)
#pragma unroll
        for (int b = 0; b < TileAcc<TILE>::RM; ++b) {
          int row = acc.row(a), col = acc.col(b);
          if (row < r && col < r) Gr[(long)row * mr + l * r + col] = acc.v[a][b];
        }
    }
  }
  if (st.gcol[m]) {   // emulation: column scales of G over its r rows, for the aggregation above
    __syncthreads();
    for (int c = threadIdx.x; c < mr; c += NT) {
      int e = -2000;
      for (int a = 0; a < r; ++a) e = max(e, xexp_of(Gr[(long)a * mr + c]));
      st.gcol[m][i * (long)mr + c] = e;
    }
  }
  if (threadIdx.x == 0) {
    double dsum = 0.0, usum = 0.0;
    const long cf = st.cfirst[m][i], cc = st.ccnt[m][i];
    for (long ci = cf; ci < cf + cc; ++ci) {
      if (m + 1 == sh.M) { dsum += lf.d[ci]; usum += lf.u[ci]; }
      else { dsum += st.dd[m + 1][ci]; usum += st.uu[m + 1][ci]; }
    }
    st.dd[m][i] = dsum + ld;
    st.uu[m][i] = usum - gg;
    if (bad) flag_error(status, ST_NOT_PD, m, i);
  }
  if (EMU) {
    em_release(cx);
    if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, m, i);
  }
}

// ---------------------------------------------------------------------------
// Aggregation into parent p of level m-1, packed block t = (k, l), k >= l,
// k, l < m:  Ahat_p^{k,l} = sum_c (Ahat_c^{k,l} - G_c^k' G_c^l)  and
// omegahat_p^k = sum_c (omegahat_c^k - G_c^k' g_c)  (Eqs. mainquantities,
// helpquantities).  The G rows of the four children are contiguous.
// ---------------------------------------------------------------------------
template <int TILE>
__global__ void __launch_bounds__(NT) aggregate_kernel(int m, const Desc* __restrict__ D,
                                                       const int2* __restrict__ work) {
  extern __shared__ double smem[];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const long p = it.i;                           // compact id at level m-1
  const int t = blockIdx.y;
  if (t >= m * (m + 1) / 2) return;
  int k = 0;
  while (tri_index(k + 1, 0) <= t) ++k;
  const int l = t - tri_index(k, 0);
  const int Tc = (m + 1) * (m + 2) / 2;   // blocks per child (level m)
  const int Tp = m * (m + 1) / 2;         // blocks per parent (level m-1)
  const long cf = st.cfirst[m - 1][p], cc = st.ccnt[m - 1][p];   // children: compact ids cf..cf+cc-1
  const double* Gb = st.G[m] + cf * (long)r * mr;
  TileAcc<TILE> acc;
  acc.zero();
  tile_mma<TILE>(acc, Gb + k * r, 1, mr, r, Gb + l * r, 1, mr, r, (int)(cc * r), smem);
  double* out = st.Acc[m - 1] + (p * Tp + t) * (long)r * r;
#pragma unroll
  for (int a = 0; a < TileAcc<TILE>::RM; ++a)
#pragma unroll
    for (int b = 0; b < TileAcc<TILE>::RM; ++b) {
      int row = acc.row(a), col = acc.col(b);
      if (row < r && col < r) {
        double s = -acc.v[a][b];
        for (long c = cf; c < cf + cc; ++c) s += st.Acc[m][(c * Tc + t) * (long)r * r + row * r + col];
        out[row * r + col] = s;
      }
    }
  if (k == l) {
    double* om = st.Om[m - 1] + (p * m + k) * (long)r;
    for (int a = threadIdx.x; a < r; a += NT) {
      double s = 0.0;
      for (long ci = cf; ci < cf + cc; ++ci) {
        s += st.Om[m][(ci * (m + 1) + k) * (long)r + a];
        const double* Gc = st.G[m] + ci * (long)r * mr;
        const double* gc = st.gv[m] + ci * r;
        for (int q = 0; q < r; ++q) s = fma(-Gc[(long)q * mr + k * r + a], gc[q], s);
      }
      om[a] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static int tile_for(int r) { return r <= 16 ? 16 : (r <= 32 ? 32 : 64); }

static size_t prior_smem(int tile) {
  return sizeof(double) * (5 * MAX_R_DEV + 32 + MAX_R_DEV * (MAX_R_DEV + 1) + 2 * KC * (tile + 2));
}
static size_t leaf_smem(int tile, int nlmax) {
  return sizeof(double) * (4 * (size_t)nlmax + 2 * MAX_R_DEV + 32 + (size_t)nlmax * (nlmax + 1) +
                           2 * KC * (tile + 2));
}
static size_t post_smem(int tile) {
  return sizeof(double) * (2 * MAX_R_DEV + 32 + MAX_R_DEV * (MAX_R_DEV + 1) + 2 * KC * (tile + 2));
}
static size_t syrk_smem(int tile) { return sizeof(double) * 2 * KC * (tile + 2); }

#define MRA_LAUNCH_ONE(T, KERNEL, grid, smem, stream, ...)                \
  {                                                                      \
    e = cudaFuncSetAttribute(KERNEL<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(smem)); \
    if (e) return e;                                                     \
    KERNEL<T><<<grid, NT, smem, stream>>>(__VA_ARGS__);                  \
  }
#define MRA_LAUNCH(tile, KERNEL, grid, smem, stream, ...)                         \
  do {                                                                            \
    if ((tile) == 16) MRA_LAUNCH_ONE(16, KERNEL, grid, smem, stream, __VA_ARGS__) \
    else if ((tile) == 32) MRA_LAUNCH_ONE(32, KERNEL, grid, smem, stream, __VA_ARGS__) \
    else MRA_LAUNCH_ONE(64, KERNEL, grid, smem, stream, __VA_ARGS__)              \
  } while (0)


static cudaError_t launch_post_level(bool emu, int tile, int m, int nblocks, cudaStream_t s, const Desc* d_desc,
                                     const int2* work, int* status) {
  cudaError_t e;
  size_t sm = post_smem(tile);
  if (emu) {
    sm += EM_STAGE_BYTES;
    if (sm < EM_SOLO_SMEM) sm = EM_SOLO_SMEM;
  }
#define MRA_POST(T, EMU)                                                                                  \
  {                                                                                                       \
    if ((e = cudaFuncSetAttribute(post_level_kernel<T, EMU>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                  (int)sm)))                                                              \
      return e;                                                                                           \
    post_level_kernel<T, EMU><<<nblocks, NT, sm, s>>>(m, d_desc, work, status);                           \
  }
  if (tile == 16) {
    if (emu) MRA_POST(16, true) else MRA_POST(16, false)
  } else if (tile == 32) {
    if (emu) MRA_POST(32, true) else MRA_POST(32, false)
  } else {
    if (emu) MRA_POST(64, true) else MRA_POST(64, false)
  }
#undef MRA_POST
  return cudaGetLastError();
}

cudaError_t launch_loglik(const Plan& pl, const Desc* d_desc, int* status, cudaStream_t s, int64_t* launches,
                          Timer* tm) {
  const int tile = pl.tile;
  cudaError_t e;
  const int prior_hi = pl.prior_hi < 0 ? pl.maxM : pl.prior_hi;
  const int post_hi = pl.post_hi < 0 ? pl.maxM : pl.post_hi;
  // prior pass, top-down
  for (int m = pl.prior_lo; m < prior_hi; ++m) {
    if (pl.n_lvl[m] == 0) continue;
    tm->start(0, s, 0, m);
    if (pl.mixed) {
      if (pl.c_pri[m]) {
        if ((e = launch_prior_tc(m, d_desc, pl.w_pri[m], pl.n_pri[m], pl.mixed == 2, status, s, pl.c_pri[m],
                                 pl.rcap)))
          return e;
      } else if ((e = launch_prior_tc(m, d_desc, pl.w_lvl[m], pl.n_lvl[m], pl.mixed == 2, status, s))) {
        return e;
      }
    } else {
      MRA_LAUNCH(tile, prior_level_kernel, pl.n_lvl[m], prior_smem(tile), s, m, d_desc, pl.w_lvl[m], status);
    }
    tm->stop(s);
    ++*launches;
  }
  // leaves
  if (pl.leaves && pl.n_leaf > 0) {
    const bool chain = pl.mixed == 2 && pl.n_syrk > 0;   // the emulated form's separate chain kernel
    tm->start(1, s, chain ? 1 : 2, pl.maxM);
    if (pl.mixed) {
      // (the emulated form's chain kernel runs per level-(M-1) region: the leaf_syrk work list)
      if ((e = launch_leaf_tc(d_desc, pl.w_leaf, pl.n_leaf, pl.nlmax, pl.mixed == 2, status, s,
                              pl.c_chn ? pl.w_chn : pl.w_syrk, pl.c_chn ? pl.n_chn : pl.n_syrk, tm, pl.maxM,
                              pl.c_leaf, pl.lrows, pl.c_chn)))
        return e;
      if (pl.mixed == 2 && pl.n_syrk > 0) ++*launches;   // the chain kernel
    } else {
      MRA_LAUNCH(tile, leaf_kernel, pl.n_leaf, leaf_smem(tile, pl.nlmax), s, d_desc, pl.w_leaf, status);
    }
    tm->stop(s);
    ++*launches;
  }
  if (pl.leaves && pl.n_syrk > 0) {
    dim3 grid(pl.n_syrk, pl.t_syrk);
    tm->start(2, s, 3, pl.maxM);
    if (pl.mixed == 2) {
      if ((e = launch_leaf_syrk_em(d_desc, pl.w_syrk, pl.n_syrk, pl.maxM, pl.r, status, s))) return e;
    } else {
      MRA_LAUNCH(tile, leaf_syrk_kernel, grid, syrk_smem(tile), s, d_desc, pl.w_syrk);
    }
    tm->stop(s);
    ++*launches;
  }
  // posterior pass, bottom-up
  for (int m = post_hi - 1; m >= pl.post_lo; --m) {
    if (pl.n_lvl[m] > 0) {
      tm->start(3, s, 4, m);
      // (the emulated form's G = Lt^{-1} Ahat products have K = r: at r <= 32 the engine's fixed cost per
      // product exceeds the FP64 tile product, measured 208 against 104 ms on the ragged batch)
      if ((e = launch_post_level(pl.mixed == 2 && pl.r > 32, tile, m, pl.n_lvl[m], s, d_desc, pl.w_lvl[m], status)))
        return e;
      tm->stop(s);
      ++*launches;
    }
    if (m > 0 && pl.n_agg[m] > 0) {
      dim3 g2(pl.n_agg[m], m * (m + 1) / 2);
      tm->start(4, s, 5, m);
      if (pl.mixed == 2) {
        if ((e = launch_aggregate_em(m, pl.r, d_desc, pl.w_agg[m], pl.n_agg[m], status, s))) return e;
      } else {
        MRA_LAUNCH(tile, aggregate_kernel, g2, syrk_smem(tile), s, m, d_desc, pl.w_agg[m]);
      }
      tm->stop(s);
      ++*launches;
    }
  }
  return cudaGetLastError();
}

int tile_for_r(int r) { return tile_for(r); }

// -2 log L terms (d, u) at the root of every dataset of a batch.
__global__ void gather_roots_kernel(const Desc* __restrict__ D, int nd, double* out) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  const Desc& ds = D[d];
  if (ds.sh.M > 0) {
    out[2 * d] = ds.st.dd[0][0];
    out[2 * d + 1] = ds.st.uu[0][0];
  } else {
    out[2 * d] = ds.lf.d[0];
    out[2 * d + 1] = ds.lf.u[0];
  }
}

cudaError_t launch_gather_roots(const Desc* d_desc, int nd, double* out, cudaStream_t s, int64_t* launches) {
  gather_roots_kernel<<<(nd + 127) / 128, 128, 0, s>>>(d_desc, nd, out);
  ++*launches;
  return cudaGetLastError();
}

size_t leaf_smem_bytes(int r, int nlmax) { return leaf_smem(tile_for(r), nlmax); }

}  // namespace mra
