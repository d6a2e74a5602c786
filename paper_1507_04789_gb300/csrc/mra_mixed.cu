// mra_mixed.cu -- mixed-precision prior and leaf kernels (MRA_PREC_MIXED).
//
// The same whitened prior pass (Eq. priorw in block-Cholesky form) and leaf
// pass (Sec. 3.1-3.2 at m = M, Sec. 4.3 nugget) as mra_loglik.cu, with the
// dense contractions -- the chain updates C - V V', the products with L^{-T},
// the leaf covariance C - V_F V_F' and the leaf solve L_Sigma^{-1} V_F -- on the
// tensor cores through tc_mma (3xTF32 with FP64 accumulation every 64 terms).
// The Cholesky factorisations, triangular inverses, log-determinants and the
// quadratic form stay in FP64, and so do all Gram products of the posterior
// pass (leaf_syrk, aggregate), which need more than FP32 accuracy.
#include "mra_launch.h"
#include "mra_tc.cuh"

namespace mra {

__global__ void __launch_bounds__(NT) prior_level_kernel_tc(int m, const Desc* __restrict__ D,
                                                             const int2* __restrict__ work, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail, bad;
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const long i = it.i;
  uint32_t* stage = reinterpret_cast<uint32_t*>(dsm);
  double* qx = reinterpret_cast<double*>(dsm + TC_STAGE_BYTES);
  double* qy = qx + MAX_R_DEV;
  double* ax = qy + MAX_R_DEV;
  double* ay = ax + MAX_R_DEV;
  double* tmp = ay + MAX_R_DEV;
  double* W = tmp + MAX_R_DEV;                 // r x (r + 1)
  if (threadIdx.x == 0) bad = 0;
  TcCtx cx{stage, &mbar, 0, 0, &fail};
  tc_init(cx, &tmem_slot);
  load_knots(sh.bbox, m, st.mort[m][i], sh.gx, sh.gy, qx, qy);
  double* Vrow = st.V[m] + i * (long)r * mr;
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  for (int l = 0; l < m && ok; ++l) {
    const long a = ancestor(st, m, i, l);
    __syncthreads();
    load_knots(sh.bbox, l, st.mort[l][a], sh.gx, sh.gy, ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    acc.zero();
    __syncthreads();
    if (l > 0) ok = tc_mma(cx, acc, Vrow, mr, 1, r, Vanc, l * r, 1, r, l * r);
    if (!ok) break;
    if (row < r)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) Vrow[(long)row * mr + l * r + col] = cov0(cv, qx[row], qy[row], ax[col], ay[col]) - acc.v[c];
      }
    __syncthreads();
    acc.zero();
    ok = tc_mma(cx, acc, Vrow + l * r, mr, 1, r, st.Li[l] + a * (long)r * r, r, 1, r, r);
    if (!ok) break;
    if (row < r)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) Vrow[(long)row * mr + l * r + col] = acc.v[c];
      }
  }
  __syncthreads();
  if (ok) {
    acc.zero();
    if (m > 0) ok = tc_mma(cx, acc, Vrow, mr, 1, r, Vrow, mr, 1, r, mr);
  }
  if (ok) {
    const int ldw = r + 1;
    if (row < r)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) W[row * ldw + col] = cov0(cv, qx[row], qy[row], qx[col], qy[col]) - acc.v[c];
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
  }
  tc_release(cx);
  if (threadIdx.x == 0) {
    if (!ok) flag_error(status, ST_TIMEOUT, m, i);
    else if (bad) flag_error(status, ST_NOT_PD, m, i);
  }
}

__global__ void __launch_bounds__(NT) leaf_kernel_tc(const Desc* __restrict__ D, const int2* __restrict__ work,
                                                     int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ int fail, bad;
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
  const long Fm = st.mort[M][F];
  const long o0 = lf.off[Fm];
  const int nF = (int)(lf.off[Fm + 1] - o0);
  if (nF == 0) {
    if (threadIdx.x == 0) { lf.d[F] = 0.0; lf.u[F] = 0.0; }
    return;
  }
  const int lds = nlmax + 1;
  uint32_t* stage = reinterpret_cast<uint32_t*>(dsm);
  double* sx = reinterpret_cast<double*>(dsm + TC_STAGE_BYTES);
  double* sy = sx + nlmax;
  double* sv = sy + nlmax;
  double* tmp = sv + nlmax;
  double* ax = tmp + nlmax;
  double* ay = ax + MAX_R_DEV;
  double* red = ay + MAX_R_DEV;
  double* S = red + 32;                         // nlmax x (nlmax + 1)
  if (threadIdx.x == 0) bad = 0;
  TcCtx cx{stage, &mbar, 0, 0, &fail};
  tc_init(cx, &tmem_slot);
  for (int t = threadIdx.x; t < nF; t += NT) {
    sx[t] = lf.xs[o0 + t];
    sy[t] = lf.ys[o0 + t];
    sv[t] = lf.yv[o0 + t];
  }
  double* Hrow = lf.H + o0 * Mr;
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  // chain: V^l_F = (C0(S_F, Q_l) - sum_{k<l} V^k_F V^k_{R_l}') L_l^{-T}  (one 128-row tile)
  for (int l = 0; l < M && ok; ++l) {
    const long a = ancestor(st, M, F, l);
    __syncthreads();
    load_knots(sh.bbox, l, st.mort[l][a], sh.gx, sh.gy, ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    acc.zero();
    __syncthreads();
    if (l > 0) ok = tc_mma(cx, acc, Hrow, Mr, 1, nF, Vanc, l * r, 1, r, l * r);
    if (!ok) break;
    if (row < nF)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) Hrow[(long)row * Mr + l * r + col] = cov0(cv, sx[row], sy[row], ax[col], ay[col]) - acc.v[c];
      }
    __syncthreads();
    acc.zero();
    ok = tc_mma(cx, acc, Hrow + l * r, Mr, 1, nF, st.Li[l] + a * (long)r * r, r, 1, r, r);
    if (!ok) break;
    if (row < nF)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) Hrow[(long)row * Mr + l * r + col] = acc.v[c];
      }
  }
  __syncthreads();
  // Sigma_F = C0(S_F, S_F) - V_F V_F' + tau2 I, 64 columns at a time
  const int nct = (nF + TC_N - 1) / TC_N;
  for (int ct = 0; ct < nct && ok; ++ct) {
    const int ncol = min(TC_N, nF - ct * TC_N);
    acc.zero();
    if (M > 0) ok = tc_mma(cx, acc, Hrow, Mr, 1, nF, Hrow + (long)ct * TC_N * Mr, Mr, 1, ncol, Mr);
    if (!ok) break;
    if (row < nF)
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < ncol) {
          const int oj = ct * TC_N + col;
          double v = cov0(cv, sx[row], sy[row], sx[oj], sy[oj]) - acc.v[c];
          if (row == oj) v += tau2;
          S[row * lds + oj] = v;
        }
      }
  }
  double ld = 0.0, zz = 0.0;
  if (ok) {
    chol_smem(S, nF, lds, &bad);
    for (int t = threadIdx.x; t < nF; t += NT) ld += log(S[t * lds + t]);
    ld = 2.0 * block_sum(ld, red);
    if (lf.LSf) {
      double* Lf = lf.LSf + lf.sq_off[Fm];
      for (int t = threadIdx.x; t < nF * nF; t += NT) Lf[t] = S[(t / nF) * lds + (t % nF)];
    }
    if (lf.VF)
      for (long t = threadIdx.x; t < (long)nF * Mr; t += NT) lf.VF[o0 * Mr + t] = Hrow[t];
    trinv_smem(S, nF, lds, tmp);
    double* LS = lf.LS + lf.sq_off[Fm];
    for (int t = threadIdx.x; t < nF * nF; t += NT) LS[t] = S[(t / nF) * lds + (t % nF)];
    for (int t = threadIdx.x; t < nF; t += NT) {
      double s = 0.0;
      for (int k = 0; k <= t; ++k) s = fma(S[t * lds + k], sv[k], s);
      lf.z[o0 + t] = s;
      zz = fma(s, s, zz);
    }
    zz = block_sum(zz, red);
    // H^l = L_Sigma^{-1} V^l_F (whole block read before it is overwritten)
    for (int l = 0; l < M && ok; ++l) {
      acc.zero();
      ok = tc_mma(cx, acc, S, lds, 1, nF, Hrow + l * r, 1, Mr, r, nF);
      if (!ok) break;
      if (row < nF)
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < r) Hrow[(long)row * Mr + l * r + col] = acc.v[c];
        }
      __syncthreads();
    }
  }
  tc_release(cx);
  if (threadIdx.x == 0) {
    lf.d[F] = ld;
    lf.u[F] = zz;
    if (!ok) flag_error(status, ST_TIMEOUT, M, F);
    else if (bad) flag_error(status, ST_NOT_PD, M, F);
  }
}

size_t prior_tc_smem_bytes() {
  return TC_STAGE_BYTES + sizeof(double) * (5 * MAX_R_DEV + MAX_R_DEV * (MAX_R_DEV + 1));
}
size_t leaf_tc_smem_bytes(int nlmax) {
  return TC_STAGE_BYTES + sizeof(double) * (4 * (size_t)nlmax + 2 * MAX_R_DEV + 32 + (size_t)nlmax * (nlmax + 1));
}

cudaError_t launch_prior_tc(int m, const Desc* d_desc, const int2* work, int nblocks, int* status, cudaStream_t s) {
  const size_t sm = prior_tc_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(prior_level_kernel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  prior_level_kernel_tc<<<nblocks, NT, sm, s>>>(m, d_desc, work, status);
  return cudaGetLastError();
}

cudaError_t launch_leaf_tc(const Desc* d_desc, const int2* work, int nblocks, int nlmax, int* status, cudaStream_t s) {
  const size_t sm = leaf_tc_smem_bytes(nlmax);
  cudaError_t e = cudaFuncSetAttribute(leaf_kernel_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e) return e;
  leaf_kernel_tc<<<nblocks, NT, sm, s>>>(d_desc, work, status);
  return cudaGetLastError();
}

}  // namespace mra
