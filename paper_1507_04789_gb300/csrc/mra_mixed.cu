// mra_mixed.cu -- tensor-core prior and leaf kernels (MRA_PREC_MIXED and
// MRA_PREC_EMU).
//
// The same whitened prior pass (Eq. priorw in block-Cholesky form) and leaf
// pass (Sec. 3.1-3.2 at m = M, Sec. 4.3 nugget) as mra_loglik.cu, with the
// dense contractions -- the chain updates C - V V', the products with L^{-T},
// the leaf covariance C - V_F V_F' and the leaf solve L_Sigma^{-1} V_F -- on the
// tensor cores, through one of two engines:
//  * MRA_PREC_MIXED: tc_mma (3xTF32 with FP64 accumulation every 64 terms);
//    the Gram products of the posterior pass (leaf_syrk, aggregate) stay in
//    the FP64 kernels, since they need more than FP32 accuracy;
//  * MRA_PREC_EMU: em_mma (bf16-slice FP64 emulation, about 1e-14 relative),
//    which also runs the two Gram products (leaf_syrk_kernel_em,
//    aggregate_kernel_em below).
// The Cholesky factorisations, triangular inverses, log-determinants and the
// quadratic form stay in FP64.
#include <algorithm>

#include "mra_emu.cuh"
#include "mra_launch.h"
#include "mra_tc.cuh"

namespace mra {

// The tensor-core engine of a kernel: 3xTF32 (EMU = false) or the FP64-grade
// bf16-slice emulation (EMU = true); both write the same TcAcc layout.  Every
// call site zeroes the accumulator first: the 3xTF32 engine adds to it, the
// emulation engine overwrites it.
template <bool EMU>
struct Engine;

template <>
struct Engine<false> {
  static constexpr int STAGE = TC_STAGE_BYTES;
  TcCtx cx;
  __device__ void init(unsigned char* stage, uint64_t* mbar, uint32_t* tmem_slot, int* fail, int*, int*) {
    cx = TcCtx{reinterpret_cast<uint32_t*>(stage), mbar, 0, 0, fail};
    tc_init(cx, tmem_slot);
  }
  __device__ bool mma(TcAcc& acc, const double* A, long sai, long sak, int na, const double* B, long sbj, long sbk,
                      int nb, int K, const int* = nullptr, int = 0, const int* = nullptr, int = 0) {
    return tc_mma(cx, acc, A, sai, sak, na, B, sbj, sbk, nb, K);
  }
  __device__ void release() { tc_release(cx); }
};

template <>
struct Engine<true> {
  static constexpr int STAGE = EM_STAGE_BYTES;
  EmCtx cx;
  __device__ void init(unsigned char* stage, uint64_t* mbar, uint32_t* tmem_slot, int* fail, int* rexp, int* cexp) {
    cx.stage = reinterpret_cast<uint16_t*>(stage);
    cx.rexp = rexp;
    cx.cexp = cexp;
    cx.mbar = mbar;
    cx.fail = fail;
    em_init(cx, tmem_slot);
  }
  // pa / pb: the operands' row scales from their producers (see em_mma), or null
  __device__ bool mma(TcAcc& acc, const double* A, long sai, long sak, int na, const double* B, long sbj, long sbk,
                      int nb, int K, const int* pa = nullptr, int pas = 0, const int* pb = nullptr, int pbs = 0) {
    return em_mma(cx, acc, A, sai, sak, na, B, sbj, sbk, nb, K, pa, pas, pb, pbs);
  }
  __device__ void release() { em_release(cx); }
};

constexpr int EM_GMAX = 6;   // 128-column groups of a row of at most MRA_MAX_M x MAX_R_DEV = 768 columns

// Prior of level m on the tensor cores.  gcnt (else null): the work item is a
// group of gcnt[b] sibling regions with consecutive compact ids from it.i
// (children of one parent, so with the same ancestors), stacked G r <= rcap
// rows deep: their chain blocks are one product per ancestor level (the
// ancestor's V and L^{-1} split once for all of them), and their W blocks are
// factorised and inverted block by block (chol_seg / trinv_seg, stacked rows).
template <bool EMU>
__global__ void __launch_bounds__(NT) prior_level_kernel_tc(int m, const Desc* __restrict__ D,
                                                             const int2* __restrict__ work, int* status,
                                                             const int* __restrict__ gcnt, int rcap) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail, bad;
  __shared__ int rexp[EMU ? EM_REXP : 1], cexp[EMU ? EM_CEXP : 1];
  // emulation: row scales of the stacked V rows per 128-column group, and of the current X^l block
  __shared__ int vsc[EMU ? EM_GMAX * TC_M : 1], xsc[EMU ? TC_M : 1];
  // c0_fast on two knot grids: squared scaled offsets between their columns and
  // between their rows (per stacked region), variance factors of the columns
  // (sigma2 in pgp), and the column and row of every knot
  __shared__ double pdx[LGRP_MAX * C0_GMAX * C0_GMAX], pdy[LGRP_MAX * C0_GMAX * C0_GMAX];
  __shared__ double pgp[LGRP_MAX * C0_GMAX], pgq[LGRP_MAX * C0_GMAX];
  __shared__ unsigned char qcol[MAX_R_DEV], qrow[MAX_R_DEV];
  __shared__ int gseg[LGRP_MAX + 1];
  __shared__ double gpv[LGRP_MAX];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const int r = sh.r, mr = m * r;
  const int G = gcnt ? gcnt[blockIdx.x] : 1;
  const int R = G * r;                         // stacked rows
  const int gx = sh.gx, gy = sh.gy;
  const bool fast = c0_fast_ok(cv, gx, gy);
  const double c0s = c0_scale(cv);
  if (R > rcap || R > TC_M) {                  // (a group larger than the layout: never formed by the host)
    if (threadIdx.x == 0) flag_error(status, ST_LIMIT, m, it.i);
    return;
  }
  for (int q = threadIdx.x; q < r; q += NT) {
    qcol[q] = (unsigned char)(q % gx);
    qrow[q] = (unsigned char)(q / gx);
  }
  if (threadIdx.x <= G) gseg[threadIdx.x] = threadIdx.x * r;
  if (EMU)
    for (int t = threadIdx.x; t < EM_GMAX * TC_M; t += NT) vsc[t] = -2000;
  const long i = it.i;                          // the first region of the group
  double* qx = reinterpret_cast<double*>(dsm + Engine<EMU>::STAGE);   // the group's knots, rcap each
  double* qy = qx + rcap;
  double* ax = qy + rcap;
  double* ay = ax + MAX_R_DEV;
  double* tmp = ay + MAX_R_DEV;                 // rcap
  double* W = tmp + rcap;                       // rcap x (r + 1): region g's block in rows g r .. g r + r - 1
  // offsets between every stacked region's knot grid (qx, qy) + g r and the grid
  // (bx, by), or (self) the region's own grid (all threads; the caller
  // synchronises before and after)
  const int gsz = gx * gx + gy * gy;
  auto grid_offsets = [&](const double* bx, const double* by, bool self) {
    for (int t = threadIdx.x; t < G * gsz; t += NT) {
      const int g = t / gsz, u = t - g * gsz;
      const double* ox = qx + g * r;
      const double* oy = qy + g * r;
      const double* px = self ? ox : bx;
      const double* py = self ? oy : by;
      if (u < gx * gx) {
        const double d = c0s * (ox[u / gx] - px[u % gx]);
        pdx[g * C0_GMAX * C0_GMAX + u] = d * d;
      } else {
        const int v = u - gx * gx;
        const double d = c0s * (oy[(v / gy) * gx] - py[(v % gy) * gx]);
        pdy[g * C0_GMAX * C0_GMAX + v] = d * d;
      }
    }
    for (int t = threadIdx.x; t < G * gx; t += NT) {
      const int g = t / gx, c = t - g * gx;
      pgp[t] = cv.sigma2 * c0_vfac(cv, qx[g * r + c]);
      pgq[t] = c0_vfac(cv, self ? qx[g * r + c] : bx[c]);
    }
  };
  // C0 between row qi of the stack (region qi / r) and knot qj of the grid the offsets were formed for
  auto c0_at = [&](int qi, int qj, const double* bx, const double* by) {
    const int g = qi / r, ql = qi - g * r;
    const int ci = qcol[ql], cj = qcol[qj];
    return fast ? c0_fast(cv.family, pdx[g * C0_GMAX * C0_GMAX + ci * gx + cj] +
                                         pdy[g * C0_GMAX * C0_GMAX + qrow[ql] * gy + qrow[qj]],
                          cv.nonstat ? pgp[g * gx + ci] * pgq[g * gx + cj] : cv.sigma2)
                : cov0(cv, qx[qi], qy[qi], bx[qj], by[qj]);
  };
  if (threadIdx.x == 0) bad = 0;
  Engine<EMU> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  for (int g = 0; g < G; ++g) load_knots(sh, m, st.mort[m][i + g], qx + g * r, qy + g * r);
  double* Vrow = st.V[m] + i * (long)r * mr;   // the group's rows are consecutive
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  for (int l = 0; l < m && ok; ++l) {
    const long a = ancestor(st, m, i, l);
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    if (EMU)
      for (int t = threadIdx.x; t < TC_M; t += NT) xsc[t] = -2000;
    __syncthreads();
    if (fast) {
      grid_offsets(ax, ay, false);
      __syncthreads();
    }
    // C0(Q_R, Q_{R_l}) into block l, spread over every warp (the FP64 pipe of
    // every SM sub-partition); the product below reads only blocks < l
    for (int t = threadIdx.x; t < R * r; t += NT) {
      const int qi = t / r, qj = t - qi * r;
      const double v = c0_at(qi, qj, ax, ay);
      Vrow[(long)qi * mr + l * r + qj] = v;
      if (EMU && l == 0) atomicMax(xsc + qi, xexp_of(v));
    }
    acc.zero();
    __syncthreads();
    if (l > 0) {
      const int* vsa = EMU ? st.vexp[l] + a * (long)((l * r + 127) / 128) * r : nullptr;
      ok = eng.mma(acc, Vrow, mr, 1, R, Vanc, l * r, 1, r, l * r, vsc, TC_M, vsa, r);
      if (!ok) break;
      if (row < R) {
        int e = -2000;
        #pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < r) {
            const double v = Vrow[(long)row * mr + l * r + col] - acc.v[c];
            Vrow[(long)row * mr + l * r + col] = v;
            e = max(e, xexp_of(v));
          }
        }
        if (EMU) atomicMax(xsc + row, e);
      }
    }
    __syncthreads();
    acc.zero();
    ok = eng.mma(acc, Vrow + l * r, mr, 1, R, st.Li[l] + a * (long)r * r, r, 1, r, r, xsc, 0,
                 EMU ? st.liexp[l] + a * r : nullptr, 0);
    if (!ok) break;
    if (row < R) {
      int e0 = -2000, e1 = -2000;       // a thread's 32 columns touch at most two groups
      const int gbase = (l * r + c0) / 128;
      #pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) {
          Vrow[(long)row * mr + l * r + col] = acc.v[c];
          const int e = xexp_of(acc.v[c]);
          if ((l * r + col) / 128 == gbase) e0 = max(e0, e);
          else e1 = max(e1, e);
        }
      }
      if (EMU) {
        atomicMax(vsc + gbase * TC_M + row, e0);
        if (e1 > -2000) atomicMax(vsc + (gbase + 1) * TC_M + row, e1);
      }
    }
  }
  __syncthreads();                             // knots loaded, chain blocks written
  const int ldw = r + 1;
  if (fast) {
    grid_offsets(qx, qy, true);
    __syncthreads();
  }
  // lower triangle of every region's C0(Q_R, Q_R), every warp
  const int T1 = r * (r + 1) / 2;
  for (int t = threadIdx.x; t < G * T1; t += NT) {
    const int g = t / T1;
    int qi, qj;
    tri_decode(t - g * T1, qi, qj);
    W[(g * r + qi) * ldw + qj] = c0_at(g * r + qi, qj, qx + g * r, qy + g * r);
  }
  __syncthreads();
  // W_R -= V_R V_R' of every region (the diagonal blocks of the stacked product)
  const int nct = (R + TC_N - 1) / TC_N;
  for (int ct = 0; ct < nct && ok && m > 0; ++ct) {
    const int ncol = min(TC_N, R - ct * TC_N);
    acc.zero();
    ok = eng.mma(acc, Vrow, mr, 1, R, Vrow + (long)ct * TC_N * mr, mr, 1, ncol, mr, vsc, TC_M, vsc + ct * TC_N,
                 TC_M);
    if (!ok) break;
    if (row < R) {
      const int rb = (row / r) * r;           // the row's block
      #pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int oj = ct * TC_N + c0 + c;
        if (c0 + c < ncol && oj >= rb && oj <= row) W[row * ldw + oj - rb] -= acc.v[c];
      }
    }
    __syncthreads();
  }
  if (ok) {
    if (G == 1) chol_smem(W, r, ldw, &bad);
    else chol_seg<true>(W, ldw, gseg, G, &bad, gpv);
    if (st.L[m]) {
      double* Lr = st.L[m] + i * (long)r * r;
      for (int t = threadIdx.x; t < R * r; t += NT) Lr[t] = W[(t / r) * ldw + (t % r)];
      __syncthreads();
    }
    if (G == 1) trinv_smem(W, r, ldw, tmp);
    else trinv_seg<true>(W, ldw, gseg, G, tmp, gpv);
    double* Li = st.Li[m] + i * (long)r * r;
    for (int t = threadIdx.x; t < R * r; t += NT) Li[t] = W[(t / r) * ldw + (t % r)];
    if (EMU) {   // row scales of V_R and L_R^{-1} for the descendants' products
      for (int t = threadIdx.x; t < R; t += NT) {
        int e = -2000;
        for (int k = 0; k <= t % r; ++k) e = max(e, xexp_of(W[t * ldw + k]));
        st.liexp[m][i * r + t] = e;
      }
      if (m > 0) {
        const int ng = (mr + 127) / 128;
        for (int t = threadIdx.x; t < ng * R; t += NT) {   // region g = q / r, group t / R, row q % r
          const int grp = t / R, q = t - grp * R, g = q / r;
          st.vexp[m][((i + g) * ng + grp) * (long)r + (q - g * r)] = vsc[grp * TC_M + q];
        }
      }
    }
  }
  eng.release();
  if (threadIdx.x == 0) {
    if (!ok) flag_error(status, ST_TIMEOUT, m, i);
    else if (bad) flag_error(status, ST_NOT_PD, m, i);
  }
}

// Leaf chain of the emulated form, per level-(M-1) region P over the
// contiguous rows of its children in 128-row tiles (their ancestors' V and
// L^{-1} are the same, so one split of those serves up to 128 rows):
//   V^l_F = (C0(S_F, Q_l) - sum_{k<l} V^k_F V^k_{R_l}') L_l^{-T},  l = 0..M-1,
// written to H, with the row scales of every 128-column group exported to
// lf.hrow for the leaf kernel.  gcnt (else null): the work item is a group of
// gcnt[b] sibling regions from P = it.i with at most 128 rows in all, one
// tile: the levels l < M - 1 (their common ancestors) are one product per
// level for the whole tile, level M - 1 one product per region on its rows.
template <bool GRP>
__global__ void __launch_bounds__(NT) chain_forward_kernel_em(const Desc* __restrict__ D,
                                                              const int2* __restrict__ work, int* status,
                                                              const int* __restrict__ gcnt) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  __shared__ int hsc[EM_GMAX * TC_M], xsc[TC_M];
  __shared__ double sx[TC_M], sy[TC_M], ax[MAX_R_DEV], ay[MAX_R_DEV];
  // c0_fast: squared scaled offsets of the tile's points to the knot grid's
  // columns and rows, the points' variance factors (sigma2 included) and the
  // knot columns'; the column and row of every knot
  __shared__ double c0dx[TC_M * C0_GMAX], c0dy[TC_M * C0_GMAX], c0gp[TC_M], c0gq[C0_GMAX];
  __shared__ unsigned char qcol[MAX_R_DEV], qrow[MAX_R_DEV];
  __shared__ int gseg[LGRP_MAX + 1];             // a group's regions: tile rows gseg[g] .. gseg[g + 1] - 1
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r, ng = (Mr + EM_KG - 1) / EM_KG;
  const long P = it.i;
  const int G = GRP && gcnt ? gcnt[blockIdx.x] : 1;   // (GRP false: one region, the loops below fold)
  const long pm = st.mort[M - 1][P];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[((long)st.mort[M - 1][P + G - 1] + 1) << leaf_bits(ds.sh)];
  if (G > 1 && row1 - row0 > TC_M) {             // (a group of more than one tile: never formed by the host)
    if (threadIdx.x == 0) flag_error(status, ST_LIMIT, M - 1, P);
    return;
  }
  if (threadIdx.x <= G)
    gseg[threadIdx.x] = (int)((threadIdx.x < G ? lf.off[(long)st.mort[M - 1][P + threadIdx.x] << leaf_bits(ds.sh)] : row1) - row0);
  const int gx = sh.gx, gy = sh.gy;
  const bool fast = c0_fast_ok(cv, gx, gy);
  const double c0s = c0_scale(cv), is2 = 1.0 / cv.sigma2;
  for (int q = threadIdx.x; q < r; q += NT) {
    qcol[q] = (unsigned char)(q % gx);
    qrow[q] = (unsigned char)(q / gx);
  }
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  for (long t0 = row0; t0 < row1 && ok; t0 += TC_M) {
    const int na = (int)min((long)TC_M, row1 - t0);
    double* Hrow = lf.H + t0 * Mr;
    __syncthreads();                             // the previous tile's points and scales are no longer read
    for (int t = threadIdx.x; t < na; t += NT) {
      sx[t] = lf.xs[t0 + t];
      sy[t] = lf.ys[t0 + t];
      if (fast) c0gp[t] = cv.sigma2 * c0_vfac(cv, sx[t]);
    }
    for (int t = threadIdx.x; t < EM_GMAX * TC_M; t += NT) hsc[t] = -2000;
    for (int l = 0; l < M && ok; ++l)
    for (int sg = 0; sg < (G > 1 && l == M - 1 ? G : 1) && ok; ++sg) {   // (level M - 1 of a group: per region)
      const bool per = G > 1 && l == M - 1;
      const long a = per ? P + sg : ancestor(st, M - 1, P, l);
      const int ra = per ? gseg[sg] : 0, nr = per ? gseg[sg + 1] - gseg[sg] : na;   // this product's rows
      if (nr == 0) continue;                     // (uniform: a region without observations)
      double* Hseg = Hrow + (long)ra * Mr;
      __syncthreads();
      load_knots(sh, l, st.mort[l][a], ax, ay);
      const double* Vanc = st.V[l] + a * (long)r * (l * r);
      for (int t = threadIdx.x; t < TC_M; t += NT) xsc[t] = -2000;
      __syncthreads();
      if (fast) {   // offsets to the knot grid's gx columns and gy rows, knot columns' variance factors
        const int gs = gx + gy;
        for (int t = threadIdx.x; t < nr * gs; t += NT) {
          const int fi = ra + t / gs, c = t - (t / gs) * gs;
          const double d = c < gx ? c0s * (sx[fi] - ax[c]) : c0s * (sy[fi] - ay[(c - gx) * gx]);
          (c < gx ? c0dx + fi * gx + c : c0dy + fi * gy + (c - gx))[0] = d * d;
        }
        for (int c = threadIdx.x; c < gx; c += NT) c0gq[c] = c0_vfac(cv, ax[c]);
        __syncthreads();
      }
      // C0(S_F, Q_l) into block l (the product below reads only blocks < l); in
      // gradient calls with its two derivatives
      for (int t = threadIdx.x; t < nr * r; t += NT) {
        const int fi = ra + t / r, qj = t - (t / r) * r;
        double v;
        if (fast) {
          const int qc = qcol[qj];
          const C0Val cz = c0_eval(cv.family, c0dx[fi * gx + qc] + c0dy[fi * gy + qrow[qj]],
                                   cv.nonstat ? c0gp[fi] * c0gq[qc] : cv.sigma2);
          v = cz.v;
          if (lf.dc) {   // (dC0/dsigma2, dC0/dkappa)
            const double ea = cz.e * cz.a * cv.ik;
            *reinterpret_cast<double2*>(lf.dc + 2 * ((t0 + fi) * Mr + l * r + qj)) =
                make_double2(v * is2, cv.family == 0 ? ea : ea * cz.a);
          }
        } else if (lf.dc) {
          double d1, d2;
          v = cov0_d(cv, sx[fi], sy[fi], ax[qj], ay[qj], d1, d2);
          *reinterpret_cast<double2*>(lf.dc + 2 * ((t0 + fi) * Mr + l * r + qj)) = make_double2(d1, d2);
        } else {
          v = cov0(cv, sx[fi], sy[fi], ax[qj], ay[qj]);
        }
        Hrow[(long)fi * Mr + l * r + qj] = v;
        if (l == 0) atomicMax(xsc + fi, xexp_of(v));
      }
      acc.zero();
      __syncthreads();
      if (l > 0) {
        const int* vsa = st.vexp[l] + a * (long)((l * r + 127) / 128) * r;
        ok = eng.mma(acc, Hseg, Mr, 1, nr, Vanc, l * r, 1, r, l * r, hsc + ra, TC_M, vsa, r);
        if (!ok) break;
        if (row < nr) {
          int e = -2000;
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int col = c0 + c;
            if (col < r) {
              const double v = Hseg[(long)row * Mr + l * r + col] - acc.v[c];
              Hseg[(long)row * Mr + l * r + col] = v;
              e = max(e, xexp_of(v));
            }
          }
          atomicMax(xsc + ra + row, e);
        }
      }
      __syncthreads();
      acc.zero();
      ok = eng.mma(acc, Hseg + l * r, Mr, 1, nr, st.Li[l] + a * (long)r * r, r, 1, r, r, xsc + ra, 0,
                   st.liexp[l] + a * r, 0);
      if (!ok) break;
      if (row < nr) {
        int e0 = -2000, e1 = -2000;       // a thread's 32 columns touch at most two groups
        const int gbase = (l * r + c0) / 128;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < r) {
            Hseg[(long)row * Mr + l * r + col] = acc.v[c];
            const int e = xexp_of(acc.v[c]);
            if ((l * r + col) / 128 == gbase) e0 = max(e0, e);
            else e1 = max(e1, e);
          }
        }
        atomicMax(hsc + gbase * TC_M + ra + row, e0);
        if (e1 > -2000) atomicMax(hsc + (gbase + 1) * TC_M + ra + row, e1);
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < na * ng; t += NT) {
      const int i = t / ng, g = t - i * ng;
      lf.hrow[(t0 + i) * ng + g] = hsc[g * TC_M + i];
    }
    if (lf.vfexp) {   // gradient calls: column scales of V_F over each region's tile (the leaf partials' operand)
      for (int g = 0; g < G; ++g) {
        const int ra = G > 1 ? gseg[g] : 0, rb = G > 1 ? gseg[g + 1] : na;
        int32_t* out = lf.vfexp + ((P + g) * 4 + (G > 1 ? 0 : (t0 - row0) / TC_M)) * (long)Mr;
        for (int c = threadIdx.x; c < Mr; c += NT) {
          int e = -2000;
          for (int i = ra; i < rb; ++i) e = max(e, xexp_of(Hrow[(long)i * Mr + c]));
          out[c] = e;
        }
      }
    }
  }
  eng.release();
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M - 1, P);
}

// chain_done (emulated form): V_F and its row scales were formed by
// chain_forward_kernel_em; the kernel starts at Sigma_F.  gcnt (emulated form
// with chain_done, else null): the work item is a group of gcnt[b] leaves with
// consecutive compact ids starting at it.i (children of one parent, at most
// LGRP_MAX, at most ds.lrows observations in all), stacked in one tile: their
// Sigma_F are the diagonal blocks of one block-diagonal matrix, factorised and
// inverted block by block (chol_seg, trinv_seg), and H = L^{-1} V_F is one
// product for all of them (the inverse is zero outside the blocks).
template <bool EMU>
__global__ void __launch_bounds__(NT) leaf_kernel_tc(const Desc* __restrict__ D, const int2* __restrict__ work,
                                                     int* status, int chain_done, const int* __restrict__ gcnt) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail, bad;
  __shared__ int rexp[EMU ? EM_REXP : 1], cexp[EMU ? EM_CEXP : 1];
  // emulation: row scales of H rows per 128-column group, of the current X^l block, of L_Sigma^{-1}
  __shared__ int hsc[EMU ? EM_GMAX * TC_M : 1], xsc[EMU ? TC_M : 1], ssc[EMU ? TC_M : 1];
  const Item it = work_item(work);
  const Desc& ds = D[it.d];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const double tau2 = ds.tau2;
  const int nlmax = max(ds.nlmax, ds.lrows);     // rows of the layout
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const long F = it.i;                           // compact leaf id (the group's first)
  const int G = EMU && gcnt ? gcnt[blockIdx.x] : 1;
  const long Fm = st.mort[M][F];
  const long o0 = lf.off[Fm];
  const int nF = (int)(lf.off[st.mort[M][F + G - 1] + 1] - o0);
  if (nF == 0) {
    if (threadIdx.x < G) { lf.d[F + threadIdx.x] = 0.0; lf.u[F + threadIdx.x] = 0.0; }
    return;
  }
  if (nF > nlmax) {                              // (a group larger than the layout: never formed by the host)
    if (threadIdx.x == 0) flag_error(status, ST_LIMIT, M, F);
    return;
  }
  const int lds = nlmax + 1;
  double* sx = reinterpret_cast<double*>(dsm + Engine<EMU>::STAGE);
  double* sy = sx + nlmax;
  double* sv = sy + nlmax;
  double* tmp = sv + nlmax;
  double* ax = tmp + nlmax;
  double* ay = ax + MAX_R_DEV;
  double* red = ay + MAX_R_DEV;                 // block sums (red[0..7]) or a group's pivots (red[0..3])
  double* S = red + 32;                         // nlmax x (nlmax + 1)
  // a group's leaves: rows gseg[k] .. gseg[k + 1] - 1, and the leaf of every row
  int* gseg = reinterpret_cast<int*>(red + 8);
  unsigned char* growb = reinterpret_cast<unsigned char*>(red + 16);
  static_assert(TC_M <= 16 * sizeof(double) && LGRP_MAX + 1 <= 8 * sizeof(double) / sizeof(int),
                "the group tables fit in red[8..31]");
  if (threadIdx.x == 0) {
    bad = 0;
    gseg[0] = 0;
    for (int k = 0; k < G; ++k) gseg[k + 1] = (int)(lf.off[st.mort[M][F + k] + 1] - o0);
  }
  __syncthreads();
  if (EMU)
    for (int t = threadIdx.x; t < nF; t += NT) growb[t] = (unsigned char)seg_block(gseg, G, t);
  Engine<EMU> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  for (int t = threadIdx.x; t < nF; t += NT) {
    sx[t] = lf.xs[o0 + t];
    sy[t] = lf.ys[o0 + t];
    sv[t] = lf.yv[o0 + t];
  }
  if (EMU)
    for (int t = threadIdx.x; t < EM_GMAX * TC_M; t += NT) hsc[t] = -2000;
  double* Hrow = lf.H + o0 * Mr;
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  if (EMU && chain_done) {
    const int ng = (Mr + EM_KG - 1) / EM_KG;
    __syncthreads();                             // after the reset of hsc above
    for (int t = threadIdx.x; t < nF * ng; t += NT) {
      const int i = t / ng, g = t - i * ng;
      hsc[g * TC_M + i] = lf.hrow[(o0 + i) * ng + g];
    }
  }
  // chain: V^l_F = (C0(S_F, Q_l) - sum_{k<l} V^k_F V^k_{R_l}') L_l^{-T}  (one 128-row tile)
  for (int l = 0; l < M && ok && !(EMU && chain_done); ++l) {
    const long a = ancestor(st, M, F, l);
    __syncthreads();
    load_knots(sh, l, st.mort[l][a], ax, ay);
    const double* Vanc = st.V[l] + a * (long)r * (l * r);
    if (EMU)
      for (int t = threadIdx.x; t < TC_M; t += NT) xsc[t] = -2000;
    __syncthreads();
    // C0(S_F, Q_l) into block l, spread over every warp; the product below
    // reads only blocks < l
    for (int t = threadIdx.x; t < nF * r; t += NT) {
      const int fi = t / r, qj = t - fi * r;
      const double v = cov0(cv, sx[fi], sy[fi], ax[qj], ay[qj]);
      Hrow[(long)fi * Mr + l * r + qj] = v;
      if (EMU && l == 0) atomicMax(xsc + fi, xexp_of(v));
    }
    acc.zero();
    __syncthreads();
    if (l > 0) {
      const int* vsa = EMU ? st.vexp[l] + a * (long)((l * r + 127) / 128) * r : nullptr;
      ok = eng.mma(acc, Hrow, Mr, 1, nF, Vanc, l * r, 1, r, l * r, hsc, TC_M, vsa, r);
      if (!ok) break;
      if (row < nF) {
        int e = -2000;
        #pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < r) {
            const double v = Hrow[(long)row * Mr + l * r + col] - acc.v[c];
            Hrow[(long)row * Mr + l * r + col] = v;
            e = max(e, xexp_of(v));
          }
        }
        if (EMU) atomicMax(xsc + row, e);
      }
    }
    __syncthreads();
    acc.zero();
    ok = eng.mma(acc, Hrow + l * r, Mr, 1, nF, st.Li[l] + a * (long)r * r, r, 1, r, r, xsc, 0,
                 EMU ? st.liexp[l] + a * r : nullptr, 0);
    if (!ok) break;
    if (row < nF) {
      int e0 = -2000, e1 = -2000;       // a thread's 32 columns touch at most two groups
      const int gbase = (l * r + c0) / 128;
      #pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) {
          Hrow[(long)row * Mr + l * r + col] = acc.v[c];
          const int e = xexp_of(acc.v[c]);
          if ((l * r + col) / 128 == gbase) e0 = max(e0, e);
          else e1 = max(e1, e);
        }
      }
      if (EMU) {
        atomicMax(hsc + gbase * TC_M + row, e0);
        if (e1 > -2000) atomicMax(hsc + (gbase + 1) * TC_M + row, e1);
      }
    }
  }
  __syncthreads();                             // points loaded, chain blocks written
  // Sigma_F = C0(S_F, S_F) - V_F V_F' + tau2 I (lower triangle), the
  // covariance by every warp first, then the product 64 columns at a time
  const bool fast = c0_fast_ok(cv, 1, 1);
  const double c0s = c0_scale(cv), c0s2 = c0s * c0s;
  static_assert(TC_M <= 2 * MAX_R_DEV, "the leaf's variance factors reuse ax and ay");
  double* lgq = ax;                              // the points' variance factors (ax, ay: 2 MAX_R_DEV >= nF doubles)
  if (fast && cv.nonstat) {
    for (int t = threadIdx.x; t < nF; t += NT) lgq[t] = c0_vfac(cv, sx[t]);
    __syncthreads();
  }
  int tri_all = 0;                               // lower triangles of the group's diagonal blocks
  for (int k = 0; k < G; ++k) tri_all += (gseg[k + 1] - gseg[k]) * (gseg[k + 1] - gseg[k] + 1) / 2;
  for (int t = threadIdx.x; t < tri_all; t += NT) {
    int b = 0, u = t;
    for (int c = gseg[1] * (gseg[1] + 1) / 2; u >= c; c = (gseg[b + 1] - gseg[b]) * (gseg[b + 1] - gseg[b] + 1) / 2) {
      u -= c;
      ++b;
    }
    int fi, fj;
    tri_decode(u, fi, fj);
    fi += gseg[b];
    fj += gseg[b];
    double v;
    if (fast) {
      const double dx = sx[fi] - sx[fj], dy = sy[fi] - sy[fj];
      v = c0_fast(cv.family, c0s2 * fma(dx, dx, dy * dy), cv.nonstat ? cv.sigma2 * lgq[fi] * lgq[fj] : cv.sigma2);
    } else {
      v = cov0(cv, sx[fi], sy[fi], sx[fj], sy[fj]);
    }
    S[fi * lds + fj] = v + (fi == fj ? tau2 : 0.0);
  }
  __syncthreads();
  const int nct = (nF + TC_N - 1) / TC_N;
  for (int ct = 0; ct < nct && ok && M > 0; ++ct) {
    const int ncol = min(TC_N, nF - ct * TC_N);
    acc.zero();
    ok = eng.mma(acc, Hrow, Mr, 1, nF, Hrow + (long)ct * TC_N * Mr, Mr, 1, ncol, Mr, hsc, TC_M,
                 hsc + ct * TC_N, TC_M);
    if (!ok) break;
    if (row < nF)
      #pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int oj = ct * TC_N + c0 + c;
        if (c0 + c < ncol && oj <= row && (G == 1 || oj >= gseg[growb[row]])) S[row * lds + oj] -= acc.v[c];
      }
  }
  double ld = 0.0, zz = 0.0;   // (a group: leaf k's in thread k)
  // the leaves' square blocks of S (n_k x n_k, row-major) to dst + sq_off of each leaf
  auto store_blocks = [&](double* dst) {
    int tot = 0;
    for (int k = 0; k < G; ++k) tot += (gseg[k + 1] - gseg[k]) * (gseg[k + 1] - gseg[k]);
    for (int t = threadIdx.x; t < tot; t += NT) {
      int b = 0, u = t;
      for (int c = gseg[1] * gseg[1]; u >= c; c = (gseg[b + 1] - gseg[b]) * (gseg[b + 1] - gseg[b])) {
        u -= c;
        ++b;
      }
      const int nb = gseg[b + 1] - gseg[b], i = u / nb, j = u - i * nb;
      dst[lf.sq_off[st.mort[M][F + b]] + u] = S[(gseg[b] + i) * lds + gseg[b] + j];
    }
  };
  // sum over the rows of leaf k of tmp (thread k)
  auto leaf_sum = [&]() {
    double v = 0.0;
    if (threadIdx.x < G)
      for (int i = gseg[threadIdx.x]; i < gseg[threadIdx.x + 1]; ++i) v += tmp[i];
    return v;
  };
  if (ok) {
    if (G == 1) {
      chol_smem(S, nF, lds, &bad);
      for (int t = threadIdx.x; t < nF; t += NT) ld += log(S[t * lds + t]);
      ld = 2.0 * block_sum(ld, red);
    } else {
      chol_seg(S, lds, gseg, G, &bad, red);
      for (int t = threadIdx.x; t < nF; t += NT) tmp[t] = log(S[t * lds + t]);
      __syncthreads();
      ld = 2.0 * leaf_sum();
    }
    if (lf.LSf) {
      if (G == 1) {
        double* Lf = lf.LSf + lf.sq_off[Fm];
        for (int t = threadIdx.x; t < nF * nF; t += NT) Lf[t] = S[(t / nF) * lds + (t % nF)];
      } else {
        store_blocks(lf.LSf);
      }
    }
    if (lf.VF)
      for (long t = threadIdx.x; t < (long)nF * Mr; t += NT) lf.VF[o0 * Mr + t] = Hrow[t];
    if (G == 1) trinv_smem(S, nF, lds, tmp);
    else trinv_seg(S, lds, gseg, G, tmp, red);
    if (EMU) {   // row scales of L_Sigma^{-1} (lower triangular) for the solve below
      for (int t = threadIdx.x; t < nF; t += NT) {
        int e = -2000;
        for (int q = G == 1 ? 0 : gseg[growb[t]]; q <= t; ++q) e = max(e, xexp_of(S[t * lds + q]));
        ssc[t] = e;
      }
    }
    if (G == 1) {
      double* LS = lf.LS + lf.sq_off[Fm];
      for (int t = threadIdx.x; t < nF * nF; t += NT) LS[t] = S[(t / nF) * lds + (t % nF)];
    } else {
      store_blocks(lf.LS);
    }
    for (int t = threadIdx.x; t < nF; t += NT) {
      double s = 0.0;
      for (int k = G == 1 ? 0 : gseg[growb[t]]; k <= t; ++k) s = fma(S[t * lds + k], sv[k], s);
      lf.z[o0 + t] = s;
      if (G == 1) zz = fma(s, s, zz);
      else tmp[t] = s * s;
    }
    if (G == 1) {
      zz = block_sum(zz, red);
    } else {
      __syncthreads();
      zz = leaf_sum();
    }
    // H^l = L_Sigma^{-1} V^l_F (whole block read before it is overwritten)
    int32_t* hcol = EMU ? lf.hcol + F * (long)Mr : nullptr;   // column scales of H_F for the Gram kernel
    if (EMU) {
      for (int t = threadIdx.x; t < G * Mr; t += NT) hcol[t] = -2000;   // (the group's leaves are consecutive)
      // hsc (the V_F row scales) is read no more: it collects the row scales of H_F
      for (int t = threadIdx.x; t < EM_GMAX * TC_M; t += NT) hsc[t] = -2000;
    }
    for (int cb = 0; cb < Mr && ok; cb += TC_N) {   // 64 columns of H a product (two levels at r = 32)
      const int nbc = min(TC_N, Mr - cb);
      acc.zero();
      ok = eng.mma(acc, S, lds, 1, nF, Hrow + cb, 1, Mr, nbc, nF, EMU ? ssc : nullptr, 0);
      if (!ok) break;
      if (row < nF) {
        int e0 = -2000, e1 = -2000;       // a thread's 32 columns touch at most two groups
        const int gbase = (cb + c0) / 128;
        #pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < nbc) {
            Hrow[(long)row * Mr + cb + col] = acc.v[c];
            const int e = xexp_of(acc.v[c]);
            if ((cb + col) / 128 == gbase) e0 = max(e0, e);
            else e1 = max(e1, e);
          }
        }
        if (EMU) {
          atomicMax(hsc + gbase * TC_M + row, e0);
          if (e1 > -2000) atomicMax(hsc + (gbase + 1) * TC_M + row, e1);
        }
      }
      if (EMU && G == 1 && ((threadIdx.x >> 5) & 3) * 32 < nF) {   // warp-uniform: the warp holds a kept row
        const int lane = threadIdx.x & 31;
        #pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int e = __reduce_max_sync(0xffffffffu, row < nF ? xexp_of(acc.v[c]) : -2000);
          if (lane == c && c0 + c < nbc && e > -2000) atomicMax(hcol + cb + c0 + c, e);
        }
      } else if (EMU && G > 1 && ((threadIdx.x >> 5) & 3) * 32 < nF) {   // per leaf: the lanes of each leaf reduce
        const int lane = threadIdx.x & 31;
        const int lk = row < nF ? (int)growb[row] : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, lk);
        #pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int e = __reduce_max_sync(grp, row < nF ? xexp_of(acc.v[c]) : -2000);
          if (lk >= 0 && lane == __ffs(grp) - 1 && c0 + c < nbc && e > -2000)
            atomicMax(hcol + (long)lk * Mr + cb + c0 + c, e);
        }
      }
      __syncthreads();
    }
    if (EMU && lf.hrow && ok) {   // row scales of H_F per 128-column group (the gradient's Hbar operand)
      const int ng = (Mr + EM_KG - 1) / EM_KG;
      for (int t = threadIdx.x; t < nF * ng; t += NT) {
        const int i = t / ng, g = t - i * ng;
        lf.hrow[(o0 + i) * ng + g] = hsc[g * TC_M + i];
      }
    }
  }
  eng.release();
  if (threadIdx.x < G) {
    lf.d[F + threadIdx.x] = ld;
    lf.u[F + threadIdx.x] = zz;
  }
  if (threadIdx.x == 0) {
    if (!ok) flag_error(status, ST_TIMEOUT, M, F);
    else if (bad) flag_error(status, ST_NOT_PD, M, F);
  }
}

// ---------------------------------------------------------------------------
// Gram products of the posterior pass on the emulation engine (MRA_PREC_EMU):
// leaf_syrk and aggregate with the same sums as the FP64 kernels.  One tile
// stacks up to S = 128 / r consecutive row blocks k0 .. k0 + S - 1 (all >= l)
// against CB = 64 / r column blocks l .. l + CB - 1 (one at r = 64), so the 128
// x 64 MMA carries S CB output blocks and the column blocks are split once for
// all of them.
// ---------------------------------------------------------------------------

// Tiles of the packed lower blocks (k >= l, k, l < nblk) for stack height S and
// CB column blocks per tile: the tile of column blocks l .. l + CB - 1 and row
// blocks k0 .. k0 + S - 1 (k0 >= l) keeps the blocks with k >= its column block.
__host__ __device__ inline int em_tiles(int nblk, int S, int CB = 1) {
  int n = 0;
  for (int l = 0; l < nblk; l += CB) n += (nblk - l + S - 1) / S;
  return n;
}

// Tile t -> first column block l (of CB) and first row block k0.
__device__ inline bool em_tile(int t, int nblk, int S, int CB, int& l, int& k0) {
  for (l = 0; l < nblk; l += CB) {
    const int nt = (nblk - l + S - 1) / S;
    if (t < nt) {
      k0 = l + t * S;
      return true;
    }
    t -= nt;
  }
  return false;
}

// Column blocks of r columns a tile takes: the 64 columns of the MMA (one block
// at r = 64, two at r = 32, four at r = 16).
__host__ __device__ inline int em_cblocks(int r) { return r <= 16 ? 4 : (r <= 32 ? 2 : 1); }

// One column block per tile (r > 32).  (A separate kernel: the same body
// compiled as a branch of the several-block kernel below ran 10 % slower.)
__global__ void __launch_bounds__(NT) leaf_syrk_kernel_em1(const Desc* __restrict__ D, const int2* __restrict__ work,
                                                          int nt, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  int tile;
  const Item it = work_item_tiled(work, nt, tile);
  const Desc& ds = D[it.d];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const long p = it.i;
  const int S = em_stack(r);
  int l, k0;
  if (!em_tile(tile, M, S, 1, l, k0)) return;     // fewer tiles in a shallower dataset
  const int nk = min(S, M - k0);                      // row blocks k0 .. k0 + nk - 1
  const long pm = st.mort[M - 1][p];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const int K = (int)(row1 - row0);
  const double* Hb = lf.H + row0 * Mr;
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  // scales per 128-row group of the parent's rows: the largest column scale of
  // the leaves whose rows meet the group (an upper bound of the group's maximum)
  const int ng = (K + EM_KG - 1) / EM_KG;
  for (int t = threadIdx.x; t < ng * (TC_M + TC_N); t += NT) {
    const bool isA = t < ng * TC_M;
    const int u = isA ? t : t - ng * TC_M;
    const int g = isA ? u / TC_M : u / TC_N, i = isA ? u % TC_M : u % TC_N;
    int e = -2000;
    if (i < (isA ? nk * r : r)) {
      const int col = isA ? k0 * r + i : l * r + i;
      for (int c = 0; c < (1 << leaf_bits(ds.sh)); ++c) {
        const long lo = lf.off[(pm << leaf_bits(ds.sh)) + c] - row0, hi = lf.off[(pm << leaf_bits(ds.sh)) + c + 1] - row0;
        if (hi > lo && lo < (long)(g + 1) * EM_KG && hi > (long)g * EM_KG) {
          const int cl = st.cid[M][(pm << leaf_bits(ds.sh)) + c];
          e = max(e, lf.hcol[(long)cl * Mr + col]);
        }
      }
    }
    (isA ? rexp : cexp)[u] = e;
  }
  __syncthreads();
  TcAcc acc;
  acc.zero();
  const bool ok = eng.mma(acc, Hb + k0 * r, 1, Mr, nk * r, Hb + l * r, 1, Mr, r, K, rexp, TC_M, cexp, TC_N);
  const int m = M - 1, T = (m + 1) * (m + 2) / 2;
  const int row = acc.row(), c0 = acc.col0();
  if (ok && row < nk * r) {
    const int k = k0 + row / r, ri = row % r;
    double* out = st.Acc[m] + (p * T + tri_index(k, l)) * (long)r * r + (long)ri * r;
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c0 + c < r) out[c0 + c] = acc.v[c];
  }
  eng.release();
  if (k0 == l) {
    double* om = st.Om[m] + (p * (m + 1) + l) * (long)r;
    for (int a = threadIdx.x; a < r; a += NT) {
      double s = 0.0;
      for (long o = 0; o < K; ++o) s = fma(Hb[o * Mr + l * r + a], lf.z[row0 + o], s);
      om[a] = s;
    }
  }
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M - 1, p);
}

// Several column blocks per tile (r <= 32).
template <bool MULTI>
__global__ void __launch_bounds__(NT) leaf_syrk_kernel_em(const Desc* __restrict__ D, const int2* __restrict__ work,
                                                          int nt, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  int tile;
  const Item it = work_item_tiled(work, nt, tile);
  const Desc& ds = D[it.d];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const long p = it.i;
  const int S = em_stack(r), CB = MULTI ? em_cblocks(r) : 1;
  int l, k0;
  if (!em_tile(tile, M, S, CB, l, k0)) return;  // fewer tiles in a shallower dataset
  const int nk = min(S, M - k0);                      // row blocks k0 .. k0 + nk - 1
  const int nl = MULTI ? min(CB, M - l) : 1;          // column blocks l .. l + nl - 1
  const long pm = st.mort[M - 1][p];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const int K = (int)(row1 - row0);
  const double* Hb = lf.H + row0 * Mr;
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  // scales per 128-row group of the parent's rows: the largest column scale of
  // the leaves whose rows meet the group (an upper bound of the group's maximum)
  const int ng = (K + EM_KG - 1) / EM_KG;
  for (int t = threadIdx.x; t < ng * (TC_M + TC_N); t += NT) {
    const bool isA = t < ng * TC_M;
    const int u = isA ? t : t - ng * TC_M;
    const int g = isA ? u / TC_M : u / TC_N, i = isA ? u % TC_M : u % TC_N;
    int e = -2000;
    if (i < (isA ? nk * r : nl * r)) {
      const int col = isA ? k0 * r + i : l * r + i;
      for (int c = 0; c < (1 << leaf_bits(ds.sh)); ++c) {
        const long lo = lf.off[(pm << leaf_bits(ds.sh)) + c] - row0, hi = lf.off[(pm << leaf_bits(ds.sh)) + c + 1] - row0;
        if (hi > lo && lo < (long)(g + 1) * EM_KG && hi > (long)g * EM_KG) {
          const int cl = st.cid[M][(pm << leaf_bits(ds.sh)) + c];
          e = max(e, lf.hcol[(long)cl * Mr + col]);
        }
      }
    }
    (isA ? rexp : cexp)[u] = e;
  }
  __syncthreads();
  TcAcc acc;
  acc.zero();
  const bool ok = eng.mma(acc, Hb + k0 * r, 1, Mr, nk * r, Hb + l * r, 1, Mr, nl * r, K, rexp, TC_M, cexp, TC_N);
  const int m = M - 1, T = (m + 1) * (m + 2) / 2;
  const int row = acc.row(), c0 = acc.col0();
  if (ok && row < nk * r) {
    const int k = k0 + row / r, ri = row % r;
    if (!MULTI) {                                     // (r > 32: one column block)
      double* out = st.Acc[m] + (p * T + tri_index(k, l)) * (long)r * r + (long)ri * r;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < r) out[c0 + c] = acc.v[c];
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c, lb = l + col / r;     // column block of this column
        if (col < nl * r && k >= lb)
          st.Acc[m][(p * T + tri_index(k, lb)) * (long)r * r + (long)ri * r + col % r] = acc.v[c];
      }
    }
  }
  eng.release();
  if (k0 == l)
    for (int lb = l; lb < l + nl; ++lb) {
      double* om = st.Om[m] + (p * (m + 1) + lb) * (long)r;
      for (int a = threadIdx.x; a < r; a += NT) {
        double s = 0.0;
        for (long o = 0; o < K; ++o) s = fma(Hb[o * Mr + lb * r + a], lf.z[row0 + o], s);
        om[a] = s;
      }
    }
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M - 1, p);
}

template <bool MULTI>
__global__ void __launch_bounds__(NT) aggregate_kernel_em(int m, const Desc* __restrict__ D,
                                                          const int2* __restrict__ work, int nt, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  int tile;
  const Item it = work_item_tiled(work, nt, tile);
  const Desc& ds = D[it.d];
  const int r = ds.sh.r, mr = m * r;
  const LevelState& st = ds.st;
  const long p = it.i;
  const int S = em_stack(r), CB = MULTI ? em_cblocks(r) : 1;
  int l, k0;
  if (!em_tile(tile, m, S, CB, l, k0)) return;
  const int nk = min(S, m - k0);
  const int nl = MULTI ? min(CB, m - l) : 1;
  const int Tc = (m + 1) * (m + 2) / 2, Tp = m * (m + 1) / 2;
  const long cf = st.cfirst[m - 1][p], cc = st.ccnt[m - 1][p];
  const double* Gb = st.G[m] + cf * (long)r * mr;
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  // scales per 128-row group of the stacked children (r rows each): the
  // largest column scale of the children whose rows meet the group
  const int K = (int)(cc * r), ng = (K + EM_KG - 1) / EM_KG;
  for (int t = threadIdx.x; t < ng * (TC_M + TC_N); t += NT) {
    const bool isA = t < ng * TC_M;
    const int u = isA ? t : t - ng * TC_M;
    const int g = isA ? u / TC_M : u / TC_N, i = isA ? u % TC_M : u % TC_N;
    int e = -2000;
    if (i < (isA ? nk * r : nl * r)) {
      const int col = isA ? k0 * r + i : l * r + i;
      for (long ch = 0; ch < cc; ++ch)
        if (ch * r < (long)(g + 1) * EM_KG && (ch + 1) * r > (long)g * EM_KG)
          e = max(e, st.gcol[m][(cf + ch) * (long)mr + col]);
    }
    (isA ? rexp : cexp)[u] = e;
  }
  __syncthreads();
  TcAcc acc;
  acc.zero();
  const bool ok = eng.mma(acc, Gb + k0 * r, 1, mr, nk * r, Gb + l * r, 1, mr, nl * r, K, rexp, TC_M, cexp, TC_N);
  const int row = acc.row(), c0 = acc.col0();
  if (ok && row < nk * r) {
    const int k = k0 + row / r, ri = row % r;
    if (!MULTI) {                                     // (r > 32: one column block)
      const int t = tri_index(k, l);
      double* out = st.Acc[m - 1] + (p * Tp + t) * (long)r * r + (long)ri * r;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (col < r) {
          double s = -acc.v[c];
          for (long ch = cf; ch < cf + cc; ++ch) s += st.Acc[m][(ch * Tc + t) * (long)r * r + (long)ri * r + col];
          out[col] = s;
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c, lb = l + col / r, cj = col % r;   // column block and column
        if (col < nl * r && k >= lb) {
          const int t = tri_index(k, lb);
          double s = -acc.v[c];
          for (long ch = cf; ch < cf + cc; ++ch) s += st.Acc[m][(ch * Tc + t) * (long)r * r + (long)ri * r + cj];
          st.Acc[m - 1][(p * Tp + t) * (long)r * r + (long)ri * r + cj] = s;
        }
      }
    }
  }
  eng.release();
  if (k0 == l)
    for (int lb = l; lb < l + nl; ++lb) {
      double* om = st.Om[m - 1] + (p * m + lb) * (long)r;
      for (int a = threadIdx.x; a < r; a += NT) {
        double s = 0.0;
        for (long ci = cf; ci < cf + cc; ++ci) {
          s += st.Om[m][(ci * (m + 1) + lb) * (long)r + a];
          const double* Gc = st.G[m] + ci * (long)r * mr;
          const double* gc = st.gv[m] + ci * r;
          for (int q = 0; q < r; ++q) s = fma(-Gc[(long)q * mr + lb * r + a], gc[q], s);
        }
        om[a] = s;
      }
    }
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, m - 1, p);
}


template <bool EMU>
static size_t prior_tc_smem(int rcap) {     // knots (2 rcap), ancestor knots, scratch (rcap), W (rcap x (r + 1))
  const size_t b = Engine<EMU>::STAGE + sizeof(double) * (3 * (size_t)rcap + 2 * MAX_R_DEV +
                                                          (size_t)rcap * (MAX_R_DEV + 1));
  return EMU ? std::max(b, EM_SOLO_SMEM) : b;
}
template <bool EMU>
static size_t leaf_tc_smem(int nlmax) {
  const size_t b =
      Engine<EMU>::STAGE + sizeof(double) * (4 * (size_t)nlmax + 2 * MAX_R_DEV + 32 + (size_t)nlmax * (nlmax + 1));
  return EMU ? std::max(b, EM_SOLO_SMEM) : b;
}
// Dynamic plus (an upper bound of) static shared memory of the leaf kernel.
size_t leaf_tc_smem_bytes(int nlmax, int emu) {
  return emu ? 1024 + sizeof(int) * (EM_REXP + EM_CEXP + EM_GMAX * TC_M + 2 * TC_M) + leaf_tc_smem<true>(nlmax)
             : 1024 + leaf_tc_smem<false>(nlmax);
}


cudaError_t launch_prior_tc(int m, const Desc* d_desc, const int2* work, int nblocks, int emu, int* status,
                            cudaStream_t s, const int* gcnt, int rcap) {
  cudaError_t e;
  rcap = gcnt ? std::max(rcap, MAX_R_DEV) : MAX_R_DEV;
  if (rcap > TC_M) return cudaErrorInvalidValue;
  if (emu) {
    const size_t sm = prior_tc_smem<true>(rcap);
    if ((e = cudaFuncSetAttribute(prior_level_kernel_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    prior_level_kernel_tc<true><<<nblocks, NT, sm, s>>>(m, d_desc, work, status, gcnt, rcap);
  } else {
    const size_t sm = prior_tc_smem<false>(rcap);
    if ((e = cudaFuncSetAttribute(prior_level_kernel_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)))
      return e;
    prior_level_kernel_tc<false><<<nblocks, NT, sm, s>>>(m, d_desc, work, status, gcnt, rcap);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_tc(const Desc* d_desc, const int2* work, int nblocks, int nlmax, int emu, int* status,
                           cudaStream_t s, const int2* w_par, int n_par, Timer* tm, int leaf_level, const int* gcnt,
                           int lrows, const int* gpar) {
  cudaError_t e;
  if (emu) {
    // the chain per parent first (work list: the level-(M-1) regions of every dataset)
    const int chain_done = n_par > 0;
    if (chain_done) {
      if ((e = cudaFuncSetAttribute(gpar ? chain_forward_kernel_em<true> : chain_forward_kernel_em<false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM)))
        return e;
      if (gpar) chain_forward_kernel_em<true><<<n_par, NT, EM_SOLO_SMEM, s>>>(d_desc, w_par, status, gpar);
      else chain_forward_kernel_em<false><<<n_par, NT, EM_SOLO_SMEM, s>>>(d_desc, w_par, status, nullptr);
      if ((e = cudaGetLastError())) return e;
      if (tm) {   // the chain and the leaf kernel are timed as two records
        tm->stop(s);
        tm->start(1, s, 2, leaf_level);
      }
    }
    if (gcnt && !chain_done) return cudaErrorInvalidValue;   // (groups need the per-parent chain kernel)
    const size_t sm = leaf_tc_smem<true>(std::max(nlmax, chain_done ? lrows : 0));
    if ((e = cudaFuncSetAttribute(leaf_kernel_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    leaf_kernel_tc<true><<<nblocks, NT, sm, s>>>(d_desc, work, status, chain_done, chain_done ? gcnt : nullptr);
  } else {
    const size_t sm = leaf_tc_smem<false>(nlmax);
    if ((e = cudaFuncSetAttribute(leaf_kernel_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
    leaf_kernel_tc<false><<<nblocks, NT, sm, s>>>(d_desc, work, status, 0, nullptr);
  }
  return cudaGetLastError();
}

cudaError_t launch_leaf_syrk_em(const Desc* d_desc, const int2* work, int nblocks, int maxM, int r, int* status,
                                cudaStream_t s) {
  cudaError_t e;
  const bool multi = em_cblocks(r) > 1;
  if ((e = cudaFuncSetAttribute(multi ? leaf_syrk_kernel_em<true> : leaf_syrk_kernel_em1,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM)))
    return e;
  const int nt = em_tiles(maxM, em_stack(r), em_cblocks(r));
  if (multi) leaf_syrk_kernel_em<true><<<nblocks * nt, NT, EM_SOLO_SMEM, s>>>(d_desc, work, nt, status);
  else leaf_syrk_kernel_em1<<<nblocks * nt, NT, EM_SOLO_SMEM, s>>>(d_desc, work, nt, status);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gradient, emulated form: the adjoint of H_F = L_Sigma^{-1} V_F of every leaf,
//     Hbar_F = 2 H_F S + z_F omegabar',
// where S (M r x M r) is the symmetric adjoint of Ahat along the leaf's
// ancestor chain and omegabar that of omegahat (Sec. 3.2 quantities in the
// whitened basis).  S and omegabar are the same for all children of one
// level-(M-1) region, so the product runs per parent over the parent's
// contiguous rows of H, in tiles of 128 rows, on the emulation engine.
// ---------------------------------------------------------------------------

// One CTA per region p of level L: St_p[l r + j][k r + kk] = S^{k,l}[kk][j],
// k, l <= L (the operand rows of the products with S, K contiguous), assembled
// from the row blocks of the adjoints of p and its ancestors, and the exponent
// of every row of St_p per 128-column group (the engine's B scales).
__global__ void __launch_bounds__(NT) s_full_kernel(int L, const Desc* __restrict__ D, GradState gs) {
  extern __shared__ double tile[];                       // r x (r + 1): one transposed block
  const Desc& ds = D[0];
  const int M = L + 1, r = ds.sh.r, Mr = M * r, ng = (Mr + EM_KG - 1) / EM_KG;
  int* sexp = reinterpret_cast<int*>(tile + r * (r + 1));   // [group][row] exponents
  const LevelState& st = ds.st;
  const long p = gs.rbase + blockIdx.x;
  const int lane = threadIdx.x & 31;
  long anc[MAXL];
  for (int l = 0; l < M; ++l) anc[l] = ancestor(st, L, p, l);
  for (int t = threadIdx.x; t < ng * Mr; t += NT) sexp[t] = -2000;
  double* St = gs.SF + p * (long)Mr * Mr;
  for (int k = 0; k < M; ++k)
    for (int l = 0; l < M; ++l) {
      const SRef b = sblock(gs, anc, r, k, l);   // B(j, kk) = b.p[j * b.sj + kk * b.sk]
      const bool tr = b.sk != 1;                 // then b.sj == 1: read along j, transpose in shared memory
      __syncthreads();                           // previous block's tile and the scale reset are done
      if (tr)
        for (int t = threadIdx.x; t < r * r; t += NT) {
          const int kk = t / r, j = t - kk * r;
          tile[kk * (r + 1) + j] = b.p[j + (long)kk * b.sk];
        }
      __syncthreads();
      for (int t0 = 0; t0 < r * r; t0 += NT) {   // uniform trip count: the warp intrinsics see full warps
        const int t = t0 + threadIdx.x;
        const bool ok = t < r * r;
        const int j = ok ? t / r : 0, kk = ok ? t - j * r : 0;
        const double v = !ok ? 0.0 : tr ? tile[kk * (r + 1) + j] : b.p[(long)j * b.sj + kk];
        const int R = l * r + j, C = k * r + kk;
        if (ok) St[(long)R * Mr + C] = v;
        const int key = ok ? (C / EM_KG) * Mr + R : -1;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int e = __reduce_max_sync(grp, ok ? em_exp(v) : -2000);
        if (ok && lane == __ffs(grp) - 1) atomicMax(&sexp[key], e);
      }
    }
  __syncthreads();
  int32_t* E = gs.SFexp + p * (long)ng * Mr;
  for (int t = threadIdx.x; t < ng * Mr; t += NT) E[t] = sexp[t];
}

// One CTA per (level-(M-1) region p, column block l), l fastest: column block l of Hbar for all rows under p.
__global__ void __launch_bounds__(NT) hbar_kernel_em(const Desc* __restrict__ D, GradState gs, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  __shared__ int hsc[EM_GMAX * TC_M];            // row scales of the current 128 rows of H per group
  __shared__ double wb[MAX_R_DEV];               // omegabar of block l
  const Desc& ds = D[0];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r, ng = (Mr + EM_KG - 1) / EM_KG;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const long p = gs.rbase + blockIdx.x / M;    // the M column blocks of one region run together
  const int l = (int)(blockIdx.x % M);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long pm = st.mort[M - 1][p];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const long al = ancestor(st, M - 1, p, l);
  for (int t = threadIdx.x; t < r; t += NT) wb[t] = gs.Obar[l][al * r + t];
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  const double* Sl = gs.SF + p * (long)Mr * Mr + (long)l * r * Mr;
  const int* Se = gs.SFexp + p * (long)ng * Mr + l * r;
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  for (long t0 = row0; t0 < row1 && ok; t0 += TC_M) {
    const int na = (int)min((long)TC_M, row1 - t0);
    const double* Ht = lf.H + t0 * Mr;
    __syncthreads();                             // the previous tile's scales are no longer read
    if (lf.hrow) {                               // exported by the leaf kernel
      for (int t = threadIdx.x; t < TC_M * ng; t += NT) {
        const int i = t / ng, g = t - i * ng;
        hsc[g * TC_M + i] = i < na ? lf.hrow[(t0 + i) * ng + g] : -2000;
      }
    } else {
      for (int i = warp; i < TC_M; i += NT / 32)
        for (int g = 0; g < ng; ++g) {
          int e = -2000;
          if (i < na)
            for (int c = g * EM_KG + lane; c < min(Mr, (g + 1) * EM_KG); c += 32)
              e = max(e, em_exp(Ht[(long)i * Mr + c]));
          e = __reduce_max_sync(0xffffffffu, e);
          if (lane == 0) hsc[g * TC_M + i] = e;
        }
    }
    __syncthreads();
    ok = eng.mma(acc, Ht, Mr, 1, na, Sl, Mr, 1, r, Mr, hsc, TC_M, Se, Mr);
    if (ok && row < na) {
      const double zr = lf.z[t0 + row];
      double* out = gs.HB + (t0 + row) * Mr + l * r;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < r) out[c0 + c] = 2.0 * acc.v[c] + zr * wb[c0 + c];
    }
  }
  eng.release();
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M, p);
}

// Leaf partials on the emulation engine: for parent p and k <= l <= M-1,
//   k < l : -sum over p's rows of Xbar^l' V^k_F,   k = l : sum of Vbar^l' V^l_F
// (the FP64 leaf_partial_kernel's tiles).  Per column block k, the diagonal
// tile (operand Vbar) runs alone and the tiles l > k (operand Xbar, adjacent
// columns) are stacked em_stack(r) high.
__global__ void __launch_bounds__(NT) leaf_partial_kernel_em(const Desc* __restrict__ D, GradState gs, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  const Desc& ds = D[0];
  const int M = ds.sh.M, r = ds.sh.r, Mr = M * r, T = M * (M + 1) / 2;
  const LeafState& lf = ds.lf;
  const int nt = partial_tiles(M, em_stack(r));
  const long p = gs.rbase + blockIdx.x / nt;
  int k, l0, nl;
  if (!partial_tile((int)(blockIdx.x % nt), M, em_stack(r), k, l0, nl)) return;
  const bool diag = l0 == k;
  const long pm = ds.st.mort[M - 1][p];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  const int K = (int)(row1 - row0);
  const double* A = (diag ? gs.VBF : gs.XBF) + row0 * Mr + l0 * r;
  const double* B = lf.VF + row0 * Mr + k * r;
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  TcAcc acc;
  // operand scales per 128-row group from the chain kernels, when they exported them
  const bool tab = gs.VFexp != nullptr;
  const long tb = p * 4 * (long)Mr;
  const bool ok = eng.mma(acc, A, 1, Mr, nl * r, B, 1, Mr, r, K,
                          tab ? (diag ? gs.VBexp : gs.XBexp) + tb + l0 * r : nullptr, Mr,
                          tab ? gs.VFexp + tb + k * r : nullptr, Mr);
  const int row = acc.row(), c0 = acc.col0();
  if (ok && row < nl * r) {
    const int l = l0 + row / r, i = row % r;
    const double sg = diag ? 1.0 : -1.0;
    double* out = gs.PartLeaf + (p * T + tri_index(l, k)) * (long)r * r + (long)i * r;
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c0 + c < r) out[c0 + c] = sg * acc.v[c];
  }
  eng.release();
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, M - 1, p);
}

cudaError_t launch_leaf_partial_em(const Desc& hd, const Desc* d_desc, const GradState& gs, int* status,
                                   cudaStream_t s, long nregions) {
  const int M = hd.sh.M, r = hd.sh.r;
  const int np = nregions < 0 ? hd.st.nreg[M - 1] : (int)nregions;
  if (np == 0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(leaf_partial_kernel_em, cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM)))
    return e;
  leaf_partial_kernel_em<<<np * partial_tiles(M, em_stack(r)), NT, EM_SOLO_SMEM, s>>>(d_desc, gs, status);
  return cudaGetLastError();
}

// Chain adjoint of the leaves on the emulation engine.  The forward chain
// V^l_F = (C0(Q_F, Q_{a_l}) - sum_{k<l} V^k_F V^k_{a_l}') L_{a_l}^{-T} reverses,
// for l = M-1..0, to
//   Xbar^l = Vbar^l L_{a_l}^{-1}   (C0 terms: Xbar^l_{o,j} dC0(s_o, q_j)/dtheta),
//   Vbar^k -= Xbar^l V^k_{a_l},    k < l,
// row by row; the ancestors a_l (l < M) are shared by all children of one
// level-(M-1) region, so one CTA takes the region's contiguous rows in tiles of
// 128.  Its C0 terms go to gradient slot slot0 + p.
__global__ void __launch_bounds__(NT) chain_adjoint_kernel_em(const Desc* __restrict__ D, GradState gs, long slot0,
                                                              int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  __shared__ double ax[MAX_R_DEV], ay[MAX_R_DEV], red[32];
  // row scales (one 64-column block = one group) of the tile's Vbar blocks and of the current Xbar block
  __shared__ int vbsc[MAXL * TC_M], xbsc[TC_M];
  const Desc& ds = D[0];
  const Shape sh = ds.sh;
  const Cov cv = ds.cv;
  const int M = sh.M, r = sh.r, Mr = M * r;
  const LevelState& st = ds.st;
  const LeafState& lf = ds.lf;
  const long p = gs.rbase + blockIdx.x;
  const long pm = st.mort[M - 1][p];
  const long row0 = lf.off[pm << leaf_bits(ds.sh)], row1 = lf.off[(pm + 1) << leaf_bits(ds.sh)];
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  TcAcc acc;
  const int row = acc.row(), c0 = acc.col0();
  double g_s2 = 0.0, g_k = 0.0, g_nu = 0.0;
  bool ok = true;
  for (long t0 = row0; t0 < row1 && ok; t0 += TC_M) {
    const int na = (int)min((long)TC_M, row1 - t0);
    double* VB = gs.VBF + t0 * Mr;
    double* XB = gs.XBF + t0 * Mr;
    const double so_x = row < na ? lf.xs[t0 + row] : 0.0, so_y = row < na ? lf.ys[t0 + row] : 0.0;
    const bool tab = st.licol[0] != nullptr;     // column scales of the ancestors' L^{-1} and V
    __syncthreads();                             // the previous tile's scales are no longer read
    {   // row scales of Vbar^{M-1} (as the leaf adjoint left it): one warp per row
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int i = warp; i < TC_M; i += NT / 32) {
        int e = -2000;
        if (i < na)
          for (int c = lane; c < r; c += 32) e = max(e, xexp_of(VB[(long)i * Mr + (M - 1) * r + c]));
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) vbsc[(M - 1) * TC_M + i] = e;
      }
    }
    for (int l = M - 1; l >= 0 && ok; --l) {
      const long a = ancestor(st, M - 1, p, l);
      const double* Lia = st.Li[l] + a * (long)r * r;
      const double* Va = st.V[l] + a * (long)r * (l * r);
      __syncthreads();                           // the previous level's knots and Xbar scales are no longer read
      load_knots(sh, l, st.mort[l][a], ax, ay);
      for (int t = threadIdx.x; t < TC_M; t += NT) {
        xbsc[t] = -2000;
        if (l > 0) vbsc[(l - 1) * TC_M + t] = -2000;   // block l - 1 takes its last update at this level
      }
      __syncthreads();
      ok = eng.mma(acc, VB + l * r, Mr, 1, na, Lia, 1, r, r, r, vbsc + l * TC_M, 0,
                   tab ? st.licol[l] + a * r : nullptr, 0);
      if (ok && row < na) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = c0 + c;
          if (col < r) {
            const double xb = acc.v[c];
            XB[(long)row * Mr + l * r + col] = xb;
            double d1, d2, d3 = 0.0;
            if (lf.dc) {   // stored by the forward chain kernel (families without d/dnu)
              const double2 dd = *reinterpret_cast<const double2*>(lf.dc + 2 * ((t0 + row) * Mr + l * r + col));
              d1 = dd.x;
              d2 = dd.y;
            } else {
              dcov0(cv, so_x, so_y, ax[col], ay[col], d1, d2, d3);
            }
            g_s2 = fma(xb, d1, g_s2);
            g_k = fma(xb, d2, g_k);
            g_nu = fma(xb, d3, g_nu);
          }
        }
        int e = -2000;   // row scale of Xbar^l (two threads per row)
#pragma unroll
        for (int c = 0; c < 32; ++c)
          if (c0 + c < r) e = max(e, xexp_of(acc.v[c]));
        atomicMax(xbsc + row, e);
      }
      // (the next product's scale pass opens with a barrier: Xbar^l is complete)
      for (int k = 0; k < l && ok; ++k) {
        ok = eng.mma(acc, XB + l * r, Mr, 1, na, Va + k * r, 1, l * r, r, r, xbsc, 0,
                     tab ? st.vcol[l] + a * (long)(l * r) + k * r : nullptr, 0);
        if (ok && row < na) {
          double* out = VB + (long)row * Mr + k * r;
          int e = -2000;
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (c0 + c < r) {
              const double v = out[c0 + c] - acc.v[c];
              out[c0 + c] = v;
              e = max(e, xexp_of(v));
            }
          if (k == l - 1) atomicMax(vbsc + k * TC_M + row, e);   // the last update of block k
        }
      }
    }
    if (ok && gs.VBexp) {   // column scales of the final Vbar_F and Xbar_F over the tile (leaf partials)
      __syncthreads();
      const long base = (p * 4 + (t0 - row0) / TC_M) * (long)Mr;
      for (int c = threadIdx.x; c < 2 * Mr; c += NT) {
        const double* X = c < Mr ? VB : XB;
        const int cc = c < Mr ? c : c - Mr;
        int e = -2000;
        for (int i = 0; i < na; ++i) e = max(e, xexp_of(X[(long)i * Mr + cc]));
        (c < Mr ? gs.VBexp : gs.XBexp)[base + cc] = e;
      }
    }
  }
  eng.release();
  g_s2 = block_sum(g_s2, red);
  g_k = block_sum(g_k, red);
  g_nu = block_sum(g_nu, red);
  if (threadIdx.x == 0) {
    gs.gpart[GP * (slot0 + p) + 0] = g_s2;
    gs.gpart[GP * (slot0 + p) + 1] = g_k;
    gs.gpart[GP * (slot0 + p) + 2] = 0.0;
    gs.gpart[GP * (slot0 + p) + 3] = g_nu;
    if (!ok) flag_error(status, ST_TIMEOUT, M - 1, p);
  }
}

cudaError_t launch_chain_adjoint_em(const Desc& hd, const Desc* d_desc, const GradState& gs, long slot0,
                                    int* status, cudaStream_t s, long nregions) {
  const int M = hd.sh.M;
  const int np = nregions < 0 ? hd.st.nreg[M - 1] : (int)nregions;
  if (np == 0) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(chain_adjoint_kernel_em, cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM)))
    return e;
  chain_adjoint_kernel_em<<<np, NT, EM_SOLO_SMEM, s>>>(d_desc, gs, slot0, status);
  return cudaGetLastError();
}

// St of the regions [gs.rbase, gs.rbase + n) of level L into gs.SF / gs.SFexp.
static cudaError_t launch_s_full(int L, const Desc& hd, const Desc* d_desc, const GradState& gs, cudaStream_t s,
                                 int n) {
  const int r = hd.sh.r, Mr = (L + 1) * r;
  const size_t sm = sizeof(double) * r * (r + 1) + sizeof(int) * ((Mr + EM_KG - 1) / EM_KG) * Mr;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(s_full_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm))) return e;
  s_full_kernel<<<n, NT, sm, s>>>(L, d_desc, gs);
  return cudaGetLastError();
}

cudaError_t launch_hbar_em(const Desc& hd, const Desc* d_desc, const GradState& gs, int* status, cudaStream_t s,
                           int64_t* launches, long nregions) {
  const int M = hd.sh.M;
  const int np = nregions < 0 ? hd.st.nreg[M - 1] : (int)nregions;
  if (np == 0) return cudaSuccess;
  cudaError_t e;
  if ((e = launch_s_full(M - 1, hd, d_desc, gs, s, np))) return e;
  if ((e = cudaFuncSetAttribute(hbar_kernel_em, cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM))) return e;
  hbar_kernel_em<<<np * M, NT, EM_SOLO_SMEM, s>>>(d_desc, gs, status);
  *launches += 2;
  return cudaGetLastError();
}

// Gbar of level m (1 <= m < M) on the emulation engine:
//     Gbar^l = -2 sum_k G^k S^{k,l} - g omegabar^l',  l < m,
// for all children of each level-(m-1) region P at once (they share P's chain
// S and omegabar; their rows of G are contiguous), from St_P assembled first.
__global__ void __launch_bounds__(NT) gbar_kernel_em(int m, const Desc* __restrict__ D, GradState gs, int* status) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int rexp[EM_REXP], cexp[EM_CEXP];
  __shared__ int gsc[EM_GMAX * TC_M];            // row scales of the current 128 rows of G per group
  __shared__ double wb[MAX_R_DEV];
  const Desc& ds = D[0];
  const int r = ds.sh.r, mr = m * r, ng = (mr + EM_KG - 1) / EM_KG;
  const LevelState& st = ds.st;
  const long P = gs.rbase + blockIdx.x / m;    // the m column blocks of one region run together
  const int l = (int)(blockIdx.x % m);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long row0 = (long)st.cfirst[m - 1][P] * r, row1 = row0 + (long)st.ccnt[m - 1][P] * r;
  const long al = ancestor(st, m - 1, P, l);
  for (int t = threadIdx.x; t < r; t += NT) wb[t] = gs.Obar[l][al * r + t];
  Engine<true> eng;
  eng.init(dsm, mbar, &tmem_slot, &fail, rexp, cexp);
  const double* Sl = gs.SF + P * (long)mr * mr + (long)l * r * mr;
  const int* Se = gs.SFexp + P * (long)ng * mr + l * r;
  TcAcc acc;
  bool ok = true;
  const int row = acc.row(), c0 = acc.col0();
  for (long t0 = row0; t0 < row1 && ok; t0 += TC_M) {
    const int na = (int)min((long)TC_M, row1 - t0);
    const double* Gt = st.G[m] + t0 * mr;
    __syncthreads();                             // the previous tile's scales are no longer read
    for (int i = warp; i < TC_M; i += NT / 32)
      for (int g = 0; g < ng; ++g) {
        int e = -2000;
        if (i < na)
          for (int c = g * EM_KG + lane; c < min(mr, (g + 1) * EM_KG); c += 32) e = max(e, em_exp(Gt[(long)i * mr + c]));
        e = __reduce_max_sync(0xffffffffu, e);
        if (lane == 0) gsc[g * TC_M + i] = e;
      }
    __syncthreads();
    ok = eng.mma(acc, Gt, mr, 1, na, Sl, mr, 1, r, mr, gsc, TC_M, Se, mr);
    if (ok && row < na) {
      const double gr = st.gv[m][t0 + row];
      double* out = gs.GB[m] + (t0 + row) * mr + l * r;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c0 + c < r) out[c0 + c] = -2.0 * acc.v[c] - gr * wb[c0 + c];
    }
  }
  eng.release();
  if (!ok && threadIdx.x == 0) flag_error(status, ST_TIMEOUT, m, P);
}

cudaError_t launch_gbar_em(int m, const Desc& hd, const Desc* d_desc, const GradState& gs, int* status,
                           cudaStream_t s, int64_t* launches, long nregions) {
  const int np = nregions < 0 ? hd.st.nreg[m - 1] : (int)nregions;
  if (np == 0) return cudaSuccess;
  cudaError_t e;
  if ((e = launch_s_full(m - 1, hd, d_desc, gs, s, np))) return e;
  if ((e = cudaFuncSetAttribute(gbar_kernel_em, cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM))) return e;
  gbar_kernel_em<<<np * m, NT, EM_SOLO_SMEM, s>>>(m, d_desc, gs, status);
  *launches += 2;
  return cudaGetLastError();
}

cudaError_t launch_aggregate_em(int m, int r, const Desc* d_desc, const int2* work, int nblocks, int* status,
                                cudaStream_t s) {
  cudaError_t e;
  const bool multi = em_cblocks(r) > 1;
  if ((e = cudaFuncSetAttribute(multi ? aggregate_kernel_em<true> : aggregate_kernel_em<false>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, EM_SOLO_SMEM)))
    return e;
  const int nt = em_tiles(m, em_stack(r), em_cblocks(r));
  if (multi) aggregate_kernel_em<true><<<nblocks * nt, NT, EM_SOLO_SMEM, s>>>(m, d_desc, work, nt, status);
  else aggregate_kernel_em<false><<<nblocks * nt, NT, EM_SOLO_SMEM, s>>>(m, d_desc, work, nt, status);
  return cudaGetLastError();
}

}  // namespace mra
