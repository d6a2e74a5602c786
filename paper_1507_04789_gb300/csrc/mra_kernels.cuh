// mra_kernels.cuh -- device-side state layout and kernel declarations.
//
// The GPU path works with the whitened form of the M-RA.  Along the ancestor
// chain R_0, ..., R_m of a region, the prior recursion of Eq. (priorw) is the
// block Cholesky factorisation of the chain covariance C0(Q_chain, Q_chain):
// with K_{R_l}^{-1} = W^l_{R_l} = L_l L_l', the blocks V^l_R = W^l_R L_l^{-T}
// satisfy W^k_R K_{R_k} W^k_{R_l}' = V^k_R V^k_{R_l}', so
//     V^l_R = (C0(Q_R, Q_{R_l}) - sum_{k<l} V^k_R V^k_{R_l}') L_l^{-T},
//     W^m_R = C0(Q_R, Q_R) - sum_{k<m} V^k_R V^k_R' = L_m L_m'.
// Basis weights are whitened, xi_l = L_l' eta_l ~ N(0, I), so B^l eta_l =
// V^l xi_l at the leaves, and the posterior quantities of Sec. 3.2 become
//     Ahat^{k,l} = L_k^{-1} A^{k,l} L_l^{-T},  omegahat^k = L_k^{-1} omega^k,
//     K~^{-1} = L_m (I + Ahat^{m,m}) L_m',
// so log|K~^{-1}| - log|K^{-1}| = log|I + Ahat^{m,m}| and
// omega' K~ omega = |Lt^{-1} omegahat^m|^2 with Lt Lt' = I + Ahat^{m,m}.
// The Sherman-Morrison-Woodbury updates of Eq. (helpquantities) keep their form:
//     Atilde^{k,l} = Ahat^{k,l} - G^k' G^l,  G^l = Lt^{-1} Ahat^{m,l}.
// The d and u of every region (Sec. 3.3) are basis-independent and equal the
// paper's.  I + Ahat has all eigenvalues >= 1, which keeps its Cholesky factor
// well conditioned.
#pragma once
#include "mra_device.cuh"

namespace mra {

constexpr int MAXL = 13;   // levels 0..12

// Pointers to the per-level state of one handle (passed to kernels by value).
struct LevelState {
  // tree: the active regions of every level (those whose subtree holds at
  // least one observation), in Morton order; a complete tree has identity tables
  int32_t* mort[MAXL];    // level m (0..M): compact id -> Morton id
  int32_t* par[MAXL];     // level m (1..M): compact id -> compact id of the parent
  int32_t* cfirst[MAXL];  // level m (0..M-1): compact id of the first active child
  int32_t* ccnt[MAXL];    // number of active children (consecutive compact ids)
  int32_t* cid[MAXL];     // level m: Morton id -> compact id, -1 if inactive (4^m entries)
  int nreg[MAXL];         // active regions per level
  // prior, internal levels m < M
  double* V[MAXL];    // 4^m x r x (m r): [V^0_R .. V^{m-1}_R] per region, row-major
  double* Li[MAXL];   // 4^m x r x r: L_R^{-1} (lower, zero above the diagonal)
  // posterior, internal levels m < M
  double* Acc[MAXL];  // 4^m x T_m x r x r, T_m = (m+1)(m+2)/2 packed lower blocks of Ahat
  double* Om[MAXL];   // 4^m x (m+1) x r: omegahat^k
  double* Lt[MAXL];   // 4^m x r x r: Lt^{-1}, Lt Lt' = I + Ahat^{m,m}
  double* G[MAXL];    // 4^m x r x (m r): [G^0 .. G^{m-1}] = Lt^{-1} [Ahat^{m,0} .. Ahat^{m,m-1}]
  double* gv[MAXL];   // 4^m x r: g = Lt^{-1} omegahat^m
  double* dd[MAXL];   // 4^m: d_R (Sec. 3.3)
  double* uu[MAXL];   // 4^m: u_R
  // row scales for the FP64-emulation engine (MRA_PREC_EMU only, else null):
  // the binary exponent e with |x| < 2^e over each 128-column group of a row
  int32_t* vexp[MAXL];   // level m >= 1: 4^m x ceil(m r / 128) x r, rows of V_R per group
  int32_t* liexp[MAXL];  // 4^m x r: rows of L_R^{-1}
  int32_t* gcol[MAXL];   // level m >= 1: 4^m x (m r): columns of G_R over its r rows
  // saved for the gradient (null when no gradient is requested)
  double* L[MAXL];    // 4^m x r x r: L_R (prior Cholesky factor)
  double* Ltf[MAXL];  // 4^m x r x r: Lt (Cholesky factor of I + Ahat^{m,m})
  // gradient of the emulated form: column exponents (|x| < 2^e over the r rows)
  int32_t* licol[MAXL];  // 4^m x r: columns of L_R^{-1}
  int32_t* vcol[MAXL];   // level m >= 1: 4^m x (m r): columns of V_R
};

// Compact id of the level-l ancestor of compact region c of level m.
__device__ __forceinline__ long ancestor(const LevelState& st, int m, long c, int l) {
  for (int t = m; t > l; --t) c = st.par[t][c];
  return c;
}

struct LeafState {
  const int64_t* off;     // 4^M + 1 leaf offsets into the sorted observations (by Morton id)
  const int64_t* sq_off;  // 4^M + 1 prefix sums of n_F^2 (by Morton id)
  const double* xs;       // sorted x
  const double* ys;       // sorted y coordinate
  const double* yv;       // sorted data
  double* H;              // n x (M r): V_F, then H_F = L_Sigma^{-1} V_F
  double* z;              // n: L_Sigma^{-1} y_F
  double* LS;             // ragged n_F x n_F: L_Sigma^{-1}
  double* d;              // per active leaf: log|Sigma_F|
  double* u;              // per active leaf: y_F' Sigma_F^{-1} y_F
  // saved for the gradient (null when no gradient is requested)
  double* VF;             // n x (M r): V_F before the L_Sigma^{-1} solve
  double* LSf;            // ragged n_F x n_F: L_Sigma
  // column scales of H_F over the leaf's rows for the emulation engine (else null)
  int32_t* hcol;          // per active leaf x (M r)
  // row scales of V_F per 128-column group from the emulated chain kernel (else null)
  int32_t* hrow;          // n x ceil(M r / 128)
  // set for gradient calls of the emulated form only: the chain kernel stores,
  // for every C0(s_o, q_j) of the chain blocks, (dC0/dsigma2, dC0/dkappa) at
  // [o][l r + j][2], which the chain adjoint then reads
  double* dc;             // n x (M r) x 2
  // set for gradient calls of the emulated form only: the exponent (|x| < 2^e)
  // of every column of V_F over each 128-row tile of a level-(M-1) region's rows
  int32_t* vfexp;         // per level-(M-1) region x 4 tiles x (M r)
};

// Components of the gradient: d/d(sigma2, kappa, tau2) and, for the Matern
// family of free smoothness, d/dnu (zero for the other families).
constexpr int GP = 4;

// Adjoint state of the gradient pass (mra_grad.cu).
struct GradState {
  double* Abar[MAXL];   // 4^m x r x (m+1) r: row m of the symmetric adjoint of Ahat
  double* Obar[MAXL];   // 4^m x r: adjoint of omegahat^m
  double* GB[MAXL];     // 4^m x r x (m r): adjoint of G
  double* VB[MAXL];     // 4^m x r x (m r): adjoint of V_R
  double* XB[MAXL];     // 4^m x r x (m r): adjoint of the chain blocks X^l_R
  double* Up[MAXL];     // 4^m x m(m+1)/2 x r x r: ancestor adjoints passed up from level m
  double* PartLeaf;     // 4^(M-1) x M(M+1)/2 x r x r: ancestor adjoints from the leaves
  double* HB;           // n x (M r): adjoint of H
  double* VBF;          // n x (M r): adjoint of V_F
  double* XBF;          // n x (M r): adjoint of X^l_F
  double* T;            // ragged 3 n_F^2 per leaf: scratch of the leaf adjoint
  double* gpart;        // GP per CTA: partial d/d(sigma2, kappa, tau2, nu)
  double* DC;           // emulated form: n x (M r) x 2 derivative pairs of the leaf chain's C0 blocks
  // emulated form: column exponents per 128-row tile of each level-(M-1)
  // region's rows (region x 4 x (M r)), the leaf partials' operand scales:
  // of V_F (from the forward chain kernel), of Vbar_F and Xbar_F (from the
  // chain adjoint)
  int32_t* VFexp;
  int32_t* VBexp;
  int32_t* XBexp;
  // emulated form only (else null): per level-(M-1) region, the full symmetric
  // adjoint S of Ahat along its ancestor chain (M r x M r, row-major) and the
  // scales of its rows per 128-column group, for the leaves' Hbar = 2 H S
  double* SF;
  int32_t* SFexp;       // [region][group][M r]
  // first compact region id of the launch (block b works on region rbase + b);
  // 0 except for the chunks of a streamed gradient
  long rbase;
};

// Symmetric adjoint block (k, l) of region chain `anc` (ancestor index per
// level): S^{k,l} is stored in the row of the level-max(k,l) ancestor.
// Returns pointer and strides for B(j, kk) = S^{k,l}[kk][j].
struct SRef {
  const double* p;
  long sj, sk;
};
__device__ __forceinline__ SRef sblock(const GradState& gs, const long* anc, int r, int k, int l) {
  if (k >= l) {   // S^{k,l}[kk][j] = row k of ancestor k, block l
    const long ld = (long)(k + 1) * r;
    return {gs.Abar[k] + anc[k] * (long)r * ld + l * r, 1, ld};
  }
  const long ld = (long)(l + 1) * r;   // S^{k,l}[kk][j] = S^{l,k}[j][kk]
  return {gs.Abar[l] + anc[l] * (long)r * ld + k * r, ld, 1};
}

// Prediction points of one mra_predict call, sorted by leaf.
struct PredState {
  const int64_t* off;     // (leaves + 1) offsets of the prediction points per leaf (4^M leaves for the quadtree)
  const int64_t* perm;    // sorted position -> caller's index
  const double* xs;
  const double* ys;
  double* U;              // np x (M r) scratch: Uhat, then the posterior basis Bhat
  double* mean;           // np, caller's order
  double* var;            // np, caller's order
  // joint modes only (mra_predict_joint, mra_simulate), else null: every leaf's
  // points are sorted stably (ascending caller index) and, per leaf F with
  // n_P points, D[sq_off[F] ..] holds its n_P x n_P delta~ covariance
  // V^P - L^M Sigma^{-1} L^M' (joint covariance) or that matrix's lower
  // Cholesky factor (simulation); U ends as [Y_0 .. Y_{M-1}] per point,
  // Y_l = Bhat^{l+1,l} Lt_l^{-T}; leaf[p] = Morton id of sorted point p's leaf
  const int64_t* sq_off;
  double* D;
  int32_t* leaf;
  // the leaves a launch covers, [leaf0, leaf0 + gridDim.x) by Morton id, and the
  // descriptor it reads (a streamed handle predicts chunk by chunk)
  long leaf0;
  int desc;
  long nleaves;           // leaves of the complete tree (the launch's grid where it covers them all)
};

struct Shape {
  int M, r, gx, gy;
  double bbox[4];
  int mixed;              // 1: tensor-core (3xTF32) prior and leaf contractions
  unsigned long long hx, hy;   // per-level midpoint halvings in x and y (4 bits per level)
};

// log2 J_M: the bits of a leaf's digit below its level-(M-1) parent (2 for the quadtree)
__host__ __device__ __forceinline__ int leaf_bits(const Shape& sh) { return lvl_bits(sh.hx, sh.hy, sh.M); }

// Quadtree halvings (one in x and one in y at every level).
constexpr unsigned long long QUAD_HALVINGS = 0x1111111111110ull;

// Fill sx/sy (shared) with the r knots of region (m, i).
__device__ __forceinline__ void load_knots(const Shape& sh, int m, long i, double* sx, double* sy) {
  Box b = region_box(sh.bbox, sh.hx, sh.hy, m, i);
  for (int q = threadIdx.x; q < sh.gx * sh.gy; q += NT) knot_xy(b, sh.gx, sh.gy, q, sx[q], sy[q]);
}

// Everything a kernel needs about one dataset, in device memory.  A single
// problem is a batch of one; batched launches map every CTA to a (dataset,
// region) pair through a work list.
struct Desc {
  Shape sh;
  Cov cv;
  double tau2;
  int nlmax;          // largest leaf occupancy (shared-memory layout of the leaf kernels)
  int lrows;          // rows of the emulated leaf kernel's layout: the largest group of leaves (>= nlmax), or 0
  LevelState st;
  LeafState lf;
};

// (dataset, compact region) of this CTA; `work` null means dataset 0, region blockIdx.x.
struct Item {
  int d;
  long i;
};
__device__ __forceinline__ Item work_item(const int2* work) {
  if (work) {
    const int2 w = work[blockIdx.x];
    return {w.x, (long)w.y};
  }
  return {0, (long)blockIdx.x};
}

// Tiled work on a flat grid of nt tiles per item, the tile index running
// fastest, so that the tiles of one item (which read the same operand rows)
// run together and share them in L2.
__device__ __forceinline__ Item work_item_tiled(const int2* work, int nt, int& tile) {
  const long b = blockIdx.x / nt;
  tile = (int)(blockIdx.x - b * nt);
  if (work) {
    const int2 w = work[b];
    return {w.x, (long)w.y};
  }
  return {0, b};
}

}  // namespace mra
