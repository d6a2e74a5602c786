// mra_launch.h -- host-side launchers of the M-RA kernels (internal to the library).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "mra_kernels.cuh"

namespace mra {

// Optional per-launch CUDA-event timing (kinds match MRA_K_* in mra.h; the
// stage and level of a record match MRA_STAGE_* and the level index of
// mra_stats_t, or -1 where a launch has none).
constexpr int MAX_TIMED = 8192;
struct Timer {
  bool on = false;
  int count = 0;
  int kind[MAX_TIMED];
  int stage[MAX_TIMED];
  int level[MAX_TIMED];
  cudaEvent_t ev[2 * MAX_TIMED];
  void start(int k, cudaStream_t s, int st = -1, int lv = -1) {
    if (!on || count >= MAX_TIMED) return;
    kind[count] = k;
    stage[count] = st;
    level[count] = lv;
    cudaEventRecord(ev[2 * count], s);
  }
  void stop(cudaStream_t s) {
    if (!on || count >= MAX_TIMED) return;
    cudaEventRecord(ev[2 * count + 1], s);
    ++count;
  }
};

// Tree build (Sec. 2.2): leaf of every observation, stable counting sort by leaf.
cudaError_t launch_bin(const double* locs, int64_t n, const double* bbox_dev, int M, unsigned long long hx,
                       unsigned long long hy, int32_t* leaf_id, int32_t* counts, int32_t* cursor, int64_t* off,
                       int64_t* sq_off, int32_t* max_count, int64_t* perm, int* status,
                       cudaStream_t s, int64_t* launches, bool stable = true);
// Gather the sorted observations: xs, ys, yv from row-major locs (n x 2) and y.
cudaError_t launch_gather(const double* locs, const double* y, const int64_t* perm, int64_t n,
                          double* xs, double* ys, double* yv, cudaStream_t s, int64_t* launches);
// Gather y only (new data on an existing partition).
cudaError_t launch_gather_y(const double* y, const int64_t* perm, int64_t n, double* yv,
                            cudaStream_t s, int64_t* launches);

// Launch plan of one evaluation: per level, the CTAs (work items, or null for
// "dataset 0, compact region blockIdx.x") of the prior/posterior kernels
// (n_lvl[m]), of the aggregation into level m-1 (n_agg[m]), of the leaves and
// of the leaf Gram products.
struct Plan {
  int maxM = 0, tile = 64, mixed = 0, nlmax = 1;   // mixed: 0 FP64, 1 3xTF32, 2 FP64 emulation
  int r = 0;
  // the part of the pass this plan runs (subtree streaming splits a pass in
  // three): prior levels [prior_lo, prior_hi), the leaves, and posterior
  // levels [post_lo, post_hi) with the aggregation of each such level m > 0
  // into level m - 1; prior_hi / post_hi < 0 mean maxM
  int prior_lo = 0, prior_hi = -1, post_lo = 0, post_hi = -1;
  bool leaves = true;
  const int2* w_lvl[MAXL] = {};
  int n_lvl[MAXL] = {};
  const int2* w_agg[MAXL] = {};
  int n_agg[MAXL] = {};
  const int2* w_leaf = nullptr;
  int n_leaf = 0;
  // emulated form: groups of leaves (c_leaf[b] leaves from compact id w_leaf[b].y;
  // n_leaf counts groups), laid out for lrows rows; null: one leaf per item
  const int* c_leaf = nullptr;
  int lrows = 0;
  // prior levels on the tensor cores: groups of sibling regions (c_pri[m][b]
  // regions from compact id w_pri[m][b].y; n_pri[m] groups), stacked at most
  // rcap rows; null: the level's regions one by one (w_lvl, n_lvl)
  const int2* w_pri[MAXL] = {};
  const int* c_pri[MAXL] = {};
  int n_pri[MAXL] = {};
  int rcap = 0;
  // the emulated leaf chain: groups of sibling level-(M-1) regions (c_chn[b]
  // regions from w_chn[b].y, one 128-row tile); null: the leaf_syrk list
  const int2* w_chn = nullptr;
  const int* c_chn = nullptr;
  int n_chn = 0;
  const int2* w_syrk = nullptr;
  int n_syrk = 0, t_syrk = 1;
};

// Prior pass, leaf pass and posterior pass (Sec. 3.1-3.3).
cudaError_t launch_loglik(const Plan& pl, const Desc* d_desc, int* status, cudaStream_t s, int64_t* launches,
                          Timer* timer);
int tile_for_r(int r);
// Root terms (d, u) of every dataset of a batch into out[2 d], out[2 d + 1].
cudaError_t launch_gather_roots(const Desc* d_desc, int nd, double* out, cudaStream_t s, int64_t* launches);
size_t leaf_smem_bytes(int r, int nlmax);

// Mixed-precision prior level and leaf pass (tensor cores, mra_mixed.cu).
// emu = 1: FP64-grade bf16-slice emulation engine; 0: 3xTF32.
cudaError_t launch_prior_tc(int m, const Desc* d_desc, const int2* work, int nblocks, int emu, int* status,
                            cudaStream_t s, const int* gcnt = nullptr, int rcap = 0);
cudaError_t launch_leaf_tc(const Desc* d_desc, const int2* work, int nblocks, int nlmax, int emu, int* status,
                           cudaStream_t s, const int2* w_par = nullptr, int n_par = 0, Timer* tm = nullptr,
                           int leaf_level = -1, const int* gcnt = nullptr, int lrows = 0,
                           const int* gpar = nullptr);
size_t leaf_tc_smem_bytes(int nlmax, int emu);
cudaError_t launch_leaf_syrk_em(const Desc* d_desc, const int2* work, int nblocks, int maxM, int r, int* status,
                                cudaStream_t s);
cudaError_t launch_aggregate_em(int m, int r, const Desc* d_desc, const int2* work, int nblocks, int* status,
                                cudaStream_t s);

// Prediction (Sec. 3.4, Prop. 2) at points binned into ps.
// nleaf > 0: only the leaves [ps.leaf0, ps.leaf0 + nleaf) (a chunk of a streamed handle)
cudaError_t launch_predict(const Desc* d_desc, int M, int r, int nlmax, const PredState& ps, int max_per_leaf,
                           int* status, cudaStream_t s, int64_t* launches, Timer* tm, long nleaf = 0);
size_t predict_smem_bytes(int r, int nlmax);
// Joint posterior predictive (Prop. 2): mode 1 keeps D and the Y_l for the
// covariance, mode 2 chol(D) and the Y_l for simulation (at most JOINT_TILE
// points per leaf); then the covariance tiles or the draws.
constexpr int JOINT_TILE = 64;
size_t joint_smem_bytes(int r, int nlmax);
cudaError_t launch_predict_joint(const Desc* d_desc, int M, int r, int nlmax, const PredState& ps, int mode,
                                 int* status, cudaStream_t s, int64_t* launches, Timer* tm);
cudaError_t launch_joint_cov(const Desc* d_desc, const PredState& ps, int64_t np, double* cov, cudaStream_t s,
                             int64_t* launches);
cudaError_t launch_simulate(const Desc* d_desc, int M, const PredState& ps, int64_t np, int64_t nsim, int64_t nxi,
                            const double* xi, const double* zeta, double* draws, cudaStream_t s, int64_t* launches);

// Reverse-mode gradient after a forward pass that saved L, Lt, V_F and L_Sigma.
cudaError_t launch_grad(const Desc& hd, const Desc* d_desc, const GradState& gs, double* grad_out_dev, int* status,
                        cudaStream_t s, int64_t* launches, Timer* tm);
// A part of the reverse pass (a streamed gradient runs it in three): posterior
// adjoint levels [post_lo, post_hi) top-down, the leaves' adjoints, prior
// adjoint levels [prior_lo, prior_hi) bottom-up; per level the regions
// [base, base + count) (count < 0: every region of the level); hi < 0 means M.
// The emulated form's column scales of L^{-1} and V (read by the leaves' and
// the prior levels' adjoints) are formed for levels [cs_lo, cs_hi), by default
// (cs_lo < 0) the prior adjoint's levels.
struct GradRange {
  int post_lo = 0, post_hi = -1, prior_lo = 0, prior_hi = -1;
  int cs_lo = -1, cs_hi = -1;
  bool leaves = true;
  // the emulated form's per-parent S buffer holds only the parents of this
  // range (a streamed chunk): its launches address it from the range's base
  bool local_sf = false;
  long base[MAXL] = {}, count[MAXL] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};
};
cudaError_t launch_grad_range(const Desc& hd, const Desc* d_desc, GradState gs, const GradRange& R, int* status,
                              cudaStream_t s, int64_t* launches);
// Sum of every CTA's partial gradient into grad_out_dev[0..GP).
cudaError_t launch_grad_reduce(const Desc& hd, const GradState& gs, double* grad_out_dev, cudaStream_t s,
                               int64_t* launches);
// Emulated form: Hbar = 2 H S + z omegabar' of every leaf on the tensor cores
// (mra_mixed.cu), from the assembled per-parent S of GradState.
// Emulated form: the leaves' partial ancestor adjoints (leaf_partial_kernel's tiles).
// (nregions < 0: every level-(M-1) region; else that many from gs.rbase)
cudaError_t launch_leaf_partial_em(const Desc& hd, const Desc* d_desc, const GradState& gs, int* status,
                                   cudaStream_t s, long nregions = -1);
// Emulated form: the leaves' chain adjoint (Xbar and the Vbar updates), per parent;
// its C0 terms go to gradient slots slot0 .. slot0 + nreg[M-1] - 1.
cudaError_t launch_chain_adjoint_em(const Desc& hd, const Desc* d_desc, const GradState& gs, long slot0,
                                    int* status, cudaStream_t s, long nregions = -1);
// Emulated form: Gbar of level m (1 <= m < M) per level-(m-1) region, from its
// assembled S (mra_mixed.cu); post_adjoint_kernel then skips its own product.
cudaError_t launch_gbar_em(int m, const Desc& hd, const Desc* d_desc, const GradState& gs, int* status,
                           cudaStream_t s, int64_t* launches, long nregions = -1);
cudaError_t launch_hbar_em(const Desc& hd, const Desc* d_desc, const GradState& gs, int* status, cudaStream_t s,
                           int64_t* launches, long nregions = -1);

// Identity tables of a complete tree with M levels (for callers without host tables).
cudaError_t launch_identity_tree(const LevelState& st, int M, unsigned long long hx, unsigned long long hy,
                                 cudaStream_t s, int64_t* launches);

// Error text and launch counter shared by every entry point (mra_api.cu).
void set_last_error(const char* msg);
int64_t* launch_counter();

}  // namespace mra
