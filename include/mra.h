/*
 * mra.h -- C ABI of the GB300 multi-resolution approximation (M-RA) library.
 *
 * The library evaluates, on one CUDA GPU, the M-RA of a Gaussian process
 * (Katzfuss, "A multi-resolution approximation for massive spatial datasets",
 * JASA 2017): its log-likelihood (Sec. 3.3), the gradient of that
 * log-likelihood in the covariance parameters, and kriging predictions with
 * variances (Sec. 3.4, Prop. 2).  The problem is stated as in the paper:
 *
 *   - n observation locations S in a 2-D bounding box and data y (Sec. 2.1);
 *   - a covariance function C0 known up to theta = (sigma2, range) (Sec. 2.1),
 *     exponential or Matern-1.5 (Eq. mat15), optionally with the
 *     nonstationary variance sigma2 * sqrt(g(s1) g(s2)), g(s) = 1 + 0.5 sin(4 pi x);
 *   - M levels of a recursive partition with J = 4 children per region
 *     (midpoint quadtree, child j = b_x + 2 b_y, half-open cells), or J_m
 *     children at level m (mra_config.J_level), Sec. 2.2;
 *   - r knots per region on a cell-centred gx x gy grid (gx = smallest divisor
 *     of r with gx^2 >= r), leaves using their observations as knots (Sec. 2.2);
 *   - measurement-error variance tau2 added to the leaf covariance (Sec. 4.3).
 *
 * Conventions for every entry point:
 *   - All floating point is IEEE binary64 (double).
 *   - Return value: MRA_OK (0) or one of the MRA_ERR_* codes below; the text of
 *     the last error of the calling thread is available from mra_last_error().
 *     No entry point throws or aborts.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the handle's device.  Unless stated otherwise, inputs are
 *     read during the call only and stay owned by the caller.
 *   - A handle owns all device memory it allocates and is used by one host
 *     thread at a time.  All its kernels run on its stream (default: the legacy
 *     default stream; see mra_set_stream).  Entry points that return results in
 *     host memory synchronise that stream before returning.
 */
#ifndef MRA_H
#define MRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MRA_OK          0
#define MRA_ERR_ARG     1   /* invalid argument: sizes, config, a location outside bbox */
#define MRA_ERR_OOM     2   /* device allocation failed */
#define MRA_ERR_CUDA    3   /* a CUDA runtime call or kernel launch failed */
#define MRA_ERR_NOT_PD  4   /* a matrix the method needs positive definite is not
                               (non-positive Cholesky pivot); level/region in the text */
#define MRA_ERR_STATE   5   /* call order: e.g. mra_predict before any mra_loglik */
#define MRA_ERR_LIMIT   6   /* a leaf holds more observations than MRA_MAX_LEAF */

/* ---- limits ------------------------------------------------------------ */
#define MRA_MAX_R       64  /* knots per internal region */
#define MRA_MAX_M       12  /* levels */
#define MRA_MAX_LEAF    128 /* observations per leaf (the leaf kernel keeps the
                               leaf covariance in shared memory) */

/* ---- enumerations ------------------------------------------------------ */
#define MRA_COV_EXP       0 /* C0 = sigma2 exp(-h / range) */
#define MRA_COV_MATERN15  1 /* C0 = sigma2 (1 + sqrt3 h / range) exp(-sqrt3 h / range), Eq. mat15 */
#define MRA_COV_MATERN    2 /* C0 = sigma2 2^(1-nu)/Gamma(nu) z^nu K_nu(z), z = sqrt(2 nu) h / range: the
                               Matern of smoothness nu = mra_params.nu (Sec. 4.1's family; nu = 1.5 is
                               Eq. mat15, 0.5 the exponential), K_nu by an exponentially convergent
                               trapezoidal rule (relative error about 1e-13, 0.05 <= nu <= 20); about
                               20-100 times the cost of the closed forms per evaluation of C0 */

#define MRA_PREC_FP64     0 /* every step in binary64 */
#define MRA_PREC_MIXED    1 /* prior chain, leaf covariance and leaf solve products on the
                               tensor cores (tcgen05, 3xTF32 with FP64 accumulation every 64
                               terms); factorisations, log-determinants, quadratic forms and
                               the Gram products of the posterior pass in binary64 */
#define MRA_PREC_EMU      2 /* every large contraction (prior chain, leaf covariance and solve,
                               leaf and child-to-parent Gram products, posterior G, and in
                               mra_loglik_grad the adjoint's products) on the tensor cores as an
                               FP64-grade emulation: operands cut into seven 7-bit bf16 slices
                               per 128-column group, exact FP32 accumulation, double-float sums
                               (about 1e-14 relative error per product); factorisations and
                               the rest in binary64 */

#define MRA_HOST          0 /* pointer argument is host memory */
#define MRA_DEVICE        1 /* pointer argument is device memory */

/* Problem shape (Sec. 2.2).  Plain data, owned by the caller, copied by mra_build. */
typedef struct {
    int    M;           /* levels; leaves are the J_1 ... J_M (4^M for the quadtree) regions of level M;
                           0 <= M <= MRA_MAX_M */
    int    J;           /* children per region at every level: must be 4 (2-D midpoint quadtree);
                           not read when J_level[0] != 0 */
    int    r;           /* knots per internal region, 1 <= r <= MRA_MAX_R */
    int    cov_family;  /* MRA_COV_EXP or MRA_COV_MATERN15 */
    int    nonstat;     /* 1: variance sigma2 * sqrt(g(s1) g(s2)), g(s) = 1 + 0.5 sin(4 pi x) */
    int    precision;   /* MRA_PREC_FP64, MRA_PREC_MIXED or MRA_PREC_EMU */
    int    prune;       /* 1: keep only regions whose subtree holds observations (empty subtrees
                           contribute nothing to the likelihood); 0: complete tree */
    double bbox[4];     /* x0, x1, y0, y1 of the domain; every location must lie inside */
    int    stream_level;/* subtree streaming: s in 1..M-1 evaluates the tree as its level-s
                           subtrees one after another in buffers sized for the largest
                           (the factors of levels > s and of the leaves are never all
                           resident; levels <= s and every region's d, u are); 0 lets
                           mra_build stream, at the smallest s that fits, only when the
                           factors of every level would exceed 80 % of the free device
                           memory; -1 never streams.  A streamed handle evaluates
                           mra_loglik (and mra_region_terms, mra_stats), mra_predict (which
                           forms each chunk's factors again from the resident coarse ones,
                           about one more evaluation) and mra_loglik_grad (each chunk's
                           factors formed again before its adjoint, the last chunk's
                           reused: about one more forward evaluation; the adjoint state of
                           levels > s and the emulated form's optional gradient buffers are
                           chunk-sized too); mra_predict_joint,
                           mra_simulate and mra_update return MRA_ERR_STATE. */
    int    J_level[MRA_MAX_M];
                        /* level-varying J (Sec. 2.2; Sec. 4.3 uses (2, 2, 4, 8, 8, 16)):
                           J_level[m-1] = J_m, the children of every level-(m-1) region,
                           m = 1..M, each 2, 4, 8 or 16 (J_M, the leaves' level, 2 or 4 for
                           MRA_PREC_EMU), and J_1 ... J_M <= 2^24; entries past M zero.  All zero: J at every
                           level.  Every region of a level splits the same way, into an
                           s_x x s_y grid of equal children (s_x s_y = J_m) by repeated
                           midpoint halving (half-open, last cell closed): with L_m =
                           log2(J_1 ... J_m), level m halves ceil(L_m/2) - ceil(L_{m-1}/2)
                           times in x and floor(L_m/2) - floor(L_{m-1}/2) times in y; child
                           j = c_x + s_x c_y.  mra_loglik_noalloc takes the quadtree only. */
} mra_config;

/* Covariance parameters theta and the measurement-error variance (Sec. 2.1, 4.3). */
typedef struct {
    double sigma2;      /* > 0 */
    double range;       /* kappa > 0 */
    double tau2;        /* >= 0 */
    double nu;          /* smoothness, 0.05 <= nu <= 20, read for MRA_COV_MATERN only */
} mra_params;

typedef struct mra_handle mra_handle;

/*
 * mra_build -- partition the domain and bin the observations (Sec. 2.2).
 *   cfg    : problem shape (host).
 *   locs   : n x 2 row-major (x, y) locations, host or device per `where`.
 *   y      : n observations, same memory space as locs.
 *   n      : number of observations, n >= 1.
 *   where  : MRA_HOST or MRA_DEVICE.
 *   out    : receives a new handle (host pointer to a handle pointer).
 * Allocates the handle's device memory (about 8 n M r + R M^2 r^2 doubles for
 * the factors of all levels, R = the leaves' count, 4^M for the quadtree), copies and sorts the observations by leaf on the
 * device (stable within a leaf).  Errors: MRA_ERR_ARG (bad config, n < 1, a
 * location outside bbox), MRA_ERR_LIMIT (a leaf above MRA_MAX_LEAF: raise M),
 * MRA_ERR_OOM, MRA_ERR_CUDA.  On error *out is NULL and nothing is leaked.
 */
int mra_build(const mra_config* cfg, const double* locs, const double* y, int64_t n,
              int where, mra_handle** out);

/*
 * mra_set_data -- replace the observations y of a built handle (same n, same
 * order as given to mra_build; host or device per `where`).  The partition is
 * kept.  Errors: MRA_ERR_ARG, MRA_ERR_CUDA.
 */
int mra_set_data(mra_handle* h, const double* y, int where);

/*
 * mra_update -- replace locations and data of a built handle with a new set of
 * the same size n (host or device per `where`), re-partitioning on the device
 * without allocating.  Errors: MRA_ERR_ARG (a location outside bbox),
 * MRA_ERR_LIMIT (the new partition needs a fuller leaf, or more leaf-factor
 * storage, than the handle was built for: build a new handle), MRA_ERR_CUDA.
 */
int mra_update(mra_handle* h, const double* locs, const double* y, int where);

/*
 * mra_loglik -- the M-RA log-likelihood at theta (Sec. 3.1-3.3):
 *   loglik = -(d + u)/2 - (n/2) log(2 pi),  -2 log L_M(theta) = d + u.
 * Runs the prior pass (Eq. priorw) top-down and the posterior pass (Eqs.
 * posterior, mainquantities, helpquantities) bottom-up; keeps the posterior
 * factors in the handle for mra_predict at the same theta.
 *   theta       : host pointer to one mra_params.
 *   loglik_out  : host pointer to one double.
 * Errors: MRA_ERR_ARG (theta out of range), MRA_ERR_NOT_PD, MRA_ERR_CUDA.
 */
int mra_loglik(mra_handle* h, const mra_params* theta, double* loglik_out);

/*
 * mra_loglik_grad -- the log-likelihood (as mra_loglik) and its gradient
 * d loglik / d(sigma2, range, tau2).  The paper gives no gradient; it serves
 * the numerical maximum-likelihood fit of Sec. 4.3.  The gradient is the exact
 * reverse-mode adjoint of the evaluation (Cholesky, triangular-solve and
 * A-update chains of Sec. 3.1-3.2 in reverse), in FP64; with MRA_PREC_EMU its
 * products run on the FP64 emulation of the tensor cores (gradient within
 * 1e-9 relative of the FP64 form's).  The first call allocates the adjoint
 * buffers (in the emulated form also, where free device memory allows, a
 * per-region S buffer of nreg[M-1] (M r)^2 doubles when that is at most four
 * times the size of H, and n M r x 2 doubles of covariance derivatives; without
 * them the same gradient is formed more slowly).
 *   theta      : host pointer to one mra_params.
 *   loglik_out : host pointer to one double.
 *   grad_out   : host pointer to 3 doubles (d/dsigma2, d/drange, d/dtau2), and a
 *                fourth, d/dnu, when cov_family = MRA_COV_MATERN (4 doubles then).
 * The first call allocates the adjoint storage (about 4 n M r doubles plus the
 * per-level adjoints); later calls allocate nothing.  Also leaves the posterior
 * factors for mra_predict at theta.  Errors: as mra_loglik, and MRA_ERR_OOM.
 */
int mra_loglik_grad(mra_handle* h, const mra_params* theta, double* loglik_out, double* grad_out);

/*
 * mra_predict -- marginal posterior predictive mean and variance of the
 * process y (not of the noisy data, Sec. 4.3) at np locations (Sec. 3.4,
 * Prop. 2, Eq. bfrecursion).  Uses the posterior factors of the last
 * mra_loglik (or mra_loglik_grad) when that was at the same theta; otherwise
 * it first evaluates the log-likelihood at theta (as mra_loglik, whose
 * factors then stay in the handle).
 *   plocs    : np x 2 row-major locations inside bbox, host or device per `where`.
 *   mean_out, var_out : np doubles each, same memory space as plocs, caller-owned.
 * The handle keeps a prediction buffer (about np (M r + 8) doubles) that is
 * allocated on the first call and grown when np exceeds every earlier call's.
 * Errors: MRA_ERR_ARG (theta out of range, a location outside bbox),
 * MRA_ERR_STATE (a batch handle), MRA_ERR_NOT_PD, MRA_ERR_OOM, MRA_ERR_CUDA.
 */
int mra_predict(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np,
                int where, double* mean_out, double* var_out);

/*
 * mra_predict_joint -- the joint posterior predictive distribution of y at np
 * locations (Prop. 2): mean (as mra_predict) and the full covariance
 *   Cov(s1, s2) = sum over the regions R_m (m < M) that contain both points of
 *                 B~^{m+1,m}(s1) K~_{R_m} B~^{m+1,m}(s2)'
 *                 + [same leaf] (V^P - L^M Sigma^{-1} L^M')(s1, s2),
 * since eta~_{R_m} is shared by every leaf under R_m and delta~ is per leaf.
 *   plocs    : np x 2 row-major, host or device per `where`; at most
 *              MRA_MAX_JOINT_LEAF points per leaf, np <= MRA_MAX_JOINT_POINTS.
 *   mean_out : np doubles; cov_out: np x np row-major (caller's point order),
 *              both in the memory space of plocs, caller-owned.
 * Uses the posterior factors at theta as mra_predict does.  Host mode stages
 * the covariance in a handle buffer of np^2 doubles (grown on demand).
 * Errors: as mra_predict; MRA_ERR_LIMIT (too many points in a leaf or in all).
 */
#define MRA_MAX_JOINT_LEAF   64
#define MRA_MAX_JOINT_POINTS 32768
int mra_predict_joint(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                      double* mean_out, double* cov_out);

/*
 * mra_simulate -- nsim conditional simulations: draws from the joint posterior
 * predictive distribution of y at np locations (Prop. 2), given standard
 * normal inputs (the caller draws them, so any generator may be used):
 *   eta~_R   = K~_R omega^m_R + L_R^{-T} Lt_R^{-T} xi_R   for every region R
 *              of levels 0..M-1 (L_R L_R' = K_R^{-1}, Lt_R Lt_R' = I +
 *              L_R^{-1} A^{m,m}_R L_R^{-T}: a square root of K~_R),
 *   delta~_F = L^M Sigma^{-1} y_F + chol(V^P - L^M Sigma^{-1} L^M') zeta_F
 *              per leaf F (its points in ascending order of their index),
 *   draw     = sum_{m<M} B~^{m+1,m} eta~_{R_m} + delta~_F.
 *   xi    : nsim x len (mra_simulate_xi_len: r per region of levels 0..M-1 of
 *           the complete tree, levels in order, regions by Morton index;
 *           entries of regions without prediction points are not read);
 *           may be NULL when M = 0.
 *   zeta  : nsim x np, one normal per prediction point (caller's order).
 *   draws_out : nsim x np.  xi, zeta, draws_out and plocs share `where`.
 * Errors: as mra_predict_joint; MRA_ERR_NOT_PD when the Cholesky factor of a
 * leaf's delta~ covariance meets a non-positive pivot (prediction points of a
 * leaf that coincide make it singular).
 */
int mra_simulate(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where, int64_t nsim,
                 const double* xi, const double* zeta, double* draws_out);
int mra_simulate_xi_len(mra_handle* h, int64_t* len_out);

/*
 * Two-phase evaluation over the level-s subtrees of a streamed handle
 * (stream_level = s >= 1), for sharding one problem over several GPUs: the
 * regions of one resolution are independent (Sec. 3.5), so every process
 * builds the same handle, evaluates its own range of the level-s subtrees,
 * all processes exchange the subtrees' summaries (one all-gather), and each
 * finishes the coarse levels s..0 itself.
 *
 * mra_summary_len -- doubles per summary (*len_out: the level-s region's
 *   A-hat blocks, T_s r^2 with T_s = (s+1)(s+2)/2, its omega-hat, (s+1) r, and
 *   the (d, u) of up to J_{s+1} children, 2 J_{s+1}: 8 for the quadtree) and
 *   the number of level-s regions (*nsub_out, compact order).
 * mra_loglik_subtrees -- at theta: the prior of levels 0..s, then the
 *   subtrees of level-s regions [first, first + count) (prior, leaves,
 *   posterior up to the level-s aggregation); out (host, count x len) gets
 *   their summaries.  count = 0 is allowed.
 * mra_loglik_combine -- all nsub summaries (host, nsub x len, in region
 *   order, from any processes' mra_loglik_subtrees at the same theta) in, the
 *   posterior of levels s..0 run, *loglik_out the log-likelihood (as
 *   mra_loglik; region terms of levels <= s then readable).
 * Errors: MRA_ERR_STATE (not a streamed handle), MRA_ERR_ARG, MRA_ERR_NOT_PD,
 * MRA_ERR_CUDA.
 */
int mra_summary_len(mra_handle* h, int64_t* len_out, int64_t* nsub_out);
int mra_loglik_subtrees(mra_handle* h, const mra_params* theta, int64_t first, int64_t count, double* out);
int mra_loglik_combine(mra_handle* h, const mra_params* theta, const double* summaries, double* loglik_out);

/*
 * mra_region_terms -- the per-region log-determinant d_R and quadratic form
 * u_R (Sec. 3.3) of every region of `level` (0..M) from the last mra_loglik.
 * d_R = log|Sigma_R| and u_R = y_R' Sigma_R^{-1} y_R of the data in region R
 * given the weights of coarser levels.  d_out, u_out: host arrays of
 * J_1 ... J_level entries (4^level for the quadtree).
 * Errors: MRA_ERR_ARG, MRA_ERR_STATE, MRA_ERR_CUDA.
 */
int mra_region_terms(mra_handle* h, int level, double* d_out, double* u_out);

/*
 * mra_leaf_offsets -- the leaf partition of the observations: off_out (host,
 * J_1 ... J_M + 1 int64, 4^M + 1 for the quadtree) receives the start of every
 * leaf in leaf order, perm_out (host, n int64, may be NULL) the original index
 * of every sorted observation.
 */
int mra_leaf_offsets(mra_handle* h, int64_t* off_out, int64_t* perm_out);

/*
 * mra_set_stream -- run the handle's kernels on `stream` (a cudaStream_t of the
 * handle's device, passed as void*; NULL = legacy default stream).
 */
int mra_set_stream(mra_handle* h, void* stream);

/*
 * mra_set_option -- tune how a handle spends device memory.  Options:
 *   MRA_OPT_GRAD_BUFFERS (default 1): with MRA_PREC_EMU, mra_loglik_grad may
 *     take two optional buffers when free device memory holds them (the
 *     per-region adjoint S of nreg[M-1] (M r)^2 doubles and n M r x 2 doubles
 *     of covariance derivatives), which make the gradient faster; 0 never
 *     takes them (the same gradient, formed by kernels that need neither).
 *     Changing it releases the gradient storage; the next mra_loglik_grad
 *     allocates it again under the new setting.
 * Errors: MRA_ERR_ARG (null handle, unknown option or value).
 */
#define MRA_OPT_GRAD_BUFFERS 0
int mra_set_option(mra_handle* h, int option, int64_t value);

/*
 * mra_build_batch -- many independent datasets evaluated together (each with
 * its own shape cfgs[d], locations locs[d] (n x 2 row-major), data ys[d] and
 * size ns[d], all in the memory space `where`).  Every dataset gets its own
 * partition and factors; the batch evaluates them with one launch per level
 * (the paper's regions of one resolution are independent, Sec. 3.5), whose
 * CTAs map to (dataset, region) pairs, and replays that launch sequence as a
 * CUDA graph.  All datasets must share r and precision; M, the covariance
 * family and the bounding box may differ.  Swath-like data should use
 * prune = 1 (empty subtrees are skipped, Sec. 3.3).  Errors: as mra_build,
 * with the failing dataset's index in the text.
 */
int mra_build_batch(const mra_config* cfgs, const double* const* locs, const double* const* ys,
                    const int64_t* ns, int ndata, int where, mra_handle** out);

/*
 * mra_loglik_batch -- log-likelihoods of every dataset of a batch handle at
 * its own parameters: thetas[d] (host, ndata entries) -> loglik_out[d] (host).
 * The first call autotunes the tile size (mra_autotune) and captures the
 * launch sequence as a CUDA graph; later calls replay it.  Errors: MRA_ERR_ARG,
 * MRA_ERR_STATE (not a batch handle), MRA_ERR_NOT_PD, MRA_ERR_CUDA.
 */
int mra_loglik_batch(mra_handle* h, const mra_params* thetas, double* loglik_out);

/*
 * mra_loglik_grad_batch -- log-likelihood and gradient (as mra_loglik_grad)
 * of every dataset of a batch handle at its own parameters: thetas[d] (host,
 * ndata entries) -> loglik_out[d] and grad_out[3 d .. 3 d + 2] =
 * d loglik_d / d(sigma2, range, tau2) (host).  The datasets are differentiated
 * one after another on the batch's stream (the forward pass and adjoint of
 * each are the single-dataset ones); the first call allocates every dataset's
 * adjoint storage.  Errors: as mra_loglik_grad, with the failing dataset's
 * index in the text; MRA_ERR_STATE if h is not a batch handle.
 */
int mra_loglik_grad_batch(mra_handle* h, const mra_params* thetas, double* loglik_out, double* grad_out);

/*
 * mra_autotune -- time the evaluation with every tile size the kernels offer
 * for this r (16, 32 or 64 rows/columns per tile, at least r) at `thetas`
 * (one mra_params, or ndata for a batch handle) and keep the fastest;
 * *tile_out (may be NULL) receives it.
 */
int mra_autotune(mra_handle* h, const mra_params* thetas, int* tile_out);

/* mra_batch_info -- number of datasets of a handle (0 for a single handle) and its tile size. */
int mra_batch_info(mra_handle* h, int* ndata_out, int* tile_out);

/*
 * Per-kernel timing with CUDA events recorded on the handle's stream around
 * every launch (for roofline measurements).  mra_enable_timing(h, 1) resets the
 * totals and starts recording; mra_kernel_times returns the summed device time
 * (ms) and launch count of one kernel kind since then.  Kinds:
 */
#define MRA_K_PRIOR      0  /* prior pass, one launch per level (Eq. priorw) */
#define MRA_K_LEAF       1  /* leaf factorisation (Sec. 3.1-3.2 at m = M) */
#define MRA_K_LEAF_SYRK  2  /* leaf Gram products summed into level M-1 */
#define MRA_K_POST       3  /* posterior factorisation, one launch per level */
#define MRA_K_AGGREGATE  4  /* child-to-parent updates (Eqs. mainquantities, helpquantities) */
#define MRA_K_PREDICT    5  /* prediction (Sec. 3.4) */
#define MRA_K_GRAD       6  /* reverse-mode gradient pass (all adjoint kernels) */
int mra_enable_timing(mra_handle* h, int on);
int mra_kernel_times(mra_handle* h, int kind, double* total_ms, int64_t* launches);

/*
 * mra_stats -- per-level work and time of the log-likelihood evaluation, for
 * roofline fractions per level kernel.  For every level m = 0..M and stage
 * (below): the device time and launches summed over the evaluations timed
 * since mra_enable_timing(h, 1) (CUDA events on the handle's stream; zero
 * while timing is off), and the algorithmic work of ONE evaluation of the
 * handle's current tree and leaf occupancy: FLOPs (multiply-add = 2,
 * symmetric and triangular products counted once, factorisations r^3/3) and
 * HBM bytes (every operand a unit of work reads and every result it writes,
 * once per unit).  A batch handle sums its datasets' work per level.
 * The units and their counts follow the paper's per-region cost (Sec. 3.6):
 *   MRA_STAGE_PRIOR      level m < M, per region: W^l chain, L_m (Eq. priorw)
 *   MRA_STAGE_CHAIN      level M, emulated form only: the leaves' chain B^l,
 *                        run per level-(M-1) region (in the other forms it is
 *                        part of MRA_STAGE_LEAF)
 *   MRA_STAGE_LEAF       level M, per leaf: Sigma, its factor, H, z, d, u
 *   MRA_STAGE_LEAF_SYRK  level M, per level-(M-1) region: the leaves' Gram
 *                        products summed into A, omega (Eq. helpquantities at
 *                        m = M and Eq. mainquantities)
 *   MRA_STAGE_POST       level m < M, per region: K~ factor, G, d_m, u_m
 *   MRA_STAGE_AGGREGATE  level m in 1..M-1, per level-(m-1) region: the
 *                        children's A~, omega~ summed (Eq. mainquantities)
 * Errors: MRA_ERR_ARG (null argument).
 */
#define MRA_STAGE_PRIOR      0
#define MRA_STAGE_CHAIN      1
#define MRA_STAGE_LEAF       2
#define MRA_STAGE_LEAF_SYRK  3
#define MRA_STAGE_POST       4
#define MRA_STAGE_AGGREGATE  5
#define MRA_STAGES           6
typedef struct {
    int     M;                                      /* deepest level (leaves) */
    int64_t evaluations;                            /* evaluations timed */
    double  ms[MRA_MAX_M + 1][MRA_STAGES];          /* device time, summed */
    int64_t launches[MRA_MAX_M + 1][MRA_STAGES];    /* kernel launches, summed */
    double  flops[MRA_MAX_M + 1][MRA_STAGES];       /* algorithmic FLOPs of one evaluation */
    double  bytes[MRA_MAX_M + 1][MRA_STAGES];       /* algorithmic HBM bytes of one evaluation */
    double  units[MRA_MAX_M + 1][MRA_STAGES];       /* units of work (regions, leaves) of one evaluation */
} mra_stats_t;
int mra_stats(mra_handle* h, mra_stats_t* out);

/*
 * mra_loglik_noalloc -- the log-likelihood of mra_build + mra_loglik in one
 * call that allocates no memory at all (no cudaMalloc, cudaFree, host pinning
 * or allocating library routine).  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory themselves or
 * let a library do so -- code running under a framework whose caching
 * allocator owns the device heap, plug-ins in processes that forbid
 * allocation after start-up, or paths that must not fail half way on memory
 * exhaustion.  Every intermediate lives in one fixed scratch array inside the
 * library image, MRA_NOALLOC_SCRATCH_BYTES per device, which every GPU that
 * loads the library holds until the process exits (enough for problems of
 * roughly n = 16k with M = 4, r = 16, or n = 4096 with M = 3, r = 64).
 *   cfg, theta : as for mra_build / mra_loglik (host), except that only
 *                precision = MRA_PREC_FP64, prune = 0 (complete tree) and the
 *                quadtree (J_level all zero) are supported; other values give
 *                MRA_ERR_ARG naming the field.
 *   locs, y    : device (or managed) pointers, n x 2 row-major locations and
 *                n data; host memory is refused with MRA_ERR_ARG before any
 *                kernel runs.
 *   stream     : cudaStream_t (as void*, NULL = legacy default stream).
 *   loglik_out : host pointer to one double.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  All calls share the array and it keeps the last call's
 * contents; calls that overlap on the GPU (several host threads or streams)
 * race on it and must be serialised by the caller.  The call synchronises
 * `stream` before returning.  Errors: MRA_ERR_ARG, MRA_ERR_LIMIT (the problem
 * needs more scratch than MRA_NOALLOC_SCRATCH_BYTES, or a leaf above
 * MRA_MAX_LEAF), MRA_ERR_NOT_PD, MRA_ERR_CUDA.
 */
#define MRA_NOALLOC_SCRATCH_BYTES (32u << 20)
int mra_loglik_noalloc(const mra_config* cfg, const mra_params* theta, const double* locs,
                       const double* y, int64_t n, void* stream, double* loglik_out);

/* mra_free -- release the handle and its device memory; NULL is a no-op. */
void mra_free(mra_handle* h);

/* Text of the calling thread's last error ("" if none).  Valid until the next call. */
const char* mra_last_error(void);

/* Kernel launches issued by the calling thread since the last reset (reset=1 clears). */
int64_t mra_launch_count(int reset);

#ifdef __cplusplus
}
#endif
#endif /* MRA_H */
