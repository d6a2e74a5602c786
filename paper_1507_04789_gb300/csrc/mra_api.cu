// mra_api.cu -- the extern "C" boundary of the library (declared in include/mra.h).
//
// A handle owns the device state of one problem: the sorted observations, the
// per-level factors of the prior and posterior passes and the leaf factors.
// Device memory is taken in two arenas at build time (the leaf-factor size
// depends on the occupancy of the leaves, known after binning) and, for
// prediction, a third arena that mra_predict grows when it is given more
// points than before; no other entry point allocates after mra_build.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mra.h"
#include "mra_launch.h"

namespace {

thread_local std::string g_err;
thread_local int64_t g_launches = 0;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(MRA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Bump allocator over one cudaMalloc'd block; 256-byte aligned pieces.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  std::vector<std::pair<void**, size_t>> plan;
  template <typename T>
  void want(T** p, size_t count) { plan.push_back({(void**)p, sizeof(T) * count}); }
  static size_t align(size_t b) { return (b + 255) & ~size_t(255); }
  cudaError_t commit() {
    size = 0;
    for (auto& q : plan) size += align(q.second);
    if (size == 0) size = 256;
    cudaError_t e = cudaMalloc((void**)&base, size);
    if (e != cudaSuccess) { base = nullptr; return e; }
    used = 0;
    for (auto& q : plan) {
      *q.first = q.second ? base + used : nullptr;
      used += align(q.second);
    }
    plan.clear();
    return cudaSuccess;
  }
  void release() {
    if (base) cudaFree(base);
    base = nullptr;
  }
};

int gx_for(int r) {
  for (int g = 1; g <= r; ++g)
    if (r % g == 0 && g * g >= r) return g;
  return r;
}

}  // namespace

namespace mra {
// Lets other translation units of the library report errors through
// mra_last_error() and count their launches in mra_launch_count().
void set_last_error(const char* msg) { g_err = msg; }
int64_t* launch_counter() { return &g_launches; }
}  // namespace mra

struct mra_handle {
  mra_config cfg;
  int64_t n = 0;
  int M = 0, r = 0, gx = 0, gy = 0;
  int nlmax = 0;
  cudaStream_t stream = nullptr;
  Arena tree, state;
  // tree (arena 1)
  double* bbox = nullptr;
  int32_t* leaf_id = nullptr;
  int32_t* counts = nullptr;
  int32_t* cursor = nullptr;
  int64_t* off = nullptr;
  int64_t* sq_off = nullptr;
  int32_t* max_count = nullptr;
  int64_t* perm = nullptr;
  int* status = nullptr;
  double* xs = nullptr;
  double* ys = nullptr;
  double* yv = nullptr;
  double* in_locs = nullptr;   // staging of host inputs
  double* in_y = nullptr;
  // state (arena 2)
  mra::LevelState st{};
  mra::LeafState lf{};
  // host
  double* pinned = nullptr;    // small pinned readback buffer
  int64_t ls_cap = 0;          // capacity of the ragged leaf-factor store (doubles)
  // prediction points (arena 3, grown on demand by mra_predict)
  Arena pred;
  int64_t pred_cap = 0;
  double *p_in = nullptr, *p_xs = nullptr, *p_ys = nullptr, *p_U = nullptr, *p_mean = nullptr, *p_var = nullptr;
  int32_t *p_leaf = nullptr, *p_counts = nullptr, *p_cursor = nullptr, *p_max = nullptr;
  int64_t *p_off = nullptr, *p_sq = nullptr, *p_perm = nullptr;
  // gradient (arena 4, allocated by the first mra_loglik_grad)
  Arena grad;
  bool have_grad_arena = false;
  mra::GradState gs{};
  double* d_grad = nullptr;
  mra::Timer timer;
  bool timer_events = false;
  double ktime[8] = {0};
  int64_t kcount[8] = {0};
  bool have_post = false;
  mra_params last{};
};

namespace {

cudaError_t sync_status(mra_handle* h, int* host_status, double* extra, int nextra,
                        const double* const* srcs) {
  cudaError_t e;
  for (int k = 0; k < nextra; ++k)
    if ((e = cudaMemcpyAsync(h->pinned + 4 + k, srcs[k], sizeof(double), cudaMemcpyDeviceToHost, h->stream)))
      return e;
  if ((e = cudaMemcpyAsync(h->pinned, h->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream))) return e;
  if ((e = cudaStreamSynchronize(h->stream))) return e;
  memcpy(host_status, h->pinned, sizeof(int) * 4);
  for (int k = 0; k < nextra; ++k) extra[k] = h->pinned[4 + k];
  return cudaSuccess;
}

void collect_times(mra_handle* h) {
  if (!h->timer.on) return;
  for (int k = 0; k < h->timer.count; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->timer.ev[2 * k], h->timer.ev[2 * k + 1]) == cudaSuccess) {
      h->ktime[h->timer.kind[k]] += ms;
      h->kcount[h->timer.kind[k]] += 1;
    }
  }
  h->timer.count = 0;
}

int status_error(const int* s) {
  if (s[0] == mra::ST_NOT_PD)
    return fail(MRA_ERR_NOT_PD, "matrix not positive definite at level %d, region %d", s[1], s[2]);
  if (s[0] == mra::ST_LIMIT)
    return fail(MRA_ERR_LIMIT, "leaf %d holds more points than the kernels accept", s[2]);
  if (s[0] == mra::ST_ARG)
    return fail(MRA_ERR_ARG, "location %d is outside the bounding box or not finite", s[2]);
  if (s[0] == mra::ST_TIMEOUT)
    return fail(MRA_ERR_CUDA, "a tensor-core wait timed out at level %d, region %d", s[1], s[2]);
  return fail(MRA_ERR_CUDA, "device status %d", s[0]);
}

mra::Shape shape_of(const mra_handle* h) {
  mra::Shape sh;
  sh.M = h->M; sh.r = h->r; sh.gx = h->gx; sh.gy = h->gy;
  for (int k = 0; k < 4; ++k) sh.bbox[k] = h->cfg.bbox[k];
  sh.mixed = h->cfg.precision == MRA_PREC_MIXED;
  return sh;
}

bool params_ok(const mra_params* t) {
  return t && std::isfinite(t->sigma2) && std::isfinite(t->range) && std::isfinite(t->tau2) &&
         t->sigma2 > 0 && t->range > 0 && t->tau2 >= 0;
}

}  // namespace

extern "C" {

const char* mra_last_error(void) { return g_err.c_str(); }

int64_t mra_launch_count(int reset) {
  int64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

void mra_free(mra_handle* h) {
  if (!h) return;
  if (h->timer_events)
    for (int k = 0; k < 2 * mra::MAX_TIMED; ++k) cudaEventDestroy(h->timer.ev[k]);
  h->tree.release();
  h->state.release();
  h->pred.release();
  h->grad.release();
  if (h->pinned) cudaFreeHost(h->pinned);
  delete h;
}

int mra_set_stream(mra_handle* h, void* stream) {
  if (!h) return fail(MRA_ERR_ARG, "null handle");
  h->stream = (cudaStream_t)stream;
  return MRA_OK;
}

int mra_build(const mra_config* cfg, const double* locs, const double* y, int64_t n, int where,
              mra_handle** out) {
  g_err.clear();
  if (!out) return fail(MRA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!cfg || !locs || !y) return fail(MRA_ERR_ARG, "null argument");
  if (n < 1) return fail(MRA_ERR_ARG, "n must be >= 1 (got %lld)", (long long)n);
  if (cfg->M < 0 || cfg->M > MRA_MAX_M) return fail(MRA_ERR_ARG, "M must be in [0, %d]", MRA_MAX_M);
  if (cfg->J != 4) return fail(MRA_ERR_ARG, "J must be 4 (2-D midpoint quadtree)");
  if (cfg->r < 1 || cfg->r > MRA_MAX_R) return fail(MRA_ERR_ARG, "r must be in [1, %d]", MRA_MAX_R);
  if (cfg->cov_family != MRA_COV_EXP && cfg->cov_family != MRA_COV_MATERN15)
    return fail(MRA_ERR_ARG, "unknown covariance family %d", cfg->cov_family);
  if (cfg->nonstat != 0 && cfg->nonstat != 1) return fail(MRA_ERR_ARG, "nonstat must be 0 or 1");
  if (cfg->precision != MRA_PREC_FP64 && cfg->precision != MRA_PREC_MIXED)
    return fail(MRA_ERR_ARG, "unknown precision %d", cfg->precision);
  if (!(cfg->bbox[0] < cfg->bbox[1]) || !(cfg->bbox[2] < cfg->bbox[3]))
    return fail(MRA_ERR_ARG, "empty or invalid bounding box");
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");

  mra_handle* h = new mra_handle();
  h->cfg = *cfg;
  h->n = n;
  h->M = cfg->M;
  h->r = cfg->r;
  h->gx = gx_for(cfg->r);
  h->gy = cfg->r / h->gx;
  const int M = h->M, r = h->r;
  const int64_t nl = int64_t(1) << (2 * M);
  cudaError_t e;
  int rc = MRA_OK;
  int hs[4];

  // ---- arena 1: inputs, tree, sorted observations --------------------------
  Arena& A = h->tree;
  A.want(&h->bbox, 4);
  A.want(&h->leaf_id, n);
  A.want(&h->counts, nl);
  A.want(&h->cursor, nl);
  A.want(&h->off, nl + 1);
  A.want(&h->sq_off, nl + 1);
  A.want(&h->max_count, 1);
  A.want(&h->perm, n);
  A.want(&h->status, 4);
  A.want(&h->xs, n);
  A.want(&h->ys, n);
  A.want(&h->yv, n);
  A.want(&h->in_locs, 2 * n);   // staging for host inputs (mra_build, mra_update, mra_set_data)
  A.want(&h->in_y, n);
  if ((e = A.commit())) { mra_free(h); return fail(MRA_ERR_OOM, "device allocation (tree): %s", cudaGetErrorString(e)); }
  if ((e = cudaMallocHost((void**)&h->pinned, 64 * sizeof(double)))) { mra_free(h); return cuda_fail(e, "cudaMallocHost"); }

  const double* dl = locs;
  const double* dy = y;
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(h->in_locs, locs, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyAsync(h->in_y, y, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream))) {
      mra_free(h); return cuda_fail(e, "copy inputs");
    }
    dl = h->in_locs;
    dy = h->in_y;
  }
  if ((e = cudaMemcpyAsync(h->bbox, cfg->bbox, sizeof(double) * 4, cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) {
    mra_free(h); return cuda_fail(e, "init");
  }
  if ((e = mra::launch_bin(dl, n, h->bbox, M, h->leaf_id, h->counts, h->cursor, h->off, h->sq_off,
                           h->max_count, h->perm, h->status, h->stream, &g_launches)) ||
      (e = mra::launch_gather(dl, dy, h->perm, n, h->xs, h->ys, h->yv, h->stream, &g_launches))) {
    mra_free(h); return cuda_fail(e, "binning");
  }
  {
    int64_t tail[2];
    double got[2];
    const double* srcs[2] = {(const double*)(h->sq_off + nl), (const double*)h->max_count};
    if ((e = sync_status(h, hs, got, 2, srcs))) { mra_free(h); return cuda_fail(e, "binning"); }
    memcpy(&tail[0], &got[0], sizeof(int64_t));
    int32_t mc;
    memcpy(&mc, &got[1], sizeof(int32_t));
    if (hs[0]) { rc = status_error(hs); mra_free(h); return rc; }
    if (mc > MRA_MAX_LEAF) {
      mra_free(h);
      return fail(MRA_ERR_LIMIT, "a leaf holds %d observations (max %d); increase M", mc, MRA_MAX_LEAF);
    }
    h->nlmax = mc < 1 ? 1 : mc;
    // ---- arena 2: factors of every level and of the leaves ------------------
    Arena& B = h->state;
    for (int m = 0; m < M; ++m) {
      const int64_t R = int64_t(1) << (2 * m);
      const int64_t T = int64_t(m + 1) * (m + 2) / 2;
      B.want(&h->st.V[m], R * r * (int64_t)m * r);
      B.want(&h->st.Li[m], R * r * r);
      B.want(&h->st.Acc[m], R * T * r * r);
      B.want(&h->st.Om[m], R * (m + 1) * r);
      B.want(&h->st.Lt[m], R * r * r);
      B.want(&h->st.G[m], R * r * (int64_t)m * r);
      B.want(&h->st.gv[m], R * r);
      B.want(&h->st.dd[m], R);
      B.want(&h->st.uu[m], R);
    }
    double *H, *z, *LS, *d, *u;
    B.want(&H, n * (int64_t)M * r);
    B.want(&z, n);
    B.want(&LS, (size_t)tail[0]);
    h->ls_cap = tail[0];
    B.want(&d, nl);
    B.want(&u, nl);
    if ((e = B.commit())) { mra_free(h); return fail(MRA_ERR_OOM, "device allocation (factors): %s", cudaGetErrorString(e)); }
    h->lf.off = h->off;
    h->lf.sq_off = h->sq_off;
    h->lf.xs = h->xs;
    h->lf.ys = h->ys;
    h->lf.yv = h->yv;
    h->lf.H = H;
    h->lf.z = z;
    h->lf.LS = LS;
    h->lf.d = d;
    h->lf.u = u;
  }
  size_t need = cfg->precision == MRA_PREC_MIXED ? mra::leaf_tc_smem_bytes(h->nlmax) : mra::leaf_smem_bytes(r, h->nlmax);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < need) {
    mra_free(h);
    return fail(MRA_ERR_LIMIT, "leaf kernel needs %zu bytes of shared memory (device allows %d)", need, optin);
  }
  *out = h;
  return MRA_OK;
}

int mra_set_data(mra_handle* h, const double* y, int where) {
  g_err.clear();
  if (!h || !y) return fail(MRA_ERR_ARG, "null argument");
  const double* dy = y;
  cudaError_t e;
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(h->in_y, y, sizeof(double) * h->n, cudaMemcpyHostToDevice, h->stream)))
      return cuda_fail(e, "copy y");
    dy = h->in_y;
  } else if (where != MRA_DEVICE) {
    return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");
  }
  if ((e = mra::launch_gather_y(dy, h->perm, h->n, h->yv, h->stream, &g_launches))) return cuda_fail(e, "gather y");
  h->have_post = false;
  return MRA_OK;
}

int mra_loglik(mra_handle* h, const mra_params* theta, double* loglik_out) {
  g_err.clear();
  if (!h || !loglik_out) return fail(MRA_ERR_ARG, "null argument");
  if (!params_ok(theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0, all finite");
  h->have_post = false;
  mra::Cov cv{theta->sigma2, theta->range, h->cfg.cov_family, h->cfg.nonstat};
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) return cuda_fail(e, "memset");
  if ((e = mra::launch_loglik(shape_of(h), cv, theta->tau2, h->st, h->lf, h->nlmax, h->status, h->stream,
                              &g_launches, &h->timer)))
    return cuda_fail(e, "loglik launch");
  int hs[4];
  double du[2];
  const double* srcs[2];
  if (h->M > 0) { srcs[0] = h->st.dd[0]; srcs[1] = h->st.uu[0]; }
  else { srcs[0] = h->lf.d; srcs[1] = h->lf.u; }
  if ((e = sync_status(h, hs, du, 2, srcs))) return cuda_fail(e, "loglik");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  *loglik_out = -0.5 * (du[0] + du[1]) - 0.5 * (double)h->n * std::log(2.0 * M_PI);
  h->have_post = true;
  h->last = *theta;
  return MRA_OK;
}

int mra_region_terms(mra_handle* h, int level, double* d_out, double* u_out) {
  g_err.clear();
  if (!h || !d_out || !u_out) return fail(MRA_ERR_ARG, "null argument");
  if (level < 0 || level > h->M) return fail(MRA_ERR_ARG, "level must be in [0, M]");
  if (!h->have_post) return fail(MRA_ERR_STATE, "no log-likelihood evaluated yet");
  const int64_t R = int64_t(1) << (2 * level);
  const double* d = level == h->M ? h->lf.d : h->st.dd[level];
  const double* u = level == h->M ? h->lf.u : h->st.uu[level];
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_out, d, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(u_out, u, sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "region terms");
  return MRA_OK;
}

int mra_leaf_offsets(mra_handle* h, int64_t* off_out, int64_t* perm_out) {
  g_err.clear();
  if (!h || !off_out) return fail(MRA_ERR_ARG, "null argument");
  const int64_t nl = int64_t(1) << (2 * h->M);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(off_out, h->off, sizeof(int64_t) * (nl + 1), cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "offsets");
  if (perm_out && (e = cudaMemcpyAsync(perm_out, h->perm, sizeof(int64_t) * h->n, cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "perm");
  if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "offsets");
  return MRA_OK;
}

static int ensure_grad_arena(mra_handle* h) {
  if (h->have_grad_arena) return MRA_OK;
  const int M = h->M, r = h->r;
  const int64_t n = h->n, nl = int64_t(1) << (2 * M);
  Arena& G = h->grad;
  for (int m = 0; m < M; ++m) {
    const int64_t R = int64_t(1) << (2 * m);
    G.want(&h->st.L[m], R * r * r);
    G.want(&h->st.Ltf[m], R * r * r);
    G.want(&h->gs.Abar[m], R * r * (int64_t)(m + 1) * r);
    G.want(&h->gs.Obar[m], R * r);
    G.want(&h->gs.GB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.VB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.XB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.Up[m], R * (int64_t)m * (m + 1) / 2 * r * r);
  }
  if (M > 0) G.want(&h->gs.PartLeaf, (nl / 4) * (int64_t)M * (M + 1) / 2 * r * r);
  G.want(&h->lf.VF, n * (int64_t)M * r);
  G.want(&h->lf.LSf, (size_t)h->ls_cap);
  G.want(&h->gs.HB, n * (int64_t)M * r);
  G.want(&h->gs.VBF, n * (int64_t)M * r);
  G.want(&h->gs.XBF, n * (int64_t)M * r);
  G.want(&h->gs.T, 3 * (size_t)h->ls_cap);
  int64_t slots = nl;
  for (int m = 0; m < M; ++m) slots += int64_t(1) << (2 * m);
  G.want(&h->gs.gpart, 3 * slots);
  G.want(&h->d_grad, 4);
  cudaError_t e = G.commit();
  if (e) {
    for (int m = 0; m < M; ++m) { h->st.L[m] = nullptr; h->st.Ltf[m] = nullptr; }
    h->lf.VF = nullptr;
    h->lf.LSf = nullptr;
    return fail(MRA_ERR_OOM, "device allocation (gradient): %s", cudaGetErrorString(e));
  }
  h->have_grad_arena = true;
  return MRA_OK;
}

int mra_loglik_grad(mra_handle* h, const mra_params* theta, double* loglik_out, double* grad_out) {
  g_err.clear();
  if (!h || !loglik_out || !grad_out) return fail(MRA_ERR_ARG, "null argument");
  if (!params_ok(theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0, all finite");
  int rc = ensure_grad_arena(h);
  if (rc) return rc;
  h->have_post = false;
  mra::Cov cv{theta->sigma2, theta->range, h->cfg.cov_family, h->cfg.nonstat};
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) return cuda_fail(e, "memset");
  if ((e = mra::launch_loglik(shape_of(h), cv, theta->tau2, h->st, h->lf, h->nlmax, h->status, h->stream,
                              &g_launches, &h->timer)))
    return cuda_fail(e, "loglik launch");
  if ((e = mra::launch_grad(shape_of(h), cv, h->st, h->lf, h->gs, h->d_grad, h->stream, &g_launches, &h->timer)))
    return cuda_fail(e, "gradient launch");
  int hs[4];
  double vals[5];
  const double* srcs[5];
  if (h->M > 0) { srcs[0] = h->st.dd[0]; srcs[1] = h->st.uu[0]; }
  else { srcs[0] = h->lf.d; srcs[1] = h->lf.u; }
  srcs[2] = h->d_grad;
  srcs[3] = h->d_grad + 1;
  srcs[4] = h->d_grad + 2;
  if ((e = sync_status(h, hs, vals, 5, srcs))) return cuda_fail(e, "gradient");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  *loglik_out = -0.5 * (vals[0] + vals[1]) - 0.5 * (double)h->n * std::log(2.0 * M_PI);
  grad_out[0] = vals[2];
  grad_out[1] = vals[3];
  grad_out[2] = vals[4];
  h->have_post = true;
  h->last = *theta;
  return MRA_OK;
}

int mra_update(mra_handle* h, const double* locs, const double* y, int where) {
  g_err.clear();
  if (!h || !locs || !y) return fail(MRA_ERR_ARG, "null argument");
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");
  const int64_t n = h->n, nl = int64_t(1) << (2 * h->M);
  cudaError_t e;
  const double* dl = locs;
  const double* dy = y;
  h->have_post = false;
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(h->in_locs, locs, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyAsync(h->in_y, y, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream)))
      return cuda_fail(e, "copy inputs");
    dl = h->in_locs;
    dy = h->in_y;
  }
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) return cuda_fail(e, "memset");
  if ((e = mra::launch_bin(dl, n, h->bbox, h->M, h->leaf_id, h->counts, h->cursor, h->off, h->sq_off,
                           h->max_count, h->perm, h->status, h->stream, &g_launches)) ||
      (e = mra::launch_gather(dl, dy, h->perm, n, h->xs, h->ys, h->yv, h->stream, &g_launches)))
    return cuda_fail(e, "binning");
  int hs[4];
  double got[2];
  const double* srcs[2] = {(const double*)(h->sq_off + nl), (const double*)h->max_count};
  if ((e = sync_status(h, hs, got, 2, srcs))) return cuda_fail(e, "binning");
  if (hs[0]) return status_error(hs);
  int64_t tail;
  int32_t mc;
  memcpy(&tail, &got[0], sizeof tail);
  memcpy(&mc, &got[1], sizeof mc);
  if (mc > h->nlmax || tail > h->ls_cap)
    return fail(MRA_ERR_LIMIT, "new partition needs leaves of %d (handle has %d) or %lld leaf-factor doubles "
                "(handle has %lld); build a new handle", mc, h->nlmax, (long long)tail, (long long)h->ls_cap);
  return MRA_OK;
}

int mra_enable_timing(mra_handle* h, int on) {
  g_err.clear();
  if (!h) return fail(MRA_ERR_ARG, "null handle");
  if (on && !h->timer_events) {
    for (int k = 0; k < 2 * mra::MAX_TIMED; ++k) {
      cudaError_t e = cudaEventCreate(&h->timer.ev[k]);
      if (e) return cuda_fail(e, "cudaEventCreate");
    }
    h->timer_events = true;
  }
  h->timer.on = on != 0;
  h->timer.count = 0;
  for (int k = 0; k < 8; ++k) { h->ktime[k] = 0.0; h->kcount[k] = 0; }
  return MRA_OK;
}

int mra_kernel_times(mra_handle* h, int kind, double* total_ms, int64_t* launches) {
  g_err.clear();
  if (!h || !total_ms || !launches) return fail(MRA_ERR_ARG, "null argument");
  if (kind < 0 || kind >= 8) return fail(MRA_ERR_ARG, "unknown kernel kind %d", kind);
  *total_ms = h->ktime[kind];
  *launches = h->kcount[kind];
  return MRA_OK;
}

int mra_predict(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                double* mean_out, double* var_out) {
  g_err.clear();
  if (!h || !theta || !plocs || !mean_out || !var_out) return fail(MRA_ERR_ARG, "null argument");
  if (np < 1) return fail(MRA_ERR_ARG, "np must be >= 1");
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");
  if (!h->have_post) return fail(MRA_ERR_STATE, "call mra_loglik before mra_predict");
  if (theta->sigma2 != h->last.sigma2 || theta->range != h->last.range || theta->tau2 != h->last.tau2)
    return fail(MRA_ERR_STATE, "theta differs from the last mra_loglik; evaluate the log-likelihood at it first");
  const int M = h->M, r = h->r;
  const int64_t nl = int64_t(1) << (2 * M);
  cudaError_t e;
  if (np > h->pred_cap) {
    h->pred.release();
  h->grad.release();
    Arena& P = h->pred;
    P.want(&h->p_in, 2 * np);
    P.want(&h->p_xs, np);
    P.want(&h->p_ys, np);
    P.want(&h->p_U, np * (int64_t)M * r);
    P.want(&h->p_mean, np);
    P.want(&h->p_var, np);
    P.want(&h->p_leaf, np);
    P.want(&h->p_counts, nl);
    P.want(&h->p_cursor, nl);
    P.want(&h->p_max, 2);
    P.want(&h->p_off, nl + 1);
    P.want(&h->p_sq, nl + 1);
    P.want(&h->p_perm, np);
    if ((e = P.commit())) {
      h->pred_cap = 0;
      return fail(MRA_ERR_OOM, "device allocation (prediction): %s", cudaGetErrorString(e));
    }
    h->pred_cap = np;
  }
  const double* dp = plocs;
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(h->p_in, plocs, sizeof(double) * 2 * np, cudaMemcpyHostToDevice, h->stream)))
      return cuda_fail(e, "copy prediction locations");
    dp = h->p_in;
  }
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) return cuda_fail(e, "memset");
  if ((e = mra::launch_bin(dp, np, h->bbox, M, h->p_leaf, h->p_counts, h->p_cursor, h->p_off, h->p_sq, h->p_max,
                           h->p_perm, h->status, h->stream, &g_launches, false)) ||
      (e = mra::launch_gather(dp, nullptr, h->p_perm, np, h->p_xs, h->p_ys, nullptr, h->stream, &g_launches)))
    return cuda_fail(e, "binning prediction points");
  int hs[4];
  double got[1];
  const double* srcs[1] = {(const double*)h->p_max};
  if ((e = sync_status(h, hs, got, 1, srcs))) return cuda_fail(e, "binning prediction points");
  if (hs[0]) return status_error(hs);
  int32_t maxp;
  memcpy(&maxp, &got[0], sizeof maxp);
  mra::PredState ps;
  ps.off = h->p_off;
  ps.perm = h->p_perm;
  ps.xs = h->p_xs;
  ps.ys = h->p_ys;
  ps.U = h->p_U;
  ps.mean = where == MRA_DEVICE ? mean_out : h->p_mean;
  ps.var = where == MRA_DEVICE ? var_out : h->p_var;
  mra::Cov cv{theta->sigma2, theta->range, h->cfg.cov_family, h->cfg.nonstat};
  if ((e = mra::launch_predict(shape_of(h), cv, h->st, h->lf, h->nlmax, ps, maxp, h->stream, &g_launches,
                               &h->timer)))
    return cuda_fail(e, "predict launch");
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(mean_out, h->p_mean, sizeof(double) * np, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(var_out, h->p_var, sizeof(double) * np, cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "copy predictions");
  }
  if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "predict");
  collect_times(h);
  return MRA_OK;
}

}  // extern "C"
