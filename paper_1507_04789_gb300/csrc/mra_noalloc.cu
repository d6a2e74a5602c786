// mra_noalloc.cu -- log-likelihood entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code running inside a framework whose
// caching allocator owns the device heap, plug-ins loaded into a process that
// forbids allocations after start-up (real-time or certified code paths), or
// code that must not fail on memory exhaustion half way through.  For them,
// mra_loglik_noalloc evaluates the same log-likelihood as mra_build followed by
// mra_loglik, with every intermediate (partition, factors of every level, leaf
// factors) carved out of one fixed scratch array that lives in the library
// image: MRA_NOALLOC_SCRATCH_BYTES bytes per device, held by every GPU that
// loads the library until the process exits.  Only the caller's inputs and the
// returned scalar live outside it.
//
// The scratch array is a file-scope __device__ variable.  Host code may not use
// its name as an address (on the host it is only a stand-in symbol), so the
// first call on each device asks the runtime for its device address with
// cudaGetSymbolAddress while that device is current, caches it, and passes it
// to the kernels.  That first call should therefore come before any stream
// capture on that device.  Every call shares the one array and it keeps the
// last call's contents: the counters and the status word that must start at
// zero are cleared by each call, everything else is written before it is read.
// Calls whose work overlaps on the GPU (other host threads, other streams)
// race on the array and must be serialised by the caller.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/mra.h"
#include "mra_launch.h"

namespace {

constexpr size_t kScratchBytes = size_t(MRA_NOALLOC_SCRATCH_BYTES);
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scratch_mu;
constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (set up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Bump allocation inside the scratch array (256-byte aligned pieces).
struct Carve {
  char* base;
  size_t cap, used = 0;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (sizeof(T) * count + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return count ? p : nullptr;
  }
  bool fits() const { return used <= cap; }
};

int err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  mra::set_last_error(buf);
  return code;
}

int cuda_err(cudaError_t e, const char* where) {
  return err(MRA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

int gx_of(int r) {
  for (int g = 1; g <= r; ++g)
    if (r % g == 0 && g * g >= r) return g;
  return r;
}

int status_code(const int* s) {
  if (s[0] == mra::ST_NOT_PD)
    return err(MRA_ERR_NOT_PD, "matrix not positive definite at level %d, region %d", s[1], s[2]);
  if (s[0] == mra::ST_LIMIT) return err(MRA_ERR_LIMIT, "leaf %d holds too many points", s[2]);
  if (s[0] == mra::ST_ARG) return err(MRA_ERR_ARG, "location %d is outside the bounding box or not finite", s[2]);
  return err(MRA_ERR_CUDA, "device status %d", s[0]);
}

}  // namespace

extern "C" int mra_loglik_noalloc(const mra_config* cfg, const mra_params* theta, const double* locs,
                                  const double* y, int64_t n, void* stream, double* loglik_out) {
  mra::set_last_error("");
  if (!cfg || !theta || !locs || !y || !loglik_out) return err(MRA_ERR_ARG, "null argument");
  if (n < 1) return err(MRA_ERR_ARG, "n must be >= 1");
  if (cfg->M < 0 || cfg->M > MRA_MAX_M) return err(MRA_ERR_ARG, "M must be in [0, %d]", MRA_MAX_M);
  if (cfg->J != 4) return err(MRA_ERR_ARG, "J must be 4 (2-D midpoint quadtree)");
  if (cfg->J_level[0] != 0)
    return err(MRA_ERR_ARG, "level-varying J needs mra_build (the allocation-free entry point takes the quadtree)");
  if (cfg->r < 1 || cfg->r > MRA_MAX_R) return err(MRA_ERR_ARG, "r must be in [1, %d]", MRA_MAX_R);
  if (cfg->cov_family != MRA_COV_EXP && cfg->cov_family != MRA_COV_MATERN15 && cfg->cov_family != MRA_COV_MATERN)
    return err(MRA_ERR_ARG, "unknown covariance family %d", cfg->cov_family);
  if (cfg->cov_family == MRA_COV_MATERN && !(std::isfinite(theta->nu) && theta->nu >= 0.05 && theta->nu <= 20.0))
    return err(MRA_ERR_ARG, "MRA_COV_MATERN needs 0.05 <= nu <= 20");
  if (cfg->nonstat != 0 && cfg->nonstat != 1) return err(MRA_ERR_ARG, "nonstat must be 0 or 1");
  if (cfg->precision != MRA_PREC_FP64)
    return err(MRA_ERR_ARG, "precision must be MRA_PREC_FP64 in the allocation-free entry point (got %d)",
               cfg->precision);
  if (cfg->prune != 0)
    return err(MRA_ERR_ARG, "prune must be 0 in the allocation-free entry point (complete tree only)");
  if (cfg->stream_level > 0)
    return err(MRA_ERR_ARG, "stream_level must be 0 or -1 in the allocation-free entry point");
  if (!(cfg->bbox[0] < cfg->bbox[1]) || !(cfg->bbox[2] < cfg->bbox[3]))
    return err(MRA_ERR_ARG, "empty or invalid bounding box");
  if (!(std::isfinite(theta->sigma2) && std::isfinite(theta->range) && std::isfinite(theta->tau2) &&
        theta->sigma2 > 0 && theta->range > 0 && theta->tau2 >= 0))
    return err(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0, all finite");

  // locs and y are read by kernels: refuse host memory here rather than let a
  // kernel dereference it (cudaPointerGetAttributes allocates nothing)
  for (int q = 0; q < 2; ++q) {
    cudaPointerAttributes pa{};
    const cudaError_t pe = cudaPointerGetAttributes(&pa, q == 0 ? (const void*)locs : (const void*)y);
    if (pe != cudaSuccess) {
      cudaGetLastError();   // a failed query leaves its error as the runtime's last error: clear it
      return err(MRA_ERR_ARG, "%s is not a pointer the CUDA runtime knows: %s", q == 0 ? "locs" : "y",
                 cudaGetErrorString(pe));
    }
    if (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged)
      return err(MRA_ERR_ARG, "%s must be device (or managed) memory", q == 0 ? "locs" : "y");
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t* launches = mra::launch_counter();
  void* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");

  const int M = cfg->M, r = cfg->r;
  const int64_t nl = int64_t(1) << (2 * M);
  Carve C{(char*)base, kScratchBytes};
  // ---- partition --------------------------------------------------------------
  double* bbox = C.take<double>(4);
  int32_t* leaf_id = C.take<int32_t>(n);
  int32_t* counts = C.take<int32_t>(nl);
  int32_t* cursor = C.take<int32_t>(nl);
  int64_t* off = C.take<int64_t>(nl + 1);
  int64_t* sq_off = C.take<int64_t>(nl + 1);
  int32_t* max_count = C.take<int32_t>(2);
  int64_t* perm = C.take<int64_t>(n);
  int* status = C.take<int>(4);
  double* xs = C.take<double>(n);
  double* ys = C.take<double>(n);
  double* yv = C.take<double>(n);
  if (!C.fits())
    return err(MRA_ERR_LIMIT, "problem needs more than the %zu bytes of scratch of the allocation-free entry point",
               kScratchBytes);
  if ((e = cudaMemcpyAsync(bbox, cfg->bbox, sizeof(double) * 4, cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemsetAsync(status, 0, sizeof(int) * 4, s)))
    return cuda_err(e, "init");
  if ((e = mra::launch_bin(locs, n, bbox, M, mra::QUAD_HALVINGS, mra::QUAD_HALVINGS, leaf_id, counts, cursor, off,
                           sq_off, max_count, perm, status, s,
                           launches)))
    return cuda_err(e, "binning");
  int hs[4];
  int64_t tail = 0;
  int32_t mc = 0;
  if ((e = cudaMemcpyAsync(&tail, sq_off + nl, sizeof tail, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(&mc, max_count, sizeof mc, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(hs, status, sizeof hs, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
    return cuda_err(e, "binning");
  if (hs[0]) return status_code(hs);
  if (mc > MRA_MAX_LEAF)
    return err(MRA_ERR_LIMIT, "a leaf holds %d observations (max %d); increase M", mc, MRA_MAX_LEAF);
  const int nlmax = mc < 1 ? 1 : mc;
  // ---- tree tables (complete tree: identity), factors of every level and of the leaves
  mra::LevelState st{};
  for (int m = 0; m <= M; ++m) {
    const int64_t R = int64_t(1) << (2 * m);
    st.nreg[m] = (int)R;
    st.mort[m] = C.take<int32_t>(R);
    st.cid[m] = C.take<int32_t>(R);
    if (m > 0) st.par[m] = C.take<int32_t>(R);
    if (m < M) {
      st.cfirst[m] = C.take<int32_t>(R);
      st.ccnt[m] = C.take<int32_t>(R);
    }
  }
  for (int m = 0; m < M; ++m) {
    const int64_t R = int64_t(1) << (2 * m);
    const int64_t T = int64_t(m + 1) * (m + 2) / 2;
    st.V[m] = C.take<double>(R * r * (int64_t)m * r);
    st.Li[m] = C.take<double>(R * r * r);
    st.Acc[m] = C.take<double>(R * T * r * r);
    st.Om[m] = C.take<double>(R * (m + 1) * r);
    st.Lt[m] = C.take<double>(R * r * r);
    st.G[m] = C.take<double>(R * r * (int64_t)m * r);
    st.gv[m] = C.take<double>(R * r);
    st.dd[m] = C.take<double>(R);
    st.uu[m] = C.take<double>(R);
  }
  mra::LeafState lf{};
  lf.off = off;
  lf.sq_off = sq_off;
  lf.xs = xs;
  lf.ys = ys;
  lf.yv = yv;
  lf.H = C.take<double>(n * (int64_t)M * r);
  lf.z = C.take<double>(n);
  lf.LS = C.take<double>((size_t)tail);
  lf.d = C.take<double>(nl);
  lf.u = C.take<double>(nl);
  mra::Desc* d_desc = C.take<mra::Desc>(1);
  if (!C.fits())
    return err(MRA_ERR_LIMIT, "problem needs %zu bytes of scratch; the allocation-free entry point has %zu",
               C.used, kScratchBytes);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < mra::leaf_smem_bytes(r, nlmax))
    return err(MRA_ERR_LIMIT, "leaf kernel needs more shared memory than the device allows");
  // ---- the evaluation -----------------------------------------------------------
  mra::Shape sh;
  sh.M = M;
  sh.r = r;
  sh.gx = gx_of(r);
  sh.gy = r / sh.gx;
  for (int k = 0; k < 4; ++k) sh.bbox[k] = cfg->bbox[k];
  sh.mixed = 0;
  sh.hx = sh.hy = mra::QUAD_HALVINGS;
  mra::Desc hd{};
  hd.sh = sh;
  hd.cv = mra::make_cov(theta->sigma2, theta->range, cfg->cov_family, cfg->nonstat, theta->nu);
  hd.tau2 = theta->tau2;
  hd.nlmax = nlmax;
  hd.st = st;
  hd.lf = lf;
  mra::Plan plan;
  plan.maxM = M;
  plan.tile = mra::tile_for_r(r);
  plan.mixed = 0;
  plan.nlmax = nlmax;
  for (int m = 0; m < M; ++m) {
    plan.n_lvl[m] = st.nreg[m];
    if (m > 0) plan.n_agg[m] = st.nreg[m - 1];
  }
  plan.n_leaf = st.nreg[M];
  if (M > 0) {
    plan.n_syrk = st.nreg[M - 1];
    plan.t_syrk = M * (M + 1) / 2;
  }
  mra::Timer no_timer;
  if ((e = mra::launch_identity_tree(st, M, mra::QUAD_HALVINGS, mra::QUAD_HALVINGS, s, launches)) ||
      (e = cudaMemcpyAsync(d_desc, &hd, sizeof hd, cudaMemcpyHostToDevice, s)) ||
      (e = mra::launch_gather(locs, y, perm, n, xs, ys, yv, s, launches)) ||
      (e = mra::launch_loglik(plan, d_desc, status, s, launches, &no_timer)))
    return cuda_err(e, "loglik launch");
  double d = 0.0, u = 0.0;
  const double* dsrc = M > 0 ? st.dd[0] : lf.d;
  const double* usrc = M > 0 ? st.uu[0] : lf.u;
  if ((e = cudaMemcpyAsync(&d, dsrc, sizeof d, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(&u, usrc, sizeof u, cudaMemcpyDeviceToHost, s)) ||
      (e = cudaMemcpyAsync(hs, status, sizeof hs, cudaMemcpyDeviceToHost, s)) || (e = cudaStreamSynchronize(s)))
    return cuda_err(e, "loglik");
  if (hs[0]) return status_code(hs);
  *loglik_out = -0.5 * (d + u) - 0.5 * (double)n * std::log(2.0 * M_PI);
  return MRA_OK;
}
