// mra_api.cu -- the extern "C" boundary of the library (declared in include/mra.h).
//
// A handle owns the device state of one problem: the sorted observations, the
// tree tables, the per-level factors of the prior and posterior passes and the
// leaf factors, plus a descriptor of all of it in device memory that every
// kernel reads.  Device memory is taken in arenas at build time (the sizes
// depend on the leaf occupancy, known after binning); mra_predict grows a
// prediction arena and the first mra_loglik_grad allocates the adjoint arena;
// no other entry point allocates after mra_build.
//
// A batch handle (mra_build_batch) owns one handle per dataset and evaluates
// all of them with one launch per level: every CTA of a launch is mapped to a
// (dataset, region) pair by a work list.  The launch sequence is captured once
// as a CUDA graph and replayed for every new set of parameters.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/mra.h"
#include "mra_launch.h"

static_assert(mra::JOINT_TILE == MRA_MAX_JOINT_LEAF, "one CTA holds a leaf's prediction points");

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
    if (e != cudaSuccess) {
      base = nullptr;
      plan.clear();
      return e;
    }
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

bool params_ok(const mra_params* t) {
  return t && std::isfinite(t->sigma2) && std::isfinite(t->range) && std::isfinite(t->tau2) && t->sigma2 > 0 &&
         t->range > 0 && t->tau2 >= 0;
}

// The smoothness of MRA_COV_MATERN must lie in the range its Bessel-function
// evaluation is accurate on.
bool nu_ok(int family, const mra_params* t) {
  return family != MRA_COV_MATERN || (std::isfinite(t->nu) && t->nu >= 0.05 && t->nu <= 20.0);
}

// Per-level midpoint halvings of a configuration (Sec. 2.2; J may vary with the
// level, Sec. 4.3): with L_m = log2(J_1 ... J_m), level m halves
// ceil(L_m / 2) - ceil(L_{m-1} / 2) times in x and floor(L_m / 2) -
// floor(L_{m-1} / 2) times in y (the halvings alternate x, y, x, ... over the
// whole sequence, so J = 4 is the quadtree).  Packed 4 bits per level.
void config_halvings(const mra_config* cfg, unsigned long long& hx, unsigned long long& hy) {
  hx = hy = 0;
  int L = 0;
  for (int m = 1; m <= cfg->M; ++m) {
    const int Jm = cfg->J_level[0] ? cfg->J_level[m - 1] : 4;
    int b = 0;
    while ((1 << b) < Jm) ++b;
    const int L1 = L + b;
    hx |= (unsigned long long)((L1 + 1) / 2 - (L + 1) / 2) << (4 * m);
    hy |= (unsigned long long)(L1 / 2 - L / 2) << (4 * m);
    L = L1;
  }
}

int check_config(const mra_config* cfg) {
  if (cfg->M < 0 || cfg->M > MRA_MAX_M) return fail(MRA_ERR_ARG, "M must be in [0, %d]", MRA_MAX_M);
  if (cfg->J_level[0] == 0) {
    if (cfg->J != 4) return fail(MRA_ERR_ARG, "J must be 4 (2-D midpoint quadtree), or J_level set");
    for (int m = 1; m < MRA_MAX_M; ++m)
      if (cfg->J_level[m]) return fail(MRA_ERR_ARG, "J_level[0] is 0 but J_level[%d] is not", m);
  } else {
    int L = 0;
    for (int m = 1; m <= MRA_MAX_M; ++m) {
      const int Jm = cfg->J_level[m - 1];
      if (m > cfg->M) {
        if (Jm) return fail(MRA_ERR_ARG, "J_level[%d] set beyond level M = %d", m - 1, cfg->M);
        continue;
      }
      if (Jm != 2 && Jm != 4 && Jm != 8 && Jm != 16)
        return fail(MRA_ERR_ARG, "J_level[%d] = %d: each J_m must be 2, 4, 8 or 16", m - 1, Jm);
      if (m == cfg->M && Jm > 4 && cfg->precision == MRA_PREC_EMU)   // (a parent's leaves in at most four 128-row tiles)
        return fail(MRA_ERR_ARG, "J_M (the leaves' level) must be 2 or 4 in the emulated form");
      L += Jm == 2 ? 1 : Jm == 4 ? 2 : Jm == 8 ? 3 : 4;
    }
    if (L > 24) return fail(MRA_ERR_ARG, "J_1 ... J_M = 2^%d leaves: at most 2^24", L);
  }
  if (cfg->r < 1 || cfg->r > MRA_MAX_R) return fail(MRA_ERR_ARG, "r must be in [1, %d]", MRA_MAX_R);
  if (cfg->cov_family != MRA_COV_EXP && cfg->cov_family != MRA_COV_MATERN15 && cfg->cov_family != MRA_COV_MATERN)
    return fail(MRA_ERR_ARG, "unknown covariance family %d", cfg->cov_family);
  if (cfg->nonstat != 0 && cfg->nonstat != 1) return fail(MRA_ERR_ARG, "nonstat must be 0 or 1");
  if (cfg->precision != MRA_PREC_FP64 && cfg->precision != MRA_PREC_MIXED && cfg->precision != MRA_PREC_EMU)
    return fail(MRA_ERR_ARG, "unknown precision %d", cfg->precision);
  if (cfg->prune != 0 && cfg->prune != 1) return fail(MRA_ERR_ARG, "prune must be 0 or 1");
  if (!(cfg->bbox[0] < cfg->bbox[1]) || !(cfg->bbox[2] < cfg->bbox[3]))
    return fail(MRA_ERR_ARG, "empty or invalid bounding box");
  return MRA_OK;
}

// Host tree tables (Sec. 2.2): active regions of every level in region-id order
// (the per-level child digits; Morton order for the quadtree).
struct Tables {
  std::vector<std::vector<int32_t>> mort, par, cfirst, ccnt, cid;
  std::vector<int32_t> nreg;
  std::vector<int> bits;   // level m: log2 J_m (bits of the child digit); entry 0 unused
};

// Groups of leaves for the emulated leaf kernel: consecutive children of one
// level-(M-1) region, at most LGRP_MAX of them and MRA_MAX_LEAF observations in
// all (the kernel stacks a group in one 128-row tile).  Parents [p0, p1).
void leaf_groups(const Tables& T, int M, const std::vector<int32_t>& counts, int64_t p0, int64_t p1, int chunk,
                 std::vector<int2>& items, std::vector<int>& cnt) {
  for (int64_t p = p0; p < p1; ++p) {
    const int32_t cf = T.cfirst[M - 1][p], ce = cf + T.ccnt[M - 1][p];
    for (int32_t F = cf; F < ce;) {
      int g = 1, rows = counts[T.mort[M][F]];
      while (F + g < ce && g < mra::LGRP_MAX && rows + counts[T.mort[M][F + g]] <= MRA_MAX_LEAF)
        rows += counts[T.mort[M][F + g++]];
      items.push_back(make_int2(chunk, F));
      cnt.push_back(g);
      F += g;
    }
  }
}

// Groups of sibling regions of level m >= 1 for the prior kernel: consecutive
// children of one level-(m-1) region, at most gmax of them.  Parents [p0, p1).
void prior_groups(const Tables& T, int m, int gmax, int64_t p0, int64_t p1, int chunk, std::vector<int2>& items,
                  std::vector<int>& cnt) {
  for (int64_t p = p0; p < p1; ++p) {
    const int32_t cf = T.cfirst[m - 1][p], ce = cf + T.ccnt[m - 1][p];
    for (int32_t c = cf; c < ce; c += gmax) {
      items.push_back(make_int2(chunk, c));
      cnt.push_back(std::min(gmax, ce - c));
    }
  }
}

// Groups of sibling level-(M-1) regions for the leaf chain kernel: consecutive
// children of one level-(M-2) region q, q in [p0, p1), at most LGRP_MAX of them
// and 128 observations in all (obs_pref: prefix sums of the leaf counts by
// Morton id); a region of more than 128 is a group of its own.
void chain_groups(const Tables& T, int M, const std::vector<int64_t>& obs_pref, int64_t p0, int64_t p1, int chunk,
                  std::vector<int2>& items, std::vector<int>& cnt) {
  auto rows = [&](int32_t P) {
    const int64_t pm = T.mort[M - 1][P];
    return obs_pref[(pm + 1) << T.bits[M]] - obs_pref[pm << T.bits[M]];
  };
  for (int64_t q = p0; q < p1; ++q) {
    const int32_t cf = T.cfirst[M - 2][q], ce = cf + T.ccnt[M - 2][q];
    for (int32_t P = cf; P < ce;) {
      int g = 1;
      int64_t n = rows(P);
      while (P + g < ce && g < mra::LGRP_MAX && n + rows(P + g) <= 128) n += rows(P + g++);
      items.push_back(make_int2(chunk, P));
      cnt.push_back(g);
      P += g;
    }
  }
}

void build_tables(int M, unsigned long long hx, unsigned long long hy, bool prune, const std::vector<int32_t>& counts,
                  Tables& T) {
  T.bits.assign(M + 1, 0);
  for (int m = 1; m <= M; ++m) T.bits[m] = mra::lvl_bits(hx, hy, m);
  T.mort.assign(M + 1, {});
  T.par.assign(M + 1, {});
  T.cfirst.assign(M + 1, {});
  T.ccnt.assign(M + 1, {});
  T.cid.assign(M + 1, {});
  T.nreg.assign(M + 1, 0);
  std::vector<std::vector<uint8_t>> act(M + 1);
  act[M].resize(counts.size());
  for (size_t f = 0; f < counts.size(); ++f) act[M][f] = !prune || counts[f] > 0;
  for (int m = M - 1; m >= 0; --m) {
    const size_t cnt = size_t(1) << mra::lvl_depth(hx, hy, m);
    const int bc = T.bits[m + 1];
    act[m].assign(cnt, 0);
    for (size_t i = 0; i < cnt; ++i) {
      bool a = !prune;
      for (size_t j = 0; j < (size_t(1) << bc) && !a; ++j) a = act[m + 1][(i << bc) + j];
      act[m][i] = a;
    }
  }
  act[0][0] = 1;
  for (int m = 0; m <= M; ++m) {
    const size_t cnt = size_t(1) << mra::lvl_depth(hx, hy, m);
    T.cid[m].assign(cnt, -1);
    for (size_t i = 0; i < cnt; ++i)
      if (act[m][i]) {
        T.cid[m][i] = (int32_t)T.mort[m].size();
        T.mort[m].push_back((int32_t)i);
      }
    T.nreg[m] = (int32_t)T.mort[m].size();
  }
  for (int m = 0; m <= M; ++m) {
    const int32_t n = T.nreg[m];
    if (m > 0) {
      T.par[m].resize(n);
      for (int32_t c = 0; c < n; ++c) T.par[m][c] = T.cid[m - 1][T.mort[m][c] >> T.bits[m]];
    }
    if (m < M) {
      T.cfirst[m].assign(n, 0);
      T.ccnt[m].assign(n, 0);
      for (int32_t c = 0; c < n; ++c) {
        const size_t base = (size_t)T.mort[m][c] << T.bits[m + 1];
        int32_t first = -1, k = 0;
        for (int j = 0; j < (1 << T.bits[m + 1]); ++j) {
          const int32_t id = T.cid[m + 1][base + j];
          if (id >= 0) {
            if (first < 0) first = id;
            ++k;
          }
        }
        T.cfirst[m][c] = first < 0 ? 0 : first;
        T.ccnt[m][c] = k;
      }
    }
  }
}

}  // namespace

namespace mra {
// Lets other translation units of the library report errors through
// mra_last_error() and count their launches in mra_launch_count().
void set_last_error(const char* msg) { g_err = msg; }
int64_t* launch_counter() { return &g_launches; }
}  // namespace mra

namespace {
// One subtree of a streamed evaluation: a level-s region and everything below
// it.  Its compact region ids of every level m > s form the range [c0, c1)
// (compact ids keep Morton order), its observations [obs0, obs1) and its
// leaves' factor blocks [ls0, ls1).
struct Chunk {
  int64_t c0[mra::MAXL], c1[mra::MAXL];
  int64_t obs0, obs1, ls0, ls1;
  int64_t f0, nf;        // its leaves by Morton id: [f0, f0 + nf)
  mra::Plan plan;
};
}  // namespace

struct mra_handle {
  mra_config cfg;
  int64_t n = 0;
  int M = 0, r = 0, gx = 0, gy = 0;
  unsigned long long hx = mra::QUAD_HALVINGS, hy = mra::QUAD_HALVINGS;   // per-level halvings of the partition
  // regions of level m in the complete tree: 2^(log2 J_1 + ... + log2 J_m)
  int64_t nfull(int m) const { return int64_t(1) << mra::lvl_depth(hx, hy, m); }
  int nlmax = 0;
  cudaStream_t stream = nullptr;
  Arena tree, state;
  // tree and sorted observations (arena 1)
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
  // factors and tables (arena 2) and the device descriptor
  Tables tab;
  mra::LevelState st{};
  mra::LeafState lf{};
  mra::Desc hd{};
  mra::Desc* d_desc = nullptr;
  mra::Plan plan;
  double* pinned = nullptr;    // small pinned readback buffer
  int64_t ls_cap = 0;          // capacity of the ragged leaf-factor store (doubles)
  int64_t obs_cap = 0;         // capacity of the per-observation leaf stores (rows)
  std::vector<int64_t> cap;    // storage of every level in regions (levels > s: one chunk's)
  // subtree streaming (cfg.stream_level): level s, its chunks, their plans and
  // descriptors (d_desc holds one per chunk; levels <= s are shared by all)
  int s_lvl = 0;
  std::vector<Chunk> chunks;
  std::vector<mra::Desc> chunk_descs;
  mra::Plan plan_coarse_prior, plan_coarse_post;
  // prediction points (arena 3, grown on demand by mra_predict)
  Arena pred;
  int64_t pred_cap = 0;
  double *p_in = nullptr, *p_xs = nullptr, *p_ys = nullptr, *p_U = nullptr, *p_mean = nullptr, *p_var = nullptr;
  int32_t *p_leaf = nullptr, *p_counts = nullptr, *p_cursor = nullptr, *p_max = nullptr;
  int64_t *p_off = nullptr, *p_sq = nullptr, *p_perm = nullptr;
  // joint prediction and simulation (arena 5, grown on demand)
  Arena joint;
  int64_t joint_np = 0, joint_io = 0;
  double *j_D = nullptr, *j_io = nullptr;      // per-leaf D blocks; staging of host inputs / outputs
  int32_t* j_leaf = nullptr;
  // gradient (arena 4, allocated by the first mra_loglik_grad)
  Arena grad;
  bool have_grad_arena = false;
  int grad_buffers = 1;        // MRA_OPT_GRAD_BUFFERS
  mra::GradState gs{};
  double* d_grad = nullptr;
  // timing
  mra::Timer timer;
  bool timer_events = false;
  double ktime[8] = {0};
  int64_t kcount[8] = {0};
  double stime[MRA_MAX_M + 1][MRA_STAGES] = {};
  int64_t scount[MRA_MAX_M + 1][MRA_STAGES] = {};
  int64_t nevals = 0;
  std::vector<int32_t> leaf_counts;   // observations per leaf (Morton order), for mra_stats
  // emulated form: groups of leaves for the leaf kernel (work item (chunk, first
  // compact leaf), leaf count), per chunk from goff[g]; device copies with room
  // for one group per leaf; lrows = the rows of the kernel's layout (0: none)
  std::vector<int2> gitems;
  std::vector<int> gcnt;
  std::vector<int64_t> goff;
  int2* d_gitems = nullptr;
  int* d_gcnt = nullptr;
  int lrows = 0;
  // emulated form: groups of sibling regions for the prior levels, whole-level
  // lists (pwo[m], pwn[m]) and (streamed) each chunk's levels > s (pco[g][m],
  // pcn[g][m]), all in pitems / pcnt; prcap = the rows of the kernel's layout
  std::vector<int2> pitems;
  std::vector<int> pcnt;
  int64_t pwo[mra::MAXL] = {}, pwn[mra::MAXL] = {};
  std::vector<std::vector<int64_t>> pco, pcn;
  int2* d_pitems = nullptr;
  int* d_pcnt = nullptr;
  int prcap = 0;
  // and of sibling level-(M-1) regions for the leaf chain (one 128-row tile each),
  // whole (cwo, cwn) and per chunk (cco[g], ccn[g]), in citems / ccnt
  std::vector<int2> citems;
  std::vector<int> ccnt;
  int64_t cwo = 0, cwn = 0;
  std::vector<int64_t> cco, ccn;
  int2* d_citems = nullptr;
  int* d_ccnt = nullptr;
  bool have_post = false;
  mra_params last{};
  // batch of datasets
  std::vector<mra_handle*> parts;
  Arena batch;
  std::vector<mra::Desc> h_descs;
  mra::Desc* pinned_descs = nullptr;
  mra::Desc* d_descs = nullptr;
  double* d_roots = nullptr;
  int own_stream = 0;
  bool tuned = false;
  int64_t graph_launches = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
};

namespace {

cudaError_t sync_status(mra_handle* h, int* host_status, double* extra, int nextra, const double* const* srcs) {
  cudaError_t e;
  for (int k = 0; k < nextra; ++k)
    if ((e = cudaMemcpyAsync(h->pinned + 4 + k, srcs[k], sizeof(double), cudaMemcpyDeviceToHost, h->stream))) return e;
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
      const int st = h->timer.stage[k], lv = h->timer.level[k];
      if (st >= 0 && lv >= 0 && lv <= MRA_MAX_M) {
        h->stime[lv][st] += ms;
        h->scount[lv][st] += 1;
      }
    }
  }
  h->timer.count = 0;
}

int status_error(const int* s) {
  if (s[0] == mra::ST_NOT_PD)
    return fail(MRA_ERR_NOT_PD, "matrix not positive definite at level %d, region %d", s[1], s[2]);
  if (s[0] == mra::ST_LIMIT) return fail(MRA_ERR_LIMIT, "leaf %d holds more points than the kernels accept", s[2]);
  if (s[0] == mra::ST_ARG) {
    if (s[1] >= 0)
      return fail(MRA_ERR_ARG, "prediction location in leaf %d lies under a level-%d region without observations "
                  "(the tree was built with prune = 1)", s[2], s[1]);
    return fail(MRA_ERR_ARG, "location %d is outside the bounding box or not finite", s[2]);
  }
  if (s[0] == mra::ST_TIMEOUT)
    return fail(MRA_ERR_CUDA, "a tensor-core wait timed out at level %d, region %d", s[1], s[2]);
  return fail(MRA_ERR_CUDA, "device status %d", s[0]);
}

void single_plan(mra_handle* h) {
  mra::Plan& p = h->plan;
  p = mra::Plan();
  p.maxM = h->M;
  p.tile = mra::tile_for_r(h->r);
  p.r = h->r;
  p.mixed = h->cfg.precision == MRA_PREC_MIXED ? 1 : (h->cfg.precision == MRA_PREC_EMU ? 2 : 0);
  p.nlmax = h->nlmax;
  for (int m = 0; m < h->M; ++m) {
    p.n_lvl[m] = h->tab.nreg[m];
    if (m > 0) p.n_agg[m] = h->tab.nreg[m - 1];
  }
  p.n_leaf = h->tab.nreg[h->M];
  if (h->M > 0) {
    p.n_syrk = h->tab.nreg[h->M - 1];
    p.t_syrk = h->M * (h->M + 1) / 2;
  }
}

cudaError_t upload_desc(mra_handle* h, const mra_params* theta) {
  h->hd.sh.M = h->M;
  h->hd.sh.r = h->r;
  h->hd.sh.gx = h->gx;
  h->hd.sh.gy = h->gy;
  h->hd.sh.hx = h->hx;
  h->hd.sh.hy = h->hy;
  for (int k = 0; k < 4; ++k) h->hd.sh.bbox[k] = h->cfg.bbox[k];
  h->hd.sh.mixed = h->cfg.precision == MRA_PREC_MIXED ? 1 : (h->cfg.precision == MRA_PREC_EMU ? 2 : 0);
  if (theta) {
    h->hd.cv = mra::make_cov(theta->sigma2, theta->range, h->cfg.cov_family, h->cfg.nonstat, theta->nu);
    h->hd.tau2 = theta->tau2;
  }
  h->hd.nlmax = h->nlmax;
  h->hd.lrows = h->lrows;
  h->hd.st = h->st;
  h->hd.lf = h->lf;
  if (!h->s_lvl) return cudaMemcpyAsync(h->d_desc, &h->hd, sizeof(mra::Desc), cudaMemcpyHostToDevice, h->stream);
  // Streamed: one descriptor per chunk.  The arrays of levels > s and the leaf
  // stores hold one chunk at a time; a chunk's descriptor points them at
  // (buffer - first id x stride), so the kernels' indexing by global compact id
  // (or observation offset) lands in the buffer for the ids of that chunk,
  // which are the only ones its work lists name.
  const int M = h->M, s = h->s_lvl;
  const int64_t r = h->r, Mr = (int64_t)M * r, ng = (Mr + 127) / 128;
  auto shift = [](auto* p, int64_t first, int64_t stride) {
    using T = std::remove_pointer_t<decltype(p)>;
    return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) - (uintptr_t)(first * stride * (int64_t)sizeof(T)))
             : p;
  };
  h->chunk_descs.assign(h->chunks.size(), h->hd);
  for (size_t g = 0; g < h->chunks.size(); ++g) {
    const Chunk& c = h->chunks[g];
    mra::Desc& D = h->chunk_descs[g];
    for (int m = s + 1; m < M; ++m) {
      const int64_t i0 = c.c0[m], T = int64_t(m + 1) * (m + 2) / 2;
      D.st.V[m] = shift(D.st.V[m], i0, r * m * r);
      D.st.Li[m] = shift(D.st.Li[m], i0, r * r);
      D.st.Acc[m] = shift(D.st.Acc[m], i0, T * r * r);
      D.st.Om[m] = shift(D.st.Om[m], i0, (m + 1) * r);
      D.st.Lt[m] = shift(D.st.Lt[m], i0, r * r);
      D.st.G[m] = shift(D.st.G[m], i0, r * m * r);
      D.st.gv[m] = shift(D.st.gv[m], i0, r);
      D.st.vexp[m] = shift(D.st.vexp[m], i0, ((m * r + 127) / 128) * r);
      D.st.gcol[m] = shift(D.st.gcol[m], i0, m * r);
      D.st.liexp[m] = shift(D.st.liexp[m], i0, r);
      D.st.L[m] = shift(D.st.L[m], i0, r * r);        // (saved for the gradient)
      D.st.Ltf[m] = shift(D.st.Ltf[m], i0, r * r);
      D.st.licol[m] = shift(D.st.licol[m], i0, r);
      D.st.vcol[m] = shift(D.st.vcol[m], i0, m * r);
    }
    D.lf.VF = shift(D.lf.VF, c.obs0, Mr);
    D.lf.LSf = shift(D.lf.LSf, c.ls0, 1);
    D.lf.dc = shift(D.lf.dc, c.obs0, 2 * Mr);
    if (M - 1 > s) D.lf.vfexp = shift(D.lf.vfexp, c.c0[M - 1], 4 * Mr);
    D.lf.H = shift(D.lf.H, c.obs0, Mr);
    D.lf.z = shift(D.lf.z, c.obs0, 1);
    D.lf.LS = shift(D.lf.LS, c.ls0, 1);
    D.lf.hcol = shift(D.lf.hcol, c.c0[M], Mr);
    D.lf.hrow = shift(D.lf.hrow, c.obs0, ng);
  }
  return cudaMemcpyAsync(h->d_desc, h->chunk_descs.data(), sizeof(mra::Desc) * h->chunk_descs.size(),
                         cudaMemcpyHostToDevice, h->stream);
}

// The launches of one evaluation: the whole plan, or (streamed) the coarse
// prior, every chunk's subtree, then the coarse posterior.
cudaError_t launch_evaluation(mra_handle* h) {
  if (!h->s_lvl) return mra::launch_loglik(h->plan, h->d_desc, h->status, h->stream, &g_launches, &h->timer);
  cudaError_t e;
  if ((e = mra::launch_loglik(h->plan_coarse_prior, h->d_desc, h->status, h->stream, &g_launches, &h->timer)))
    return e;
  for (const Chunk& c : h->chunks)
    if ((e = mra::launch_loglik(c.plan, h->d_desc, h->status, h->stream, &g_launches, &h->timer))) return e;
  return mra::launch_loglik(h->plan_coarse_post, h->d_desc, h->status, h->stream, &g_launches, &h->timer);
}

// Binning into an existing tree arena (used by mra_build and mra_update).
cudaError_t bin(mra_handle* h, const double* dl, const double* dy, int* hs, int64_t* tail, int32_t* mc) {
  const int64_t nl = h->nfull(h->M);
  cudaError_t e;
  if ((e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream))) return e;
  if ((e = mra::launch_bin(dl, h->n, h->bbox, h->M, h->hx, h->hy, h->leaf_id, h->counts, h->cursor, h->off,
                           h->sq_off, h->max_count, h->perm, h->status, h->stream, &g_launches)) ||
      (e = mra::launch_gather(dl, dy, h->perm, h->n, h->xs, h->ys, h->yv, h->stream, &g_launches)))
    return e;
  double got[2];
  const double* srcs[2] = {(const double*)(h->sq_off + nl), (const double*)h->max_count};
  if ((e = sync_status(h, hs, got, 2, srcs))) return e;
  memcpy(tail, &got[0], sizeof(int64_t));
  memcpy(mc, &got[1], sizeof(int32_t));
  return cudaSuccess;
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
  for (mra_handle* p : h->parts) mra_free(p);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->timer_events)
    for (int k = 0; k < 2 * mra::MAX_TIMED; ++k) cudaEventDestroy(h->timer.ev[k]);
  h->tree.release();
  h->state.release();
  h->pred.release();
  h->joint.release();
  h->grad.release();
  h->batch.release();
  if (h->pinned) cudaFreeHost(h->pinned);
  if (h->pinned_descs) cudaFreeHost(h->pinned_descs);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

int mra_set_stream(mra_handle* h, void* stream) {
  if (!h) return fail(MRA_ERR_ARG, "null handle");
  if (!h->parts.empty() && !stream) return fail(MRA_ERR_ARG, "a batch handle needs a non-default stream");
  if (h->own_stream) {
    cudaStreamDestroy(h->stream);
    h->own_stream = 0;
  }
  h->stream = (cudaStream_t)stream;
  if (h->gexec) {   // the captured graph belongs to the old stream's work; recapture on next use
    cudaGraphExecDestroy(h->gexec);
    cudaGraphDestroy(h->graph);
    h->gexec = nullptr;
    h->graph = nullptr;
  }
  return MRA_OK;
}

int mra_set_option(mra_handle* h, int option, int64_t value) {
  g_err.clear();
  if (!h) return fail(MRA_ERR_ARG, "null handle");
  if (option == MRA_OPT_GRAD_BUFFERS) {
    if (value != 0 && value != 1) return fail(MRA_ERR_ARG, "MRA_OPT_GRAD_BUFFERS takes 0 or 1");
    if (h->grad_buffers != (int)value && h->have_grad_arena) {   // re-planned by the next gradient call
      h->grad.release();
      h->have_grad_arena = false;
      h->gs = mra::GradState{};
      for (int m = 0; m < mra::MAXL; ++m) {
        h->st.L[m] = h->st.Ltf[m] = nullptr;
        h->st.licol[m] = h->st.vcol[m] = nullptr;
      }
      h->lf.VF = h->lf.LSf = nullptr;
      h->d_grad = nullptr;
      h->have_post = false;
    }
    h->grad_buffers = (int)value;
    for (mra_handle* p : h->parts) p->grad_buffers = (int)value;
    return MRA_OK;
  }
  return fail(MRA_ERR_ARG, "unknown option %d", option);
}

int mra_build(const mra_config* cfg, const double* locs, const double* y, int64_t n, int where,
              mra_handle** out) {
  g_err.clear();
  if (!out) return fail(MRA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!cfg || !locs || !y) return fail(MRA_ERR_ARG, "null argument");
  if (n < 1) return fail(MRA_ERR_ARG, "n must be >= 1 (got %lld)", (long long)n);
  int rc = check_config(cfg);
  if (rc) return rc;
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");

  mra_handle* h = new mra_handle();
  h->cfg = *cfg;
  h->n = n;
  h->M = cfg->M;
  h->r = cfg->r;
  h->gx = gx_for(cfg->r);
  h->gy = cfg->r / h->gx;
  config_halvings(cfg, h->hx, h->hy);
  const int M = h->M, r = h->r;
  const int64_t nl = h->nfull(M);
  cudaError_t e;
  int hs[4];

  // ---- arena 1: inputs, partition, sorted observations -----------------------
  Arena& A = h->tree;
  A.want(&h->bbox, 4);
  A.want(&h->leaf_id, n);
  A.want(&h->counts, nl);
  A.want(&h->cursor, nl);
  A.want(&h->off, nl + 1);
  A.want(&h->sq_off, nl + 1);
  A.want(&h->max_count, 2);
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
  if ((e = cudaMemcpyAsync(h->bbox, cfg->bbox, sizeof(double) * 4, cudaMemcpyHostToDevice, h->stream))) {
    mra_free(h); return cuda_fail(e, "init");
  }
  int64_t tail = 0;
  int32_t mc = 0;
  if ((e = bin(h, dl, dy, hs, &tail, &mc))) { mra_free(h); return cuda_fail(e, "binning"); }
  if (hs[0]) { rc = status_error(hs); mra_free(h); return rc; }
  if (mc > MRA_MAX_LEAF) {
    mra_free(h);
    return fail(MRA_ERR_LIMIT, "a leaf holds %d observations (max %d); increase M", mc, MRA_MAX_LEAF);
  }
  h->nlmax = mc < 1 ? 1 : mc;
  // ---- tree tables (active regions) ------------------------------------------
  {
    std::vector<int32_t> counts(nl);
    if ((e = cudaMemcpyAsync(counts.data(), h->counts, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaStreamSynchronize(h->stream))) {
      mra_free(h); return cuda_fail(e, "leaf counts");
    }
    build_tables(M, h->hx, h->hy, cfg->prune != 0, counts, h->tab);
    h->leaf_counts = counts;
  }
  const std::vector<int32_t>& nreg = h->tab.nreg;
  const bool emu = cfg->precision == MRA_PREC_EMU;
  // ---- subtree streaming: the level s and the chunks (one per level-s region) ----
  int s_lvl = 0;
  if (cfg->stream_level > 0) {
    if (cfg->stream_level >= M) { mra_free(h); return fail(MRA_ERR_ARG, "stream_level must be < M"); }
    s_lvl = cfg->stream_level;
  }
  std::vector<int64_t> obs_pref(nl + 1, 0), ls_pref(nl + 1, 0);   // by leaf Morton id
  for (int64_t f = 0; f < nl; ++f) {
    obs_pref[f + 1] = obs_pref[f] + h->leaf_counts[f];
    ls_pref[f + 1] = ls_pref[f] + (int64_t)h->leaf_counts[f] * h->leaf_counts[f];
  }
  auto make_chunks = [&](int sl, std::vector<Chunk>& out, std::vector<int64_t>& cmax, int64_t& omax, int64_t& lmax) {
    out.assign(nreg[sl], Chunk{});
    cmax.assign(M + 1, 0);
    omax = lmax = 0;
    for (int32_t g = 0; g < nreg[sl]; ++g) {
      Chunk& c = out[g];
      const int64_t ms = h->tab.mort[sl][g];
      for (int m = 0; m <= M; ++m) c.c0[m] = c.c1[m] = 0;
      c.c0[sl] = g;
      c.c1[sl] = g + 1;
      for (int m = sl + 1; m <= M; ++m) {
        const int dm = mra::lvl_depth(h->hx, h->hy, m) - mra::lvl_depth(h->hx, h->hy, sl);
        const int64_t lo = ms << dm, hi = (ms + 1) << dm;
        const auto& mt = h->tab.mort[m];
        c.c0[m] = std::lower_bound(mt.begin(), mt.end(), (int32_t)lo) - mt.begin();
        c.c1[m] = std::lower_bound(mt.begin(), mt.end(), (int32_t)std::min<int64_t>(hi, INT32_MAX)) - mt.begin();
        if (hi > INT32_MAX) c.c1[m] = (int64_t)mt.size();
        cmax[m] = std::max(cmax[m], c.c1[m] - c.c0[m]);
      }
      const int dM = mra::lvl_depth(h->hx, h->hy, M) - mra::lvl_depth(h->hx, h->hy, sl);
      const int64_t f0 = ms << dM, f1 = (ms + 1) << dM;
      c.f0 = f0;
      c.nf = f1 - f0;
      c.obs0 = obs_pref[f0];
      c.obs1 = obs_pref[f1];
      c.ls0 = ls_pref[f0];
      c.ls1 = ls_pref[f1];
      omax = std::max(omax, c.obs1 - c.obs0);
      lmax = std::max(lmax, c.ls1 - c.ls0);
    }
  };
  // bytes of the factors with rc[m] regions' storage at every level and the leaf stores sized (obs, ls, leaves)
  auto factor_bytes = [&](const std::vector<int64_t>& rc, int64_t obs, int64_t ls, int64_t leaves) {
    double b = 0;
    for (int m = 0; m < M; ++m) {
      const double R = (double)rc[m], T = (m + 1) * (m + 2) / 2.0;
      b += 8.0 * R * ((double)r * m * r * 2 + r * r * 2 + T * r * r + (m + 1) * r + r);
      if (emu) b += 4.0 * R * (((m * r + 127) / 128) * r + m * r + r);
    }
    b += 8.0 * ((double)obs * M * r + obs + ls) + (emu ? 4.0 * ((double)leaves * M * r + obs * ((M * r + 127) / 128)) : 0);
    return b;
  };
  std::vector<int64_t> full(M + 1);
  for (int m = 0; m <= M; ++m) full[m] = nreg[m];
  if (cfg->stream_level == 0 && M >= 2) {   // automatic: stream only when the factors of every level do not fit
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      fr = SIZE_MAX;
      cudaGetLastError();
    }
    if (factor_bytes(full, n, tail, nreg[M]) > 0.8 * (double)fr) {
      for (int sl = 1; sl < M && !s_lvl; ++sl) {
        std::vector<Chunk> ch;
        std::vector<int64_t> cm;
        int64_t om, lm;
        make_chunks(sl, ch, cm, om, lm);
        std::vector<int64_t> rc(M + 1);
        for (int m = 0; m <= M; ++m) rc[m] = m <= sl ? nreg[m] : cm[m];
        if (factor_bytes(rc, om, lm, cm[M]) <= 0.5 * (double)fr) s_lvl = sl;
      }
      if (!s_lvl) { mra_free(h); return fail(MRA_ERR_OOM, "the factors do not fit in device memory even streamed"); }
    }
  }
  h->s_lvl = s_lvl;
  std::vector<int64_t> cap(full);      // storage in regions (levels) and leaf stores
  int64_t obs_cap = n, ls_cap = tail;
  if (s_lvl) {
    std::vector<int64_t> cm;
    int64_t om, lm;
    make_chunks(s_lvl, h->chunks, cm, om, lm);
    for (int m = s_lvl + 1; m <= M; ++m) cap[m] = cm[m];
    obs_cap = std::max<int64_t>(om, 1);
    ls_cap = std::max<int64_t>(lm, 1);
  }
  const int ndesc = s_lvl ? nreg[s_lvl] : 1;
  // ---- arena 2: tables, factors of every level and of the leaves -------------
  Arena& B = h->state;
  for (int m = 0; m <= M; ++m) {
    h->st.nreg[m] = nreg[m];
    B.want(&h->st.mort[m], nreg[m]);
    B.want(&h->st.cid[m], (size_t)h->nfull(m));
    if (m > 0) B.want(&h->st.par[m], nreg[m]);
    if (m < M) {
      B.want(&h->st.cfirst[m], nreg[m]);
      B.want(&h->st.ccnt[m], nreg[m]);
    }
  }
  for (int m = 0; m < M; ++m) {
    const int64_t R = cap[m];
    const int64_t T = int64_t(m + 1) * (m + 2) / 2;
    B.want(&h->st.V[m], R * r * (int64_t)m * r);
    B.want(&h->st.Li[m], R * r * r);
    B.want(&h->st.Acc[m], R * T * r * r);
    B.want(&h->st.Om[m], R * (m + 1) * r);
    B.want(&h->st.Lt[m], R * r * r);
    B.want(&h->st.G[m], R * r * (int64_t)m * r);
    B.want(&h->st.gv[m], R * r);
    B.want(&h->st.dd[m], (int64_t)nreg[m]);     // region terms of every level stay whole
    B.want(&h->st.uu[m], (int64_t)nreg[m]);
    if (emu) {
      if (m > 0) B.want(&h->st.vexp[m], R * ((int64_t)(m * r + 127) / 128) * r);
      if (m > 0) B.want(&h->st.gcol[m], R * (int64_t)m * r);
      B.want(&h->st.liexp[m], R * r);
    }
  }
  double *H, *z, *LS, *d, *u;
  B.want(&H, obs_cap * (int64_t)M * r);
  B.want(&z, obs_cap);
  B.want(&LS, (size_t)ls_cap);
  B.want(&d, nreg[M]);
  B.want(&u, nreg[M]);
  int32_t *hcol = nullptr, *hrow = nullptr;
  if (emu) {
    B.want(&hcol, cap[M] * (int64_t)M * r);
    B.want(&hrow, obs_cap * (int64_t)((M * r + 127) / 128));
  }
  B.want(&h->d_desc, ndesc);
  if (emu && M > 0) {   // groups of leaves (the emulated leaf kernel), with room for one per leaf
    h->gitems.clear();
    h->gcnt.clear();
    h->goff.assign(1, 0);
    if (!s_lvl) {
      leaf_groups(h->tab, M, h->leaf_counts, 0, nreg[M - 1], 0, h->gitems, h->gcnt);
      h->goff.push_back((int64_t)h->gitems.size());
    } else {
      for (size_t g = 0; g < h->chunks.size(); ++g) {
        leaf_groups(h->tab, M, h->leaf_counts, h->chunks[g].c0[M - 1], h->chunks[g].c1[M - 1], (int)g, h->gitems,
                    h->gcnt);
        h->goff.push_back((int64_t)h->gitems.size());
      }
    }
    B.want(&h->d_gitems, std::max<int64_t>(nreg[M], 1));
    B.want(&h->d_gcnt, std::max<int64_t>(nreg[M], 1));
    h->lrows = MRA_MAX_LEAF;
    // and groups of sibling regions for the prior levels, stacked up to 128 rows
    const int gmax = std::min(mra::LGRP_MAX, 128 / r);
    if (gmax > 1) {
      h->pitems.clear();
      h->pcnt.clear();
      for (int m = 1; m < M; ++m) {
        h->pwo[m] = (int64_t)h->pitems.size();
        prior_groups(h->tab, m, gmax, 0, nreg[m - 1], 0, h->pitems, h->pcnt);
        h->pwn[m] = (int64_t)h->pitems.size() - h->pwo[m];
      }
      if (s_lvl) {
        h->pco.assign(h->chunks.size(), std::vector<int64_t>(M + 1, 0));
        h->pcn.assign(h->chunks.size(), std::vector<int64_t>(M + 1, 0));
        for (size_t g = 0; g < h->chunks.size(); ++g)
          for (int m = s_lvl + 1; m < M; ++m) {
            h->pco[g][m] = (int64_t)h->pitems.size();
            prior_groups(h->tab, m, gmax, h->chunks[g].c0[m - 1], h->chunks[g].c1[m - 1], (int)g, h->pitems, h->pcnt);
            h->pcn[g][m] = (int64_t)h->pitems.size() - h->pco[g][m];
          }
      }
      B.want(&h->d_pitems, std::max<size_t>(h->pitems.size(), 1));
      B.want(&h->d_pcnt, std::max<size_t>(h->pcnt.size(), 1));
      h->prcap = gmax * r;
    }
    // and groups of sibling level-(M-1) regions for the leaf chain
    h->citems.clear();
    h->ccnt.clear();
    if (M >= 2) {
      h->cwo = 0;
      chain_groups(h->tab, M, obs_pref, 0, nreg[M - 2], 0, h->citems, h->ccnt);
      h->cwn = (int64_t)h->citems.size();
      if (s_lvl) {
        h->cco.assign(h->chunks.size(), 0);
        h->ccn.assign(h->chunks.size(), 0);
        for (size_t g = 0; g < h->chunks.size(); ++g) {
          h->cco[g] = (int64_t)h->citems.size();
          if (M - 1 > s_lvl) {
            chain_groups(h->tab, M, obs_pref, h->chunks[g].c0[M - 2], h->chunks[g].c1[M - 2], (int)g, h->citems,
                         h->ccnt);
          } else {   // (the chunk is one level-(M-1) region)
            h->citems.push_back(make_int2((int)g, (int)h->chunks[g].c0[M - 1]));
            h->ccnt.push_back(1);
          }
          h->ccn[g] = (int64_t)h->citems.size() - h->cco[g];
        }
      }
      // (room for one group per region: mra_update regroups for the new occupancy)
      B.want(&h->d_citems, std::max<size_t>(h->citems.size(), (size_t)nreg[M - 1]));
      B.want(&h->d_ccnt, std::max<size_t>(h->ccnt.size(), (size_t)nreg[M - 1]));
    }
  }
  int2* d_work = nullptr;
  std::vector<int2> work;
  if (s_lvl) {   // work lists of every chunk: (chunk, compact region) per level, leaves, Gram products
    for (size_t g = 0; g < h->chunks.size(); ++g) {
      Chunk& c = h->chunks[g];
      for (int m = s_lvl; m <= M; ++m)   // (level s: the chunk's own region, the parent of its aggregation)
        for (int64_t i = c.c0[m]; i < c.c1[m]; ++i) work.push_back(make_int2((int)g, (int)i));
    }
    B.want(&d_work, std::max<size_t>(work.size(), 1));
  }
  h->ls_cap = ls_cap;
  h->obs_cap = obs_cap;
  h->cap = cap;
  if ((e = B.commit())) { mra_free(h); return fail(MRA_ERR_OOM, "device allocation (factors): %s", cudaGetErrorString(e)); }
  for (int m = 0; m <= M; ++m) {
    if ((e = cudaMemcpyAsync(h->st.mort[m], h->tab.mort[m].data(), sizeof(int32_t) * nreg[m], cudaMemcpyHostToDevice, h->stream)) ||
        (e = cudaMemcpyAsync(h->st.cid[m], h->tab.cid[m].data(), sizeof(int32_t) * h->tab.cid[m].size(), cudaMemcpyHostToDevice, h->stream)) ||
        (m > 0 && (e = cudaMemcpyAsync(h->st.par[m], h->tab.par[m].data(), sizeof(int32_t) * nreg[m], cudaMemcpyHostToDevice, h->stream))) ||
        (m < M && (e = cudaMemcpyAsync(h->st.cfirst[m], h->tab.cfirst[m].data(), sizeof(int32_t) * nreg[m], cudaMemcpyHostToDevice, h->stream))) ||
        (m < M && (e = cudaMemcpyAsync(h->st.ccnt[m], h->tab.ccnt[m].data(), sizeof(int32_t) * nreg[m], cudaMemcpyHostToDevice, h->stream)))) {
      mra_free(h); return cuda_fail(e, "tree tables");
    }
  }
  if (!work.empty() &&
      (e = cudaMemcpyAsync(d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, h->stream))) {
    mra_free(h); return cuda_fail(e, "chunk work lists");
  }
  if (!h->citems.empty() &&
      ((e = cudaMemcpyAsync(h->d_citems, h->citems.data(), sizeof(int2) * h->citems.size(), cudaMemcpyHostToDevice,
                            h->stream)) ||
       (e = cudaMemcpyAsync(h->d_ccnt, h->ccnt.data(), sizeof(int) * h->ccnt.size(), cudaMemcpyHostToDevice,
                            h->stream)))) {
    mra_free(h); return cuda_fail(e, "chain groups");
  }
  if (!h->pitems.empty() &&
      ((e = cudaMemcpyAsync(h->d_pitems, h->pitems.data(), sizeof(int2) * h->pitems.size(), cudaMemcpyHostToDevice,
                            h->stream)) ||
       (e = cudaMemcpyAsync(h->d_pcnt, h->pcnt.data(), sizeof(int) * h->pcnt.size(), cudaMemcpyHostToDevice,
                            h->stream)))) {
    mra_free(h); return cuda_fail(e, "prior groups");
  }
  if (!h->gitems.empty() &&
      ((e = cudaMemcpyAsync(h->d_gitems, h->gitems.data(), sizeof(int2) * h->gitems.size(), cudaMemcpyHostToDevice,
                            h->stream)) ||
       (e = cudaMemcpyAsync(h->d_gcnt, h->gcnt.data(), sizeof(int) * h->gcnt.size(), cudaMemcpyHostToDevice,
                            h->stream)))) {
    mra_free(h); return cuda_fail(e, "leaf groups");
  }
  if ((e = cudaStreamSynchronize(h->stream))) { mra_free(h); return cuda_fail(e, "tree tables"); }
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
  h->lf.hcol = hcol;
  h->lf.hrow = hrow;
  if (s_lvl) {   // per-chunk plans over the work lists, and the two coarse plans
    size_t w = 0;
    for (size_t g = 0; g < h->chunks.size(); ++g) {
      Chunk& c = h->chunks[g];
      mra::Plan& p = c.plan;
      p = mra::Plan();
      p.maxM = M;
      p.tile = mra::tile_for_r(r);
      p.r = r;
      p.mixed = cfg->precision == MRA_PREC_MIXED ? 1 : (emu ? 2 : 0);
      p.nlmax = h->nlmax;
      p.prior_lo = p.post_lo = s_lvl + 1;
      const int2* at[mra::MAXL + 1];
      for (int m = s_lvl; m <= M; ++m) {
        at[m] = d_work + w;
        w += c.c1[m] - c.c0[m];
      }
      for (int m = s_lvl + 1; m < M; ++m) {
        p.n_lvl[m] = (int)(c.c1[m] - c.c0[m]);
        p.w_lvl[m] = at[m];
        p.n_agg[m] = (int)(c.c1[m - 1] - c.c0[m - 1]);
        p.w_agg[m] = at[m - 1];
      }
      p.n_leaf = (int)(c.c1[M] - c.c0[M]);
      p.w_leaf = at[M];
      if (h->lrows) {   // the chunk's groups of leaves
        p.w_leaf = h->d_gitems + h->goff[g];
        p.c_leaf = h->d_gcnt + h->goff[g];
        p.n_leaf = (int)(h->goff[g + 1] - h->goff[g]);
        p.lrows = h->lrows;
      }
      if (!h->citems.empty() && h->ccn[g] < c.c1[M - 1] - c.c0[M - 1]) {   // the chunk's groups for the leaf chain
        p.w_chn = h->d_citems + h->cco[g];
        p.c_chn = h->d_ccnt + h->cco[g];
        p.n_chn = (int)h->ccn[g];
      }
      if (h->prcap) {   // the chunk's groups of sibling regions
        for (int m = s_lvl + 1; m < M; ++m) {
          p.w_pri[m] = h->d_pitems + h->pco[g][m];
          p.c_pri[m] = h->d_pcnt + h->pco[g][m];
          p.n_pri[m] = (int)h->pcn[g][m];
        }
        p.rcap = h->prcap;
      }
      p.n_syrk = (int)(c.c1[M - 1] - c.c0[M - 1]);
      p.w_syrk = at[M - 1];
      p.t_syrk = M * (M + 1) / 2;
    }
  }
  single_plan(h);
  if (h->prcap) {   // whole-level groups of sibling regions (also the coarse levels of a streamed handle)
    for (int m = 1; m < M; ++m) {
      h->plan.w_pri[m] = h->d_pitems + h->pwo[m];
      h->plan.c_pri[m] = h->d_pcnt + h->pwo[m];
      h->plan.n_pri[m] = (int)h->pwn[m];
    }
    h->plan.rcap = h->prcap;
  }
  if (!h->citems.empty() && !s_lvl && h->cwn < nreg[M - 1]) {   // (only if some group holds two or more)
    h->plan.w_chn = h->d_citems + h->cwo;
    h->plan.c_chn = h->d_ccnt + h->cwo;
    h->plan.n_chn = (int)h->cwn;
  }
  if (h->lrows && !s_lvl) {
    h->plan.w_leaf = h->d_gitems;
    h->plan.c_leaf = h->d_gcnt;
    h->plan.n_leaf = (int)h->gitems.size();
    h->plan.lrows = h->lrows;
  }
  if (s_lvl) {
    h->plan_coarse_prior = h->plan;        // levels 0..s of the prior pass
    h->plan_coarse_prior.prior_hi = s_lvl + 1;
    h->plan_coarse_prior.leaves = false;
    h->plan_coarse_prior.post_hi = 0;
    h->plan_coarse_post = h->plan;         // levels s..0 of the posterior pass
    h->plan_coarse_post.prior_hi = 0;
    h->plan_coarse_post.leaves = false;
    h->plan_coarse_post.post_hi = s_lvl + 1;
  }
  size_t need = cfg->precision != MRA_PREC_FP64
                    ? mra::leaf_tc_smem_bytes(std::max(h->nlmax, h->lrows), cfg->precision == MRA_PREC_EMU)
                    : mra::leaf_smem_bytes(r, h->nlmax);
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
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
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
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "use mra_loglik_batch on a batch handle");
  if (!params_ok(theta) || !nu_ok(h->cfg.cov_family, theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0 (and 0.05 <= nu <= 20 for MRA_COV_MATERN), all finite");
  h->have_post = false;
  cudaError_t e;
  if ((e = upload_desc(h, theta)) || (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream)))
    return cuda_fail(e, "descriptor");
  if ((e = launch_evaluation(h))) return cuda_fail(e, "loglik launch");
  int hs[4];
  double du[2];
  const double* srcs[2];
  if (h->M > 0) { srcs[0] = h->st.dd[0]; srcs[1] = h->st.uu[0]; }
  else { srcs[0] = h->lf.d; srcs[1] = h->lf.u; }
  if ((e = sync_status(h, hs, du, 2, srcs))) return cuda_fail(e, "loglik");
  if (h->timer.on) ++h->nevals;
  collect_times(h);
  if (hs[0]) return status_error(hs);
  *loglik_out = -0.5 * (du[0] + du[1]) - 0.5 * (double)h->n * std::log(2.0 * M_PI);
  h->have_post = true;
  h->last = *theta;
  return MRA_OK;
}

// ---------------------------------------------------------------------------
// Two-phase evaluation over level-s subtrees (multi-GPU sharding)
// ---------------------------------------------------------------------------
// Summary of a level-s region R after its subtree: A-hat_R (T_s packed r x r
// blocks), omega-hat_R ((s + 1) r) and the (d, u) of each of its J_{s+1}
// possible children (8 doubles for the quadtree).
static int64_t summary_len(const mra_handle* h) {
  const int64_t s = h->s_lvl, r = h->r;
  return (s + 1) * (s + 2) / 2 * r * r + (s + 1) * r + 2 * (int64_t(1) << h->tab.bits[s + 1]);
}

int mra_summary_len(mra_handle* h, int64_t* len_out, int64_t* nsub_out) {
  g_err.clear();
  if (!h || !len_out || !nsub_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->s_lvl) return fail(MRA_ERR_STATE, "not a streamed handle (stream_level >= 1)");
  *len_out = summary_len(h);
  *nsub_out = (int64_t)h->chunks.size();
  return MRA_OK;
}

int mra_loglik_subtrees(mra_handle* h, const mra_params* theta, int64_t first, int64_t count, double* out) {
  g_err.clear();
  if (!h || !theta || (count > 0 && !out)) return fail(MRA_ERR_ARG, "null argument");
  if (!h->s_lvl) return fail(MRA_ERR_STATE, "not a streamed handle (stream_level >= 1)");
  if (!params_ok(theta) || !nu_ok(h->cfg.cov_family, theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0 (and 0.05 <= nu <= 20 for MRA_COV_MATERN), all finite");
  const int64_t nsub = (int64_t)h->chunks.size();
  if (first < 0 || count < 0 || first + count > nsub)
    return fail(MRA_ERR_ARG, "subtrees [%lld, %lld) outside [0, %lld)", (long long)first, (long long)(first + count),
                (long long)nsub);
  h->have_post = false;
  cudaError_t e;
  if ((e = upload_desc(h, theta)) || (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream)))
    return cuda_fail(e, "descriptor");
  if ((e = mra::launch_loglik(h->plan_coarse_prior, h->d_desc, h->status, h->stream, &g_launches, &h->timer)))
    return cuda_fail(e, "coarse prior");
  for (int64_t g = first; g < first + count; ++g)
    if ((e = mra::launch_loglik(h->chunks[g].plan, h->d_desc, h->status, h->stream, &g_launches, &h->timer)))
      return cuda_fail(e, "subtree");
  int hs[4];
  if ((e = sync_status(h, hs, nullptr, 0, nullptr))) return cuda_fail(e, "subtrees");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  if (count == 0) return MRA_OK;
  const int s = h->s_lvl, M = h->M;
  const int64_t r = h->r, T = int64_t(s + 1) * (s + 2) / 2, L = summary_len(h);
  std::vector<double> A(count * T * r * r), Om(count * (s + 1) * r);
  const int32_t c_lo = h->tab.cfirst[s][first];
  const int32_t c_hi = h->tab.cfirst[s][first + count - 1] + h->tab.ccnt[s][first + count - 1];
  std::vector<double> dk(std::max(c_hi - c_lo, 1)), uk(dk.size());
  const double* dsrc = s + 1 == M ? h->lf.d : h->st.dd[s + 1];
  const double* usrc = s + 1 == M ? h->lf.u : h->st.uu[s + 1];
  if ((e = cudaMemcpyAsync(A.data(), h->st.Acc[s] + first * T * r * r, sizeof(double) * A.size(),
                           cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(Om.data(), h->st.Om[s] + first * (s + 1) * r, sizeof(double) * Om.size(),
                           cudaMemcpyDeviceToHost, h->stream)) ||
      (c_hi > c_lo && (e = cudaMemcpyAsync(dk.data(), dsrc + c_lo, sizeof(double) * (c_hi - c_lo),
                                           cudaMemcpyDeviceToHost, h->stream))) ||
      (c_hi > c_lo && (e = cudaMemcpyAsync(uk.data(), usrc + c_lo, sizeof(double) * (c_hi - c_lo),
                                           cudaMemcpyDeviceToHost, h->stream))) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "summaries");
  for (int64_t k = 0; k < count; ++k) {
    double* o = out + k * L;
    memcpy(o, A.data() + k * T * r * r, sizeof(double) * T * r * r);
    memcpy(o + T * r * r, Om.data() + k * (s + 1) * r, sizeof(double) * (s + 1) * r);
    double* du = o + T * r * r + (s + 1) * r;
    for (int j = 0; j < 2 << h->tab.bits[s + 1]; ++j) du[j] = 0.0;
    const int32_t cf = h->tab.cfirst[s][first + k], cc = h->tab.ccnt[s][first + k];
    for (int32_t j = 0; j < cc; ++j) {
      du[2 * j] = dk[cf + j - c_lo];
      du[2 * j + 1] = uk[cf + j - c_lo];
    }
  }
  return MRA_OK;
}

int mra_loglik_combine(mra_handle* h, const mra_params* theta, const double* summaries, double* loglik_out) {
  g_err.clear();
  if (!h || !theta || !summaries || !loglik_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->s_lvl) return fail(MRA_ERR_STATE, "not a streamed handle (stream_level >= 1)");
  if (!params_ok(theta) || !nu_ok(h->cfg.cov_family, theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0 (and 0.05 <= nu <= 20 for MRA_COV_MATERN), all finite");
  const int s = h->s_lvl, M = h->M;
  const int64_t nsub = (int64_t)h->chunks.size(), r = h->r, T = int64_t(s + 1) * (s + 2) / 2, L = summary_len(h);
  std::vector<double> A(nsub * T * r * r), Om(nsub * (s + 1) * r);
  const int64_t nkids = h->tab.nreg[s + 1];
  std::vector<double> dk(std::max<int64_t>(nkids, 1), 0.0), uk(dk.size(), 0.0);
  for (int64_t k = 0; k < nsub; ++k) {
    const double* o = summaries + k * L;
    memcpy(A.data() + k * T * r * r, o, sizeof(double) * T * r * r);
    memcpy(Om.data() + k * (s + 1) * r, o + T * r * r, sizeof(double) * (s + 1) * r);
    const double* du = o + T * r * r + (s + 1) * r;
    const int32_t cf = h->tab.cfirst[s][k], cc = h->tab.ccnt[s][k];
    for (int32_t j = 0; j < cc; ++j) {
      dk[cf + j] = du[2 * j];
      uk[cf + j] = du[2 * j + 1];
    }
  }
  h->have_post = false;
  cudaError_t e;
  double* ddst = s + 1 == M ? h->lf.d : h->st.dd[s + 1];
  double* udst = s + 1 == M ? h->lf.u : h->st.uu[s + 1];
  if ((e = upload_desc(h, theta)) || (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream)) ||
      (e = cudaMemcpyAsync(h->st.Acc[s], A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(h->st.Om[s], Om.data(), sizeof(double) * Om.size(), cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(ddst, dk.data(), sizeof(double) * nkids, cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemcpyAsync(udst, uk.data(), sizeof(double) * nkids, cudaMemcpyHostToDevice, h->stream)))
    return cuda_fail(e, "summaries");
  if ((e = mra::launch_loglik(h->plan_coarse_post, h->d_desc, h->status, h->stream, &g_launches, &h->timer)))
    return cuda_fail(e, "coarse posterior");
  int hs[4];
  double du[2];
  const double* srcs[2] = {h->st.dd[0], h->st.uu[0]};
  if ((e = sync_status(h, hs, du, 2, srcs))) return cuda_fail(e, "combine");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  *loglik_out = -0.5 * (du[0] + du[1]) - 0.5 * (double)h->n * std::log(2.0 * M_PI);
  h->have_post = true;    // (region terms of levels <= s are now the whole problem's)
  h->last = *theta;
  return MRA_OK;
}

int mra_region_terms(mra_handle* h, int level, double* d_out, double* u_out) {
  g_err.clear();
  if (!h || !d_out || !u_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  if (level < 0 || level > h->M) return fail(MRA_ERR_ARG, "level must be in [0, M]");
  if (!h->have_post) return fail(MRA_ERR_STATE, "no log-likelihood evaluated yet");
  const int64_t full = h->nfull(level);
  const int32_t cnt = h->tab.nreg[level];
  const double* d = level == h->M ? h->lf.d : h->st.dd[level];
  const double* u = level == h->M ? h->lf.u : h->st.uu[level];
  std::vector<double> dv(cnt), uv(cnt);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dv.data(), d, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(uv.data(), u, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "region terms");
  for (int64_t k = 0; k < full; ++k) d_out[k] = u_out[k] = 0.0;     // inactive regions contribute 0 (R10)
  for (int32_t c = 0; c < cnt; ++c) {
    d_out[h->tab.mort[level][c]] = dv[c];
    u_out[h->tab.mort[level][c]] = uv[c];
  }
  return MRA_OK;
}

int mra_leaf_offsets(mra_handle* h, int64_t* off_out, int64_t* perm_out) {
  g_err.clear();
  if (!h || !off_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  const int64_t nl = h->nfull(h->M);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(off_out, h->off, sizeof(int64_t) * (nl + 1), cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "offsets");
  if (perm_out && (e = cudaMemcpyAsync(perm_out, h->perm, sizeof(int64_t) * h->n, cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "perm");
  if ((e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "offsets");
  return MRA_OK;
}

int mra_update(mra_handle* h, const double* locs, const double* y, int where) {
  g_err.clear();
  if (!h || !locs || !y) return fail(MRA_ERR_ARG, "null argument");
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  if (h->s_lvl) return fail(MRA_ERR_STATE, "a streamed handle keeps its partition: build a new handle");
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");
  const int64_t n = h->n, nl = h->nfull(h->M);
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
  int hs[4];
  int64_t tail = 0;
  int32_t mc = 0;
  if ((e = bin(h, dl, dy, hs, &tail, &mc))) return cuda_fail(e, "binning");
  if (hs[0]) return status_error(hs);
  if (mc > h->nlmax || tail > h->ls_cap)
    return fail(MRA_ERR_LIMIT, "new partition needs leaves of %d (handle has %d) or %lld leaf-factor doubles "
                "(handle has %lld); build a new handle", mc, h->nlmax, (long long)tail, (long long)h->ls_cap);
  std::vector<int32_t> counts(nl);
  if ((e = cudaMemcpyAsync(counts.data(), h->counts, sizeof(int32_t) * nl, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "leaf counts");
  if (h->cfg.prune)   // the active regions must not change
    for (int64_t f = 0; f < nl; ++f)
      if ((counts[f] > 0) != (h->tab.cid[h->M][f] >= 0))
        return fail(MRA_ERR_LIMIT, "the new data occupies other leaves than the pruned tree; build a new handle");
  h->leaf_counts.swap(counts);
  if (h->lrows) {   // the groups of leaves follow the new occupancy
    h->gitems.clear();
    h->gcnt.clear();
    leaf_groups(h->tab, h->M, h->leaf_counts, 0, h->tab.nreg[h->M - 1], 0, h->gitems, h->gcnt);
    h->goff.assign({0, (int64_t)h->gitems.size()});
    if ((e = cudaMemcpyAsync(h->d_gitems, h->gitems.data(), sizeof(int2) * h->gitems.size(), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaMemcpyAsync(h->d_gcnt, h->gcnt.data(), sizeof(int) * h->gcnt.size(), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
      return cuda_fail(e, "leaf groups");
    h->plan.n_leaf = (int)h->gitems.size();
  }
  if (!h->citems.empty()) {   // and the leaf chain's groups
    std::vector<int64_t> obs_pref(h->leaf_counts.size() + 1, 0);
    for (size_t f = 0; f < h->leaf_counts.size(); ++f) obs_pref[f + 1] = obs_pref[f] + h->leaf_counts[f];
    h->citems.clear();
    h->ccnt.clear();
    chain_groups(h->tab, h->M, obs_pref, 0, h->tab.nreg[h->M - 2], 0, h->citems, h->ccnt);
    h->cwo = 0;
    h->cwn = (int64_t)h->citems.size();
    if ((e = cudaMemcpyAsync(h->d_citems, h->citems.data(), sizeof(int2) * h->citems.size(), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaMemcpyAsync(h->d_ccnt, h->ccnt.data(), sizeof(int) * h->ccnt.size(), cudaMemcpyHostToDevice,
                             h->stream)) ||
        (e = cudaStreamSynchronize(h->stream)))
      return cuda_fail(e, "chain groups");
    if (h->cwn < h->tab.nreg[h->M - 1]) {   // (only if some group holds two or more)
      h->plan.w_chn = h->d_citems + h->cwo;
      h->plan.c_chn = h->d_ccnt + h->cwo;
      h->plan.n_chn = (int)h->cwn;
    } else {
      h->plan.w_chn = nullptr;
      h->plan.c_chn = nullptr;
      h->plan.n_chn = 0;
    }
  }
  return MRA_OK;
}

// ---------------------------------------------------------------------------
// Gradient
// ---------------------------------------------------------------------------
static int ensure_grad_arena(mra_handle* h) {
  if (h->have_grad_arena) return MRA_OK;
  const int M = h->M, r = h->r;
  const int64_t n = h->n;
  const std::vector<int32_t>& nreg = h->tab.nreg;
  Arena& G = h->grad;
  // Streamed handles (stream level s): the levels > s and the leaf stores hold
  // one chunk at a time, as the forward factors do; the ancestor adjoints that
  // level s+1 passes up and the leaves' partials of a level-s parent are read
  // by the coarse adjoint after every chunk, so they stay whole.
  const int s = h->s_lvl;
  auto rcap = [&](int m) -> int64_t { return s && m > s ? h->cap[m] : (int64_t)nreg[m]; };
  const int64_t nobs = s ? h->obs_cap : n;
  for (int m = 0; m < M; ++m) {
    const int64_t R = rcap(m);
    G.want(&h->st.L[m], R * r * r);
    G.want(&h->st.Ltf[m], R * r * r);
    G.want(&h->gs.Abar[m], R * r * (int64_t)(m + 1) * r);
    G.want(&h->gs.Obar[m], R * r);
    G.want(&h->gs.GB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.VB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.XB[m], R * r * (int64_t)m * r);
    G.want(&h->gs.Up[m], (m == s + 1 ? (int64_t)nreg[m] : R) * (int64_t)m * (m + 1) / 2 * r * r);
    h->st.licol[m] = h->st.vcol[m] = nullptr;
    if (h->cfg.precision == MRA_PREC_EMU) {
      G.want(&h->st.licol[m], R * r);
      if (m > 0) G.want(&h->st.vcol[m], R * (int64_t)m * r);
    }
  }
  if (M > 0) G.want(&h->gs.PartLeaf, rcap(M - 1) * M * (M + 1) / 2 * r * r);
  h->gs.SF = nullptr;
  h->gs.SFexp = nullptr;
  h->gs.DC = nullptr;
  h->gs.VFexp = h->gs.VBexp = h->gs.XBexp = nullptr;
  G.want(&h->lf.VF, nobs * (int64_t)M * r);
  G.want(&h->lf.LSf, (size_t)h->ls_cap);
  G.want(&h->gs.HB, nobs * (int64_t)M * r);
  if (h->cfg.precision == MRA_PREC_EMU && M > 0) {
    G.want(&h->gs.VFexp, rcap(M - 1) * 4 * M * r);
    G.want(&h->gs.VBexp, rcap(M - 1) * 4 * M * r);
    G.want(&h->gs.XBexp, rcap(M - 1) * 4 * M * r);
  }
  G.want(&h->gs.VBF, nobs * (int64_t)M * r);
  G.want(&h->gs.XBF, nobs * (int64_t)M * r);
  G.want(&h->gs.T, 3 * (size_t)h->ls_cap);
  int64_t slots = 0;
  for (int m = 0; m <= M; ++m) slots += nreg[m];
  if (M > 0) slots += nreg[M - 1];   // the emulated chain adjoint's, one per level-(M-1) region
  G.want(&h->gs.gpart, mra::GP * slots);
  // Emulated form, two optional buffers, each taken only while 85 % of the free
  // device memory holds it after everything above (the kernels have paths
  // without them): the per-parent adjoint S for Hbar and Gbar on the tensor
  // cores (else the FP64 kernels form Hbar and Gbar from the ancestors'
  // blocks; slower even where S is many times the size of H, as on sparse
  // leaves), then the chain's covariance derivative pairs (else the chain
  // adjoint evaluates them).  On a streamed handle both are chunk-sized: S
  // holds the parents of one launch (a chunk's, or a coarse level's), the
  // pairs one chunk's observations.
  if (M > 0 && h->cfg.precision == MRA_PREC_EMU && h->grad_buffers) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      fr = 0;
      cudaGetLastError();   // else the next launch check would report this query's error
    }
    size_t base = 0;
    for (auto& q : G.plan) base += Arena::align(q.second);
    int64_t budget = (int64_t)(0.85 * (double)fr) - (int64_t)base;
    const int64_t Mr = (int64_t)M * r;
    // parents of one S launch at level L (Gbar of level L + 1, Hbar for L = M - 1)
    auto parents = [&](int L) -> int64_t { return !s || L < s ? (int64_t)nreg[L] : (L == s ? 1 : h->cap[L]); };
    int64_t sfd = 0, sfe = 0;
    for (int L = 0; L < M; ++L) {
      const int64_t w = (int64_t)(L + 1) * r;
      sfd = std::max(sfd, parents(L) * w * w);
      sfe = std::max(sfe, parents(L) * ((w + 127) / 128) * w);
    }
    sfe += 8;                                               // + the rows the engine rounds up to 8
    const int64_t sf = (int64_t)Arena::align(8 * sfd) + (int64_t)Arena::align(4 * sfe);
    if (sf <= budget) {
      G.want(&h->gs.SF, sfd);
      G.want(&h->gs.SFexp, sfe);
      budget -= sf;
    }
    if ((int64_t)Arena::align(16 * nobs * Mr) <= budget && h->cfg.cov_family != MRA_COV_MATERN)
      G.want(&h->gs.DC, 2 * nobs * Mr);   // (pairs d/dsigma2, d/dkappa: the free-smoothness family also needs d/dnu)
  }
  G.want(&h->d_grad, 4);
  cudaError_t e = G.commit();
  if (e) {
    for (int m = 0; m < M; ++m) {
      h->st.L[m] = nullptr;
      h->st.Ltf[m] = nullptr;
      h->st.licol[m] = h->st.vcol[m] = nullptr;
    }
    h->lf.VF = nullptr;
    h->lf.LSf = nullptr;
    h->gs.SF = nullptr;
    h->gs.SFexp = nullptr;
    h->gs.DC = nullptr;
    h->gs.VFexp = h->gs.VBexp = h->gs.XBexp = nullptr;
    return fail(MRA_ERR_OOM, "device allocation (gradient): %s", cudaGetErrorString(e));
  }
  h->have_grad_arena = true;
  return MRA_OK;
}

}  // extern "C"

namespace {

// Adjoint state of one chunk of a streamed handle: the arrays of levels > s
// and the per-observation and ragged leaf stores point at (buffer - first id x
// stride), as the chunk's descriptor does for the forward factors.
template <class T>
T* shifted(T* p, int64_t first, int64_t stride) {
  return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) - (uintptr_t)(first * stride * (int64_t)sizeof(T)))
           : p;
}

mra::GradState chunk_grad_state(const mra_handle* h, const Chunk& c) {
  const int M = h->M, s = h->s_lvl;
  const int64_t r = h->r, Mr = (int64_t)M * r;
  mra::GradState g = h->gs;
  for (int m = s + 1; m < M; ++m) {
    const int64_t i0 = c.c0[m];
    g.Abar[m] = shifted(g.Abar[m], i0, r * (m + 1) * r);
    g.Obar[m] = shifted(g.Obar[m], i0, r);
    g.GB[m] = shifted(g.GB[m], i0, r * m * r);
    g.VB[m] = shifted(g.VB[m], i0, r * m * r);
    g.XB[m] = shifted(g.XB[m], i0, r * m * r);
    if (m > s + 1) g.Up[m] = shifted(g.Up[m], i0, (int64_t)m * (m + 1) / 2 * r * r);
  }
  if (M - 1 > s) {
    const int64_t p0 = c.c0[M - 1];
    g.PartLeaf = shifted(g.PartLeaf, p0, (int64_t)M * (M + 1) / 2 * r * r);
    g.VFexp = shifted(g.VFexp, p0, 4 * Mr);
    g.VBexp = shifted(g.VBexp, p0, 4 * Mr);
    g.XBexp = shifted(g.XBexp, p0, 4 * Mr);
  }
  g.HB = shifted(g.HB, c.obs0, Mr);
  g.VBF = shifted(g.VBF, c.obs0, Mr);
  g.XBF = shifted(g.XBF, c.obs0, Mr);
  g.T = shifted(g.T, c.ls0, 3);
  return g;
}

// Reverse pass of a streamed handle, after its forward evaluation: the
// posterior adjoint of the coarse levels 0..s, then per chunk (last first: the
// last chunk's forward factors are still resident, the others' are recomputed
// from the coarse levels, which stay whole) the posterior adjoint of its levels
// > s, its leaves' adjoints and its prior adjoint up to level s+1, and last the
// prior adjoint of the coarse levels s..0.
cudaError_t streamed_grad(mra_handle* h) {
  const int M = h->M, s = h->s_lvl;
  cudaError_t e;
  mra::GradRange coarse_post;
  coarse_post.post_hi = s + 1;
  coarse_post.leaves = false;
  coarse_post.prior_hi = 0;
  coarse_post.cs_lo = 0;                 // (the column scales of levels <= s serve every chunk)
  coarse_post.cs_hi = s + 1;
  h->timer.start(6, h->stream);
  e = mra::launch_grad_range(h->hd, h->d_desc, h->gs, coarse_post, h->status, h->stream, &g_launches);
  h->timer.stop(h->stream);
  if (e) return e;
  for (size_t k = h->chunks.size(); k-- > 0;) {
    const Chunk& c = h->chunks[k];
    if (k + 1 < h->chunks.size() &&
        (e = mra::launch_loglik(c.plan, h->d_desc, h->status, h->stream, &g_launches, &h->timer)))
      return e;
    mra::GradRange R;
    R.post_lo = R.prior_lo = s + 1;
    R.local_sf = true;
    for (int m = s; m <= M; ++m) {
      R.base[m] = c.c0[m];
      R.count[m] = c.c1[m] - c.c0[m];
    }
    h->timer.start(6, h->stream);
    e = mra::launch_grad_range(h->chunk_descs[k], h->d_desc + k, chunk_grad_state(h, c), R, h->status, h->stream,
                               &g_launches);
    h->timer.stop(h->stream);
    if (e) return e;
  }
  mra::GradRange coarse_prior;
  coarse_prior.post_hi = 0;
  coarse_prior.leaves = false;
  coarse_prior.prior_hi = s + 1;
  coarse_prior.cs_lo = coarse_prior.cs_hi = 0;
  h->timer.start(6, h->stream);
  e = mra::launch_grad_range(h->hd, h->d_desc, h->gs, coarse_prior, h->status, h->stream, &g_launches);
  if (!e) e = mra::launch_grad_reduce(h->hd, h->gs, h->d_grad, h->stream, &g_launches);
  h->timer.stop(h->stream);
  return e;
}

}  // namespace

extern "C" {

int mra_loglik_grad(mra_handle* h, const mra_params* theta, double* loglik_out, double* grad_out) {
  g_err.clear();
  if (!h || !loglik_out || !grad_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  if (!params_ok(theta) || !nu_ok(h->cfg.cov_family, theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0 (and 0.05 <= nu <= 20 for MRA_COV_MATERN), all finite");
  int rc = ensure_grad_arena(h);
  if (rc) return rc;
  h->have_post = false;
  cudaError_t e;
  h->lf.dc = h->gs.DC;                 // the chain kernel stores its C0 derivatives (emulated form)
  h->lf.vfexp = h->gs.VFexp;           // and the column scales of V_F per tile
  e = upload_desc(h, theta);
  h->lf.dc = nullptr;                  // (the descriptor was copied: later loglik calls store nothing)
  h->lf.vfexp = nullptr;
  if (e || (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream)))
    return cuda_fail(e, "descriptor");
  if ((e = launch_evaluation(h))) return cuda_fail(e, "loglik launch");
  if (h->s_lvl) e = streamed_grad(h);
  else e = mra::launch_grad(h->hd, h->d_desc, h->gs, h->d_grad, h->status, h->stream, &g_launches, &h->timer);
  if (e) return cuda_fail(e, "gradient launch");
  int hs[4];
  double vals[6];
  const double* srcs[6];
  if (h->M > 0) { srcs[0] = h->st.dd[0]; srcs[1] = h->st.uu[0]; }
  else { srcs[0] = h->lf.d; srcs[1] = h->lf.u; }
  for (int c = 0; c < 4; ++c) srcs[2 + c] = h->d_grad + c;
  if ((e = sync_status(h, hs, vals, 6, srcs))) return cuda_fail(e, "gradient");
  if (h->timer.on) ++h->nevals;
  collect_times(h);
  if (hs[0]) return status_error(hs);
  *loglik_out = -0.5 * (vals[0] + vals[1]) - 0.5 * (double)h->n * std::log(2.0 * M_PI);
  grad_out[0] = vals[2];
  grad_out[1] = vals[3];
  grad_out[2] = vals[4];
  if (h->cfg.cov_family == MRA_COV_MATERN) grad_out[3] = vals[5];
  h->have_post = true;
  h->last = *theta;
  return MRA_OK;
}

// ---------------------------------------------------------------------------
// Timing
// ---------------------------------------------------------------------------
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
  memset(h->stime, 0, sizeof h->stime);
  memset(h->scount, 0, sizeof h->scount);
  h->nevals = 0;
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

// Algorithmic work of one evaluation per level and stage (mra_stats): FLOPs
// with multiply-add = 2, symmetric and triangular products counted once and
// factorisations (Cholesky with triangular inverse) 2 r^3 / 3; bytes = 8 x the
// doubles each unit reads and writes once.  T_m = (m+1)(m+2)/2 packed blocks.
static void stage_model(const mra_handle* p, double fl[][MRA_STAGES], double by[][MRA_STAGES],
                        double un[][MRA_STAGES]) {
  const int M = p->M;
  const double r = p->r, r2 = r * r, tri = r * (r + 1) / 2.0, Mr = M * r;
  const bool emu = p->cfg.precision == MRA_PREC_EMU;
  const std::vector<int32_t>& nreg = p->tab.nreg;
  for (int m = 0; m < M; ++m) {
    const double R = nreg[m];
    double f = 2.0 * tri * (m * r) + 2.0 * r * r2 / 3.0;
    for (int l = 0; l < m; ++l) f += 2.0 * r2 * (l * r) + 2.0 * r * tri;
    fl[m][MRA_STAGE_PRIOR] += R * f;
    // reads: ancestors' V rows (r x l r, l < m) and L_l^{-1}; writes V (r x m r) and L^{-1}
    by[m][MRA_STAGE_PRIOR] += 8.0 * R * (r2 * m * (m - 1) / 2.0 + m * r2 + m * r2 + r2);
    un[m][MRA_STAGE_PRIOR] += R;
    const double Tm = (m + 1) * (m + 2) / 2.0;
    fl[m][MRA_STAGE_POST] += R * (2.0 * r * r2 / 3.0 + m * r2 * (r + 1) + r * (r + 1));
    // reads A-hat (T_m blocks) and omega-hat; writes Lt^{-1}, G (r x m r), g, d, u
    by[m][MRA_STAGE_POST] += 8.0 * R * (Tm * r2 + (m + 1) * r + r2 + m * r2 + r + 2);
    un[m][MRA_STAGE_POST] += R;
    if (m > 0) {
      const double mr = m * r, Tp = m * (m + 1) / 2.0;
      // per child: A~ = A-hat - G'G over its lower blocks (k, l < m), omega~
      fl[m][MRA_STAGE_AGGREGATE] += R * (mr * (mr + 1) * r + 2.0 * mr * r);
      // per child reads A-hat blocks (k, l < m), G, g, omega-hat; per parent writes A-hat, omega-hat
      by[m][MRA_STAGE_AGGREGATE] += 8.0 * (R * (Tp * r2 + m * r2 + r + m * r) + nreg[m - 1] * (Tp * r2 + m * r));
      un[m][MRA_STAGE_AGGREGATE] += nreg[m - 1];
    }
  }
  double chain_f = 0, leaf_f = 0, leaf_b = 0, nobs = 0, nleaf = 0;
  for (size_t f = 0; f < p->leaf_counts.size(); ++f) {
    const double c = p->leaf_counts[f];
    if (c == 0 && p->cfg.prune) continue;
    nleaf += 1;
    nobs += c;
    double ch = 0;
    for (int l = 0; l < M; ++l) ch += 2.0 * c * r * (l * r) + 2.0 * c * tri;
    chain_f += ch;
    leaf_f += c * (c + 1) * Mr + 2.0 * c * c * c / 3.0 + c * (c + 1) + Mr * c * (c + 1);
    // reads x, y, data; writes H (c x M r), z, L_Sigma^{-1} (c^2), d, u
    leaf_b += 8.0 * (3 * c + c * Mr + c + c * c + 2);
  }
  const double anc = r2 * (M * (M - 1) / 2.0 + M);   // the ancestors' V rows and L^{-1} of a leaf's chain
  const double P = M > 0 ? nreg[M - 1] : 0;
  if (emu && M > 0) {
    fl[M][MRA_STAGE_CHAIN] += chain_f;
    by[M][MRA_STAGE_CHAIN] += 8.0 * (2 * nobs + P * anc + nobs * Mr);
    un[M][MRA_STAGE_CHAIN] += P;
    fl[M][MRA_STAGE_LEAF] += leaf_f;
    by[M][MRA_STAGE_LEAF] += leaf_b + 8.0 * nobs * Mr;           // V_F read back
  } else {
    fl[M][MRA_STAGE_LEAF] += chain_f + leaf_f;
    by[M][MRA_STAGE_LEAF] += leaf_b + 8.0 * nleaf * anc;
  }
  un[M][MRA_STAGE_LEAF] += nleaf;
  if (M > 0) {
    const double T = M * (M + 1) / 2.0;
    fl[M][MRA_STAGE_LEAF_SYRK] += (Mr * (Mr + 1) + 2.0 * Mr) * nobs;
    // reads H and z; writes the parents' A-hat (T blocks) and omega-hat
    by[M][MRA_STAGE_LEAF_SYRK] += 8.0 * (nobs * (Mr + 1) + P * (T * r2 + Mr));
    un[M][MRA_STAGE_LEAF_SYRK] += P;
  }
}

extern "C" int mra_stats(mra_handle* h, mra_stats_t* out) {
  g_err.clear();
  if (!h || !out) return fail(MRA_ERR_ARG, "null argument");
  memset(out, 0, sizeof *out);
  out->M = h->M;
  out->evaluations = h->nevals;
  for (int m = 0; m <= MRA_MAX_M; ++m)
    for (int k = 0; k < MRA_STAGES; ++k) {
      out->ms[m][k] = h->stime[m][k];
      out->launches[m][k] = h->scount[m][k];
    }
  if (h->parts.empty()) {
    stage_model(h, out->flops, out->bytes, out->units);
  } else {
    for (mra_handle* p : h->parts) stage_model(p, out->flops, out->bytes, out->units);
  }
  return MRA_OK;
}

// ---------------------------------------------------------------------------
// Prediction
// ---------------------------------------------------------------------------
// The steps every prediction entry point shares: the posterior factors at
// theta, the prediction buffers, and the binning of the points by leaf (stable
// for the joint modes, whose per-leaf factors depend on the points' order).
static int pred_prepare(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                        bool stable, int32_t* maxp_out) {
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  if (h->s_lvl && stable)
    return fail(MRA_ERR_STATE, "the joint predictive needs the factors of every level: not on a streamed handle");
  if (np < 1) return fail(MRA_ERR_ARG, "np must be >= 1");
  if (where != MRA_HOST && where != MRA_DEVICE) return fail(MRA_ERR_ARG, "where must be MRA_HOST or MRA_DEVICE");
  if (!params_ok(theta) || !nu_ok(h->cfg.cov_family, theta)) return fail(MRA_ERR_ARG, "theta needs sigma2 > 0, range > 0, tau2 >= 0 (and 0.05 <= nu <= 20 for MRA_COV_MATERN), all finite");
  if (!h->have_post || theta->sigma2 != h->last.sigma2 || theta->range != h->last.range ||
      theta->tau2 != h->last.tau2 || (h->cfg.cov_family == MRA_COV_MATERN && theta->nu != h->last.nu)) {
    // the posterior factors of Sec. 3.2 at this theta: one evaluation first
    double ll;
    const int rc = mra_loglik(h, theta, &ll);
    if (rc) return rc;
  }
  const int M = h->M, r = h->r;
  const int64_t nl = h->nfull(M);
  cudaError_t e;
  if (np > h->pred_cap) {
    h->pred.release();
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
  if ((e = mra::launch_bin(dp, np, h->bbox, M, h->hx, h->hy, h->p_leaf, h->p_counts, h->p_cursor, h->p_off, h->p_sq, h->p_max,
                           h->p_perm, h->status, h->stream, &g_launches, stable)) ||
      (e = mra::launch_gather(dp, nullptr, h->p_perm, np, h->p_xs, h->p_ys, nullptr, h->stream, &g_launches)))
    return cuda_fail(e, "binning prediction points");
  int hs[4];
  double got[1];
  const double* srcs[1] = {(const double*)h->p_max};
  if ((e = sync_status(h, hs, got, 1, srcs))) return cuda_fail(e, "binning prediction points");
  if (hs[0]) return status_error(hs);
  memcpy(maxp_out, &got[0], sizeof(int32_t));
  return MRA_OK;
}

static mra::PredState pred_state(mra_handle* h) {
  mra::PredState ps{};
  ps.off = h->p_off;
  ps.perm = h->p_perm;
  ps.xs = h->p_xs;
  ps.ys = h->p_ys;
  ps.U = h->p_U;
  ps.mean = h->p_mean;
  ps.var = h->p_var;
  ps.nleaves = (long)h->nfull(h->M);
  return ps;
}

int mra_predict(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                double* mean_out, double* var_out) {
  g_err.clear();
  if (!h || !theta || !plocs || !mean_out || !var_out) return fail(MRA_ERR_ARG, "null argument");
  int32_t maxp = 0;
  int rc = pred_prepare(h, theta, plocs, np, where, false, &maxp);
  if (rc) return rc;
  const int M = h->M, r = h->r;
  cudaError_t e;
  int hs[4];
  double got[1];
  const double* srcs[1] = {(const double*)h->p_max};
  mra::PredState ps = pred_state(h);
  ps.mean = where == MRA_DEVICE ? mean_out : h->p_mean;
  ps.var = where == MRA_DEVICE ? var_out : h->p_var;
  if (!h->s_lvl) {
    if ((e = mra::launch_predict(h->d_desc, M, r, h->nlmax, ps, maxp, h->status, h->stream, &g_launches, &h->timer)))
      return cuda_fail(e, "predict launch");
  } else {
    // Streamed: the coarse factors (levels <= s) are resident from the
    // evaluation; each chunk's own factors are formed again from them (its
    // prior, leaves and posterior, as in the evaluation, with the same
    // results) and its leaves' points predicted before the next chunk reuses
    // the buffers.
    for (size_t g = 0; g < h->chunks.size(); ++g) {
      const Chunk& c = h->chunks[g];
      ps.desc = (int)g;
      ps.leaf0 = (long)c.f0;
      if ((e = mra::launch_loglik(c.plan, h->d_desc, h->status, h->stream, &g_launches, &h->timer)) ||
          (e = mra::launch_predict(h->d_desc, M, r, h->nlmax, ps, maxp, h->status, h->stream, &g_launches, &h->timer,
                                   (long)c.nf)))
        return cuda_fail(e, "predict launch");
    }
  }
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(mean_out, h->p_mean, sizeof(double) * np, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(var_out, h->p_var, sizeof(double) * np, cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "copy predictions");
  }
  if ((e = sync_status(h, hs, got, 0, srcs))) return cuda_fail(e, "predict");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  return MRA_OK;
}

// Joint modes: D blocks (at most JOINT_TILE points per leaf, so sum n_P^2 <=
// JOINT_TILE np), sorted leaf ids, and `io` doubles of staging for host data.
static int ensure_joint(mra_handle* h, int64_t np, int64_t io) {
  if (np <= h->joint_np && io <= h->joint_io) return MRA_OK;
  h->joint.release();
  h->joint_np = h->joint_io = 0;
  Arena& A = h->joint;
  A.want(&h->j_D, (int64_t)mra::JOINT_TILE * np);
  A.want(&h->j_leaf, np);
  A.want(&h->j_io, io);
  cudaError_t e = A.commit();
  if (e) return fail(MRA_ERR_OOM, "device allocation (joint prediction): %s", cudaGetErrorString(e));
  h->joint_np = np;
  h->joint_io = io;
  return MRA_OK;
}

static int joint_factors(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                         int mode, int64_t io, mra::PredState* ps_out) {
  int32_t maxp = 0;
  int rc = pred_prepare(h, theta, plocs, np, where, true, &maxp);
  if (rc) return rc;
  if (maxp > mra::JOINT_TILE)
    return fail(MRA_ERR_LIMIT, "a leaf holds %d prediction points; the joint predictive takes at most %d per "
                "leaf", maxp, mra::JOINT_TILE);
  if ((rc = ensure_joint(h, np, io))) return rc;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < mra::joint_smem_bytes(h->r, h->nlmax))
    return fail(MRA_ERR_LIMIT, "joint prediction needs more shared memory than the device allows");
  mra::PredState ps = pred_state(h);
  ps.sq_off = h->p_sq;
  ps.D = h->j_D;
  ps.leaf = h->j_leaf;
  cudaError_t e;
  if ((e = mra::launch_predict_joint(h->d_desc, h->M, h->r, h->nlmax, ps, mode, h->status, h->stream, &g_launches,
                                     &h->timer)))
    return cuda_fail(e, "joint prediction launch");
  *ps_out = ps;
  return MRA_OK;
}

int mra_predict_joint(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where,
                      double* mean_out, double* cov_out) {
  g_err.clear();
  if (!h || !theta || !plocs || !mean_out || !cov_out) return fail(MRA_ERR_ARG, "null argument");
  if (np > MRA_MAX_JOINT_POINTS)
    return fail(MRA_ERR_LIMIT, "np = %lld exceeds MRA_MAX_JOINT_POINTS (%d)", (long long)np, MRA_MAX_JOINT_POINTS);
  mra::PredState ps;
  int rc = joint_factors(h, theta, plocs, np, where, 1, where == MRA_HOST ? np * np : 0, &ps);
  if (rc) return rc;
  cudaError_t e;
  double* cov = where == MRA_HOST ? h->j_io : cov_out;
  if ((e = mra::launch_joint_cov(h->d_desc, ps, np, cov, h->stream, &g_launches))) return cuda_fail(e, "joint covariance");
  if (where == MRA_HOST) {
    if ((e = cudaMemcpyAsync(mean_out, h->p_mean, sizeof(double) * np, cudaMemcpyDeviceToHost, h->stream)) ||
        (e = cudaMemcpyAsync(cov_out, cov, sizeof(double) * np * np, cudaMemcpyDeviceToHost, h->stream)))
      return cuda_fail(e, "copy joint prediction");
  } else if ((e = cudaMemcpyAsync(mean_out, h->p_mean, sizeof(double) * np, cudaMemcpyDeviceToDevice, h->stream))) {
    return cuda_fail(e, "copy joint prediction");
  }
  int hs[4];
  if ((e = sync_status(h, hs, nullptr, 0, nullptr))) return cuda_fail(e, "joint prediction");
  collect_times(h);
  if (hs[0]) return status_error(hs);
  return MRA_OK;
}

int mra_simulate_xi_len(mra_handle* h, int64_t* len_out) {
  g_err.clear();
  if (!h || !len_out) return fail(MRA_ERR_ARG, "null argument");
  if (!h->parts.empty()) return fail(MRA_ERR_STATE, "not available on a batch handle");
  int64_t regions = 0;
  for (int m = 0; m < h->M; ++m) regions += h->nfull(m);
  *len_out = regions * h->r;
  return MRA_OK;
}

int mra_simulate(mra_handle* h, const mra_params* theta, const double* plocs, int64_t np, int where, int64_t nsim,
                 const double* xi, const double* zeta, double* draws_out) {
  g_err.clear();
  if (!h || !theta || !plocs || !draws_out || (!xi && h->M > 0) || !zeta) return fail(MRA_ERR_ARG, "null argument");
  if (nsim < 1) return fail(MRA_ERR_ARG, "nsim must be >= 1");
  int64_t nxi = 0;
  int rc = mra_simulate_xi_len(h, &nxi);
  if (rc) return rc;
  const int64_t io = where == MRA_HOST ? nsim * (nxi + 2 * np) : 0;
  mra::PredState ps;
  if ((rc = joint_factors(h, theta, plocs, np, where, 2, io, &ps))) return rc;
  cudaError_t e;
  const double *dxi = xi, *dz = zeta;
  double* dd = draws_out;
  if (where == MRA_HOST) {
    double* x = h->j_io;
    if ((nxi > 0 && (e = cudaMemcpyAsync(x, xi, sizeof(double) * nsim * nxi, cudaMemcpyHostToDevice, h->stream))) ||
        (e = cudaMemcpyAsync(x + nsim * nxi, zeta, sizeof(double) * nsim * np, cudaMemcpyHostToDevice, h->stream)))
      return cuda_fail(e, "copy normals");
    dxi = x;
    dz = x + nsim * nxi;
    dd = x + nsim * (nxi + np);
  }
  if ((e = mra::launch_simulate(h->d_desc, h->M, ps, np, nsim, nxi, dxi, dz, dd, h->stream, &g_launches)))
    return cuda_fail(e, "simulation launch");
  if (where == MRA_HOST &&
      (e = cudaMemcpyAsync(draws_out, dd, sizeof(double) * nsim * np, cudaMemcpyDeviceToHost, h->stream)))
    return cuda_fail(e, "copy draws");
  int hs[4];
  if ((e = sync_status(h, hs, nullptr, 0, nullptr))) return cuda_fail(e, "simulation");
  collect_times(h);
  if (hs[0]) {
    if (hs[0] == mra::ST_NOT_PD && hs[1] == h->M + 1)
      return fail(MRA_ERR_NOT_PD, "the predictive covariance of the points in leaf %d is not positive definite "
                  "(coincident or nearly coincident prediction points)", hs[2]);
    return status_error(hs);
  }
  return MRA_OK;
}

// ---------------------------------------------------------------------------
// Batches of datasets
// ---------------------------------------------------------------------------
int mra_build_batch(const mra_config* cfgs, const double* const* locs, const double* const* ys, const int64_t* ns,
                    int ndata, int where, mra_handle** out) {
  g_err.clear();
  if (!out) return fail(MRA_ERR_ARG, "out is null");
  *out = nullptr;
  if (!cfgs || !locs || !ys || !ns || ndata < 1) return fail(MRA_ERR_ARG, "need at least one dataset");
  for (int d = 1; d < ndata; ++d)
    if (cfgs[d].r != cfgs[0].r || cfgs[d].precision != cfgs[0].precision)
      return fail(MRA_ERR_ARG, "all datasets of a batch need the same r and precision (dataset %d differs)", d);
  mra_handle* h = new mra_handle();
  h->cfg = cfgs[0];
  h->r = cfgs[0].r;
  for (int d = 0; d < ndata; ++d) {
    mra_handle* p = nullptr;
    int rc = mra_build(&cfgs[d], locs[d], ys[d], ns[d], where, &p);
    if (rc) {
      std::string msg = g_err;
      mra_free(h);
      return fail(rc, "dataset %d: %s", d, msg.c_str());
    }
    h->parts.push_back(p);
    if (p->s_lvl) {
      mra_free(h);
      return fail(MRA_ERR_ARG, "dataset %d: a batch evaluates its datasets whole (set stream_level = -1, or "
                  "evaluate it on its own handle)", d);
    }
    h->M = std::max(h->M, p->M);
    h->nlmax = std::max(h->nlmax, p->nlmax);
    h->n += p->n;
  }
  // work lists: one launch per level over every dataset's regions at that depth
  std::vector<int2> items;
  std::vector<std::pair<int, size_t>> lists;   // (count, start) in the order below
  auto add_list = [&](auto&& gen) {
    const size_t start = items.size();
    gen();
    lists.push_back({(int)(items.size() - start), start});
  };
  const int maxM = h->M;
  for (int m = 0; m < maxM; ++m)
    add_list([&] {
      for (int d = 0; d < ndata; ++d)
        if (h->parts[d]->M > m)
          for (int32_t c = 0; c < h->parts[d]->tab.nreg[m]; ++c) items.push_back(make_int2(d, c));
    });
  for (int m = 1; m < maxM; ++m)
    add_list([&] {
      for (int d = 0; d < ndata; ++d)
        if (h->parts[d]->M > m)
          for (int32_t c = 0; c < h->parts[d]->tab.nreg[m - 1]; ++c) items.push_back(make_int2(d, c));
    });
  add_list([&] {
    for (int d = 0; d < ndata; ++d)
      for (int32_t c = 0; c < h->parts[d]->tab.nreg[h->parts[d]->M]; ++c) items.push_back(make_int2(d, c));
  });
  add_list([&] {
    for (int d = 0; d < ndata; ++d)
      if (h->parts[d]->M > 0)
        for (int32_t c = 0; c < h->parts[d]->tab.nreg[h->parts[d]->M - 1]; ++c) items.push_back(make_int2(d, c));
  });
  // emulated form: the datasets' groups of leaves, as one list
  std::vector<int2> bgi;
  std::vector<int> bgc;
  if (h->cfg.precision == MRA_PREC_EMU) {
    h->lrows = MRA_MAX_LEAF;
    for (int d = 0; d < ndata; ++d) {
      const mra_handle* q = h->parts[d];
      if (q->lrows) {
        for (size_t k = 0; k < q->gitems.size(); ++k) {
          bgi.push_back(make_int2(d, q->gitems[k].y));
          bgc.push_back(q->gcnt[k]);
        }
      } else {
        for (int32_t c = 0; c < q->tab.nreg[q->M]; ++c) {
          bgi.push_back(make_int2(d, c));
          bgc.push_back(1);
        }
      }
    }
  }
  // and their groups of sibling regions per prior level
  std::vector<int2> bpi;
  std::vector<int> bpc;
  int64_t bpo[mra::MAXL] = {}, bpn[mra::MAXL] = {};
  int brcap = 0;
  if (h->cfg.precision == MRA_PREC_EMU) {
    for (int m = 1; m < h->M; ++m) {
      bpo[m] = (int64_t)bpi.size();
      for (int d = 0; d < ndata; ++d) {
        const mra_handle* q = h->parts[d];
        if (q->M <= m) continue;
        if (q->prcap) {
          brcap = std::max(brcap, q->prcap);
          for (int64_t k = q->pwo[m]; k < q->pwo[m] + q->pwn[m]; ++k) {
            bpi.push_back(make_int2(d, q->pitems[k].y));
            bpc.push_back(q->pcnt[k]);
          }
        } else {
          for (int32_t c = 0; c < q->tab.nreg[m]; ++c) {
            bpi.push_back(make_int2(d, c));
            bpc.push_back(1);
          }
        }
      }
      bpn[m] = (int64_t)bpi.size() - bpo[m];
    }
  }
  // and their groups for the leaf chain
  std::vector<int2> bci;
  std::vector<int> bcc;
  if (h->cfg.precision == MRA_PREC_EMU) {
    for (int d = 0; d < ndata; ++d) {
      const mra_handle* q = h->parts[d];
      if (q->M == 0) continue;
      if (!q->citems.empty()) {
        for (size_t k = 0; k < q->citems.size(); ++k) {
          bci.push_back(make_int2(d, q->citems[k].y));
          bcc.push_back(q->ccnt[k]);
        }
      } else {
        for (int32_t c = 0; c < q->tab.nreg[q->M - 1]; ++c) {
          bci.push_back(make_int2(d, c));
          bcc.push_back(1);
        }
      }
    }
  }
  int2* d_items = nullptr;
  int2* d_bgi = nullptr;
  int* d_bgc = nullptr;
  int2* d_bpi = nullptr;
  int* d_bpc = nullptr;
  int2* d_bci = nullptr;
  int* d_bcc = nullptr;
  Arena& A = h->batch;
  A.want(&d_items, std::max<size_t>(items.size(), 1));
  if (!bgi.empty()) {
    A.want(&d_bgi, bgi.size());
    A.want(&d_bgc, bgc.size());
  }
  if (!bpi.empty()) {
    A.want(&d_bpi, bpi.size());
    A.want(&d_bpc, bpc.size());
  }
  if (!bci.empty()) {
    A.want(&d_bci, bci.size());
    A.want(&d_bcc, bcc.size());
  }
  A.want(&h->d_descs, ndata);
  A.want(&h->d_roots, 2 * (size_t)ndata);
  A.want(&h->status, 4);
  cudaError_t e;
  if ((e = A.commit())) { mra_free(h); return fail(MRA_ERR_OOM, "device allocation (batch): %s", cudaGetErrorString(e)); }
  if ((e = cudaMallocHost((void**)&h->pinned, (64 + 2 * (size_t)ndata) * sizeof(double))) ||
      (e = cudaMallocHost((void**)&h->pinned_descs, sizeof(mra::Desc) * ndata))) {
    mra_free(h); return cuda_fail(e, "cudaMallocHost");
  }
  if ((e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking))) { mra_free(h); return cuda_fail(e, "stream"); }
  h->own_stream = 1;
  if (!items.empty() &&
      (e = cudaMemcpy(d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice))) {
    mra_free(h); return cuda_fail(e, "work lists");
  }
  if (!bgi.empty() && ((e = cudaMemcpy(d_bgi, bgi.data(), sizeof(int2) * bgi.size(), cudaMemcpyHostToDevice)) ||
                       (e = cudaMemcpy(d_bgc, bgc.data(), sizeof(int) * bgc.size(), cudaMemcpyHostToDevice)))) {
    mra_free(h); return cuda_fail(e, "leaf groups");
  }
  if (!bci.empty() && ((e = cudaMemcpy(d_bci, bci.data(), sizeof(int2) * bci.size(), cudaMemcpyHostToDevice)) ||
                       (e = cudaMemcpy(d_bcc, bcc.data(), sizeof(int) * bcc.size(), cudaMemcpyHostToDevice)))) {
    mra_free(h); return cuda_fail(e, "chain groups");
  }
  if (!bpi.empty() && ((e = cudaMemcpy(d_bpi, bpi.data(), sizeof(int2) * bpi.size(), cudaMemcpyHostToDevice)) ||
                       (e = cudaMemcpy(d_bpc, bpc.data(), sizeof(int) * bpc.size(), cudaMemcpyHostToDevice)))) {
    mra_free(h); return cuda_fail(e, "prior groups");
  }
  mra::Plan& p = h->plan;
  p = mra::Plan();
  p.maxM = maxM;
  p.tile = mra::tile_for_r(h->r);
  p.r = h->r;
  p.mixed = h->cfg.precision == MRA_PREC_MIXED ? 1 : (h->cfg.precision == MRA_PREC_EMU ? 2 : 0);
  p.nlmax = h->nlmax;
  int li = 0;
  for (int m = 0; m < maxM; ++m, ++li) { p.n_lvl[m] = lists[li].first; p.w_lvl[m] = d_items + lists[li].second; }
  for (int m = 1; m < maxM; ++m, ++li) { p.n_agg[m] = lists[li].first; p.w_agg[m] = d_items + lists[li].second; }
  p.n_leaf = lists[li].first; p.w_leaf = d_items + lists[li].second; ++li;
  if (!bgi.empty()) {
    p.n_leaf = (int)bgi.size();
    p.w_leaf = d_bgi;
    p.c_leaf = d_bgc;
    p.lrows = h->lrows;
  }
  if (!bci.empty()) {
    p.w_chn = d_bci;
    p.c_chn = d_bcc;
    p.n_chn = (int)bci.size();
  }
  if (!bpi.empty() && brcap) {
    for (int m = 1; m < maxM; ++m) {
      p.w_pri[m] = d_bpi + bpo[m];
      p.c_pri[m] = d_bpc + bpo[m];
      p.n_pri[m] = (int)bpn[m];
    }
    p.rcap = brcap;
  }
  p.n_syrk = lists[li].first; p.w_syrk = d_items + lists[li].second; ++li;
  for (int d = 0; d < ndata; ++d) p.t_syrk = std::max(p.t_syrk, h->parts[d]->M * (h->parts[d]->M + 1) / 2);
  h->h_descs.resize(ndata);
  for (int d = 0; d < ndata; ++d) {
    mra_handle* q = h->parts[d];
    mra_params th{1.0, 1.0, 0.0};
    upload_desc(q, &th);               // fills q->hd (the copy to q's own descriptor is harmless)
    h->h_descs[d] = q->hd;
    h->h_descs[d].nlmax = h->nlmax;    // one shared-memory layout for the whole batch
    h->h_descs[d].lrows = h->lrows;
  }
  if ((e = cudaDeviceSynchronize())) { mra_free(h); return cuda_fail(e, "batch set-up"); }
  size_t need = p.mixed ? mra::leaf_tc_smem_bytes(std::max(h->nlmax, h->lrows), p.mixed == 2)
                        : mra::leaf_smem_bytes(h->r, h->nlmax);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((size_t)optin < need) { mra_free(h); return fail(MRA_ERR_LIMIT, "leaf kernel shared memory exceeds the device limit"); }
  *out = h;
  return MRA_OK;
}

}  // extern "C"

namespace {

// Descriptors, one batched evaluation, roots to the pinned buffer (stream-ordered).
cudaError_t batch_sequence(mra_handle* h) {
  const int nd = (int)h->parts.size();
  cudaError_t e;
  if ((e = cudaMemcpyAsync(h->d_descs, h->pinned_descs, sizeof(mra::Desc) * nd, cudaMemcpyHostToDevice, h->stream)) ||
      (e = cudaMemsetAsync(h->status, 0, sizeof(int) * 4, h->stream)))
    return e;
  if ((e = mra::launch_loglik(h->plan, h->d_descs, h->status, h->stream, &g_launches, &h->timer))) return e;
  if ((e = mra::launch_gather_roots(h->d_descs, nd, h->d_roots, h->stream, &g_launches))) return e;
  if ((e = cudaMemcpyAsync(h->pinned + 64, h->d_roots, sizeof(double) * 2 * nd, cudaMemcpyDeviceToHost, h->stream)) ||
      (e = cudaMemcpyAsync(h->pinned, h->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, h->stream)))
    return e;
  return cudaSuccess;
}

int batch_results(mra_handle* h, double* loglik_out) {
  int hs[4];
  memcpy(hs, h->pinned, sizeof hs);
  if (hs[0]) return status_error(hs);
  for (size_t d = 0; d < h->parts.size(); ++d)
    loglik_out[d] = -0.5 * (h->pinned[64 + 2 * d] + h->pinned[64 + 2 * d + 1]) -
                    0.5 * (double)h->parts[d]->n * std::log(2.0 * M_PI);
  return MRA_OK;
}

int set_batch_params(mra_handle* h, const mra_params* thetas) {
  for (size_t d = 0; d < h->parts.size(); ++d) {
    if (!params_ok(&thetas[d]) || !nu_ok(h->parts[d]->cfg.cov_family, &thetas[d]))
      return fail(MRA_ERR_ARG, "theta of dataset %zu is invalid", d);
    h->h_descs[d].cv = mra::make_cov(thetas[d].sigma2, thetas[d].range, h->parts[d]->cfg.cov_family,
                                     h->parts[d]->cfg.nonstat, thetas[d].nu);
    h->h_descs[d].tau2 = thetas[d].tau2;
  }
  memcpy(h->pinned_descs, h->h_descs.data(), sizeof(mra::Desc) * h->parts.size());
  return MRA_OK;
}

void drop_graph(mra_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
}

}  // namespace

extern "C" {

int mra_autotune(mra_handle* h, const mra_params* thetas, int* tile_out) {
  g_err.clear();
  if (!h || !thetas) return fail(MRA_ERR_ARG, "null argument");
  const bool is_batch = !h->parts.empty();
  int cands[3], nc = 0;
  const int base = mra::tile_for_r(h->r);
  for (int t : {16, 32, 64})
    if (t >= base) cands[nc++] = t;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) || cudaEventCreate(&e1)) return fail(MRA_ERR_CUDA, "cudaEventCreate failed");
  float best = 1e30f;
  int best_tile = base;
  std::vector<double> tmp(is_batch ? h->parts.size() : 1);
  const bool timer_was_on = h->timer.on;
  h->timer.on = false;
  int rc = MRA_OK;
  for (int k = 0; k < nc && !rc; ++k) {
    h->plan.tile = cands[k];
    float ms = 0.f;
    for (int rep = 0; rep < 2 && !rc; ++rep) {
      cudaEventRecord(e0, h->stream);
      if (is_batch) {
        rc = set_batch_params(h, thetas);
        if (!rc) {
          cudaError_t e = batch_sequence(h);
          if (!e) e = cudaStreamSynchronize(h->stream);
          rc = e ? cuda_fail(e, "autotune") : batch_results(h, tmp.data());
        }
      } else {
        rc = mra_loglik(h, thetas, tmp.data());
      }
      cudaEventRecord(e1, h->stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
    }
    if (!rc && ms < best) { best = ms; best_tile = cands[k]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timer.on = timer_was_on;
  h->plan.tile = best_tile;
  if (rc) return rc;
  h->tuned = true;
  drop_graph(h);
  if (tile_out) *tile_out = best_tile;
  return MRA_OK;
}

int mra_loglik_batch(mra_handle* h, const mra_params* thetas, double* loglik_out) {
  g_err.clear();
  if (!h || !thetas || !loglik_out) return fail(MRA_ERR_ARG, "null argument");
  if (h->parts.empty()) return fail(MRA_ERR_STATE, "not a batch handle (use mra_build_batch)");
  int rc;
  if (!h->tuned && (rc = mra_autotune(h, thetas, nullptr))) return rc;
  if ((rc = set_batch_params(h, thetas))) return rc;
  cudaError_t e;
  if (h->timer.on) {   // per-kernel events: run the launches directly
    if ((e = batch_sequence(h)) || (e = cudaStreamSynchronize(h->stream))) return cuda_fail(e, "batch");
    ++h->nevals;
    collect_times(h);
    return batch_results(h, loglik_out);
  }
  if (!h->gexec) {
    if ((e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal))) return cuda_fail(e, "graph capture");
    const int64_t before = g_launches;
    cudaError_t e1 = batch_sequence(h);
    h->graph_launches = g_launches - before;
    g_launches = before;
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &h->graph);
    if (e1 || e2) {
      drop_graph(h);
      return cuda_fail(e1 ? e1 : e2, "graph capture");
    }
    if ((e = cudaGraphInstantiate(&h->gexec, h->graph, 0))) {
      drop_graph(h);
      return cuda_fail(e, "graph instantiate");
    }
  }
  if ((e = cudaGraphLaunch(h->gexec, h->stream)) || (e = cudaStreamSynchronize(h->stream)))
    return cuda_fail(e, "graph launch");
  g_launches += h->graph_launches;
  return batch_results(h, loglik_out);
}

int mra_loglik_grad_batch(mra_handle* h, const mra_params* thetas, double* loglik_out, double* grad_out) {
  g_err.clear();
  if (!h || !thetas || !loglik_out || !grad_out) return fail(MRA_ERR_ARG, "null argument");
  if (h->parts.empty()) return fail(MRA_ERR_STATE, "not a batch handle (use mra_build_batch)");
  for (size_t d = 0; d < h->parts.size(); ++d) {
    if (!params_ok(&thetas[d]) || !nu_ok(h->parts[d]->cfg.cov_family, &thetas[d]))
      return fail(MRA_ERR_ARG, "theta of dataset %zu is invalid", d);
    if (h->parts[d]->cfg.cov_family == MRA_COV_MATERN)
      return fail(MRA_ERR_ARG, "dataset %zu: the free-smoothness gradient has four components; use "
                  "mra_loglik_grad on its own handle", d);
  }
  // Dataset by dataset on the batch's stream: the adjoint of each dataset keeps
  // its own gradient storage (allocated by its first call).
  for (size_t d = 0; d < h->parts.size(); ++d) {
    mra_handle* p = h->parts[d];
    cudaStream_t keep = p->stream;
    p->stream = h->stream;
    const int rc = mra_loglik_grad(p, &thetas[d], loglik_out + d, grad_out + 3 * d);
    p->stream = keep;
    if (rc) {
      std::string msg = g_err;
      return fail(rc, "dataset %zu: %s", d, msg.c_str());
    }
  }
  return MRA_OK;
}

int mra_batch_info(mra_handle* h, int* ndata_out, int* tile_out) {
  g_err.clear();
  if (!h || !ndata_out) return fail(MRA_ERR_ARG, "null argument");
  *ndata_out = (int)h->parts.size();
  if (tile_out) *tile_out = h->plan.tile;
  return MRA_OK;
}

}  // extern "C"
