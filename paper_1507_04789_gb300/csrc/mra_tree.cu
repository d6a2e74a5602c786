// mra_tree.cu -- partition of the observations (Sec. 2.2) on the device.
//
// Every point descends the partition to its leaf (reading: half-open cells
// [lo, mid), [mid, hi], the last cell closed at the bounding box; level m cuts
// every region into 2^hx_m x 2^hy_m children by repeated midpoint halving, child
// j = c_x + 2^hx_m c_y; the quadtree is hx = hy = 1, j = b_x + 2 b_y), then a
// counting sort by leaf gives contiguous leaves in region-id (for the quadtree
// Morton) order; a per-leaf rank sort restores the original order inside a
// leaf so that the result does not depend on atomic ordering.
#include "mra_launch.h"

namespace mra {

__global__ void leaf_id_kernel(const double* __restrict__ locs, int64_t n,
                               const double* __restrict__ bbox, int M, unsigned long long hx,
                               unsigned long long hy, int32_t* __restrict__ leaf_id,
                               int32_t* __restrict__ counts, int* status) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = locs[2 * i], y = locs[2 * i + 1];
  double x0 = bbox[0], x1 = bbox[1], y0 = bbox[2], y1 = bbox[3];
  if (!(x >= x0 && x <= x1 && y >= y0 && y <= y1)) {   // also rejects NaN
    flag_error(status, ST_ARG, -1, (long)i);
    leaf_id[i] = -1;
    return;
  }
  int32_t idx = 0;
  for (int t = 1; t <= M; ++t) {
    const int a = lvl_hx(hx, t), c = lvl_hx(hy, t);
    int cx = 0, cy = 0;
    for (int q = 0; q < a; ++q) {
      const double xm = 0.5 * (x0 + x1);
      const int b = x >= xm;
      if (b) x0 = xm; else x1 = xm;
      cx = 2 * cx + b;
    }
    for (int q = 0; q < c; ++q) {
      const double ym = 0.5 * (y0 + y1);
      const int b = y >= ym;
      if (b) y0 = ym; else y1 = ym;
      cy = 2 * cy + b;
    }
    idx = (idx << (a + c)) + cx + (cy << a);
  }
  leaf_id[i] = idx;
  atomicAdd(&counts[idx], 1);
}

// Exclusive scan of counts (nl entries) into off and of counts^2 into sq_off,
// plus the largest count.  One CTA of 1024 threads, each owning a contiguous
// chunk.
__global__ void __launch_bounds__(1024) scan_kernel(const int32_t* __restrict__ counts, int64_t nl,
                                                    int64_t* __restrict__ off, int64_t* __restrict__ sq_off,
                                                    int32_t* __restrict__ max_count) {
  __shared__ int64_t s1[1024], s2[1024];
  __shared__ int32_t smax[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (nl + 1023) / 1024;
  const int64_t b = t * chunk, e = min(nl, b + chunk);
  int64_t a1 = 0, a2 = 0;
  int32_t mx = 0;
  for (int64_t i = b; i < e; ++i) {
    int64_t c = counts[i];
    a1 += c;
    a2 += c * c;
    mx = max(mx, (int32_t)c);
  }
  s1[t] = a1; s2[t] = a2; smax[t] = mx;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {       // Hillis-Steele inclusive scan
    int64_t v1 = t >= o ? s1[t - o] : 0, v2 = t >= o ? s2[t - o] : 0;
    int32_t vm = t >= o ? smax[t - o] : 0;
    __syncthreads();
    s1[t] += v1; s2[t] += v2; smax[t] = max(smax[t], vm);
    __syncthreads();
  }
  int64_t p1 = t ? s1[t - 1] : 0, p2 = t ? s2[t - 1] : 0;
  for (int64_t i = b; i < e; ++i) {
    off[i] = p1;
    sq_off[i] = p2;
    int64_t c = counts[i];
    p1 += c;
    p2 += c * c;
  }
  if (t == 1023) {
    off[nl] = s1[1023];
    sq_off[nl] = s2[1023];
    *max_count = smax[1023];
  }
}

__global__ void scatter_kernel(const int32_t* __restrict__ leaf_id, int64_t n, const int64_t* __restrict__ off,
                               int32_t* __restrict__ cursor, int64_t* __restrict__ perm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t f = leaf_id[i];
  if (f < 0) return;
  int64_t pos = off[f] + atomicAdd(&cursor[f], 1);
  perm[pos] = i;
}

// Sort each leaf's indices increasingly (rank sort in shared memory).
constexpr int SEG_MAX = 1024;
__global__ void __launch_bounds__(256) segsort_kernel(const int64_t* __restrict__ off, int64_t* __restrict__ perm,
                                                      int* status) {
  __shared__ int64_t v[SEG_MAX];
  const int64_t f = blockIdx.x;
  const int64_t o0 = off[f];
  const int nf = (int)(off[f + 1] - o0);
  if (nf <= 1) return;
  if (nf > SEG_MAX) {
    if (threadIdx.x == 0) flag_error(status, ST_LIMIT, -1, (long)f);
    return;
  }
  for (int t = threadIdx.x; t < nf; t += blockDim.x) v[t] = perm[o0 + t];
  __syncthreads();
  for (int t = threadIdx.x; t < nf; t += blockDim.x) {
    int64_t x = v[t];
    int rank = 0;
    for (int k = 0; k < nf; ++k) rank += v[k] < x;
    perm[o0 + rank] = x;
  }
}

__global__ void gather_kernel(const double* __restrict__ locs, const double* __restrict__ y,
                              const int64_t* __restrict__ perm, int64_t n, double* __restrict__ xs,
                              double* __restrict__ ys, double* __restrict__ yv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t p = perm[i];
  xs[i] = locs[2 * p];
  ys[i] = locs[2 * p + 1];
  if (yv && y) yv[i] = y[p];
}

__global__ void gather_y_kernel(const double* __restrict__ y, const int64_t* __restrict__ perm, int64_t n,
                                double* __restrict__ yv) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  yv[i] = y[perm[i]];
}

static unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256); }

cudaError_t launch_bin(const double* locs, int64_t n, const double* bbox_dev, int M, unsigned long long hx,
                       unsigned long long hy, int32_t* leaf_id, int32_t* counts, int32_t* cursor, int64_t* off,
                       int64_t* sq_off, int32_t* max_count, int64_t* perm, int* status,
                       cudaStream_t s, int64_t* launches, bool stable) {
  const int64_t nl = int64_t(1) << lvl_depth(hx, hy, M);
  cudaError_t e;
  if ((e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * nl, s))) return e;
  if ((e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * nl, s))) return e;
  leaf_id_kernel<<<blocks_for(n), 256, 0, s>>>(locs, n, bbox_dev, M, hx, hy, leaf_id, counts, status);
  scan_kernel<<<1, 1024, 0, s>>>(counts, nl, off, sq_off, max_count);
  scatter_kernel<<<blocks_for(n), 256, 0, s>>>(leaf_id, n, off, cursor, perm);
  if (stable) segsort_kernel<<<(unsigned)nl, 256, 0, s>>>(off, perm, status);
  *launches += stable ? 4 : 3;
  return cudaGetLastError();
}

cudaError_t launch_gather(const double* locs, const double* y, const int64_t* perm, int64_t n,
                          double* xs, double* ys, double* yv, cudaStream_t s, int64_t* launches) {
  gather_kernel<<<blocks_for(n), 256, 0, s>>>(locs, y, perm, n, xs, ys, yv);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_gather_y(const double* y, const int64_t* perm, int64_t n, double* yv,
                            cudaStream_t s, int64_t* launches) {
  gather_y_kernel<<<blocks_for(n), 256, 0, s>>>(y, perm, n, yv);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace mra

namespace mra {

// Tables of a complete tree (every region active): identity maps.
__global__ void identity_tree_kernel(LevelState st, int M, unsigned long long hx, unsigned long long hy) {
  for (int m = 0; m <= M; ++m) {
    const long cnt = 1L << lvl_depth(hx, hy, m);
    const int bm = m > 0 ? lvl_bits(hx, hy, m) : 0, bc = m < M ? lvl_bits(hx, hy, m + 1) : 0;
    for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < cnt; c += (long)gridDim.x * blockDim.x) {
      st.mort[m][c] = (int32_t)c;
      st.cid[m][c] = (int32_t)c;
      if (m > 0) st.par[m][c] = (int32_t)(c >> bm);
      if (m < M) {
        st.cfirst[m][c] = (int32_t)(c << bc);
        st.ccnt[m][c] = 1 << bc;
      }
    }
  }
}

cudaError_t launch_identity_tree(const LevelState& st, int M, unsigned long long hx, unsigned long long hy,
                                 cudaStream_t s, int64_t* launches) {
  identity_tree_kernel<<<256, 256, 0, s>>>(st, M, hx, hy);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace mra
