// Nearest-previous-neighbour search (Section 2.1) and test-point neighbours
// (Section 4.1), bit-exact: candidates are ranked by the key (d2, index) with d2
// evaluated in float64 without contraction, ties to the lower index.
//
// Points are bucketed into a uniform grid (about two points per cell, points of
// a cell sorted by index). A query scans rings of cells around its own cell; in a
// cell it stops at the first index not earlier than the query. It stops after a
// ring once it holds its k candidates and the distance from the query to the
// boundary of the scanned square (less a slack of 1e-9 cell widths) exceeds the
// k-th candidate distance, so no unscanned point can tie or beat it. Early rows
// (index < kBrute) scan all earlier points directly.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "vl_device.cuh"

namespace vl {

constexpr int kMaxM = 64;
constexpr int kBrute = 2048;

__device__ __forceinline__ bool key_less(double d2, int j, double bd, int bj) {
  return d2 < bd || (d2 == bd && j < bj);
}

__device__ __forceinline__ void topk_insert(double* bd, int* bj, int& cnt, int want, double d2, int j) {
  if (cnt == want) {
    if (!key_less(d2, j, bd[want - 1], bj[want - 1])) return;
    --cnt;
  }
  int p = cnt;
  while (p > 0 && key_less(d2, j, bd[p - 1], bj[p - 1])) {
    bd[p] = bd[p - 1];
    bj[p] = bj[p - 1];
    --p;
  }
  bd[p] = d2;
  bj[p] = j;
  ++cnt;
}

struct Grid {
  double x0, y0, h, inv_h;
  int gx, gy;
  const int* cell_start;   // gx*gy + 1
  const int* cell_idx;     // point index, sorted by (cell, index)
  const double2* cell_pts; // coordinates in the same order
};

__device__ __forceinline__ int cell_of(double v, double v0, double inv_h, int g) {
  double f = floor((v - v0) * inv_h);
  int c = (f < 0.0) ? 0 : (f >= (double)g ? g - 1 : (int)f);
  return c;
}

// Ring search; `limit` = only indices < limit count (prev search), n for cross.
__device__ void ring_search(const Grid& G, double qx, double qy, int limit, int want, double* bd,
                            int* bj, int& cnt) {
  const int cx = cell_of(qx, G.x0, G.inv_h, G.gx);
  const int cy = cell_of(qy, G.y0, G.inv_h, G.gy);
  const int rmax = max(G.gx, G.gy);
  for (int R = 0; R <= rmax; ++R) {
    for (int dy = -R; dy <= R; ++dy) {
      const int iy = cy + dy;
      if (iy < 0 || iy >= G.gy) continue;
      const bool edge = (dy == -R || dy == R);
      for (int dx = -R; dx <= R; dx += (edge || R == 0) ? 1 : 2 * R) {
        const int ix = cx + dx;
        if (ix >= 0 && ix < G.gx) {
          const int c = iy * G.gx + ix;
          const int e = G.cell_start[c + 1];
          for (int p = G.cell_start[c]; p < e; ++p) {
            const int j = G.cell_idx[p];
            if (j >= limit) break;
            const double2 pt = G.cell_pts[p];
            topk_insert(bd, bj, cnt, want, dist2_exact(qx, qy, pt.x, pt.y), j);
          }
        }
        if (R == 0) break;
      }
    }
    const bool all = (cx - R <= 0) && (cx + R >= G.gx - 1) && (cy - R <= 0) && (cy + R >= G.gy - 1);
    if (all) return;
    if (cnt == want) {
      double lb = INFINITY;
      if (cx - R - 1 >= 0) lb = fmin(lb, qx - (G.x0 + (double)(cx - R) * G.h));
      if (cx + R + 1 <= G.gx - 1) lb = fmin(lb, (G.x0 + (double)(cx + R + 1) * G.h) - qx);
      if (cy - R - 1 >= 0) lb = fmin(lb, qy - (G.y0 + (double)(cy - R) * G.h));
      if (cy + R + 1 <= G.gy - 1) lb = fmin(lb, (G.y0 + (double)(cy + R + 1) * G.h) - qy);
      lb -= 1e-9 * G.h;
      if (lb > 0.0 && lb * lb > bd[want - 1]) return;
    }
  }
}

__global__ void knn_prev_kernel(const double2* __restrict__ pts, int n, int m, Grid G,
                                int32_t* __restrict__ N_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int want = min(k, m);
  double bd[kMaxM];
  int bj[kMaxM];
  int cnt = 0;
  const double2 q = pts[k];
  if (want > 0) {
    if (k < kBrute) {
      for (int j = 0; j < k; ++j) {
        const double2 p = pts[j];
        topk_insert(bd, bj, cnt, want, dist2_exact(q.x, q.y, p.x, p.y), j);
      }
    } else {
      ring_search(G, q.x, q.y, k, want, bd, bj, cnt);
    }
  }
  for (int c = 0; c < m; ++c) N_out[(int64_t)k * m + c] = c < cnt ? bj[c] : -1;
}

__global__ void knn_cross_kernel(const double2* __restrict__ test, int np, int n, int m, Grid G,
                                 int32_t* __restrict__ N_out) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= np) return;
  const int want = min(m, n);
  double bd[kMaxM];
  int bj[kMaxM];
  int cnt = 0;
  const double2 q = test[a];
  if (want > 0) ring_search(G, q.x, q.y, n, want, bd, bj, cnt);
  for (int c = 0; c < m; ++c) N_out[(int64_t)a * m + c] = c < cnt ? bj[c] : -1;
}

// ----------------------------------------------------------------------------- bbox
__global__ void minmax_kernel(const double2* __restrict__ a, int n, double4* __restrict__ part) {
  double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double2 p = a[i];
    x0 = fmin(x0, p.x);
    x1 = fmax(x1, p.x);
    y0 = fmin(y0, p.y);
    y1 = fmax(y1, p.y);
  }
  __shared__ double4 sh[256];
  sh[threadIdx.x] = make_double4(x0, x1, y0, y1);
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      double4 o = sh[threadIdx.x + s], me = sh[threadIdx.x];
      sh[threadIdx.x] = make_double4(fmin(me.x, o.x), fmax(me.y, o.y), fmin(me.z, o.z), fmax(me.w, o.w));
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

vl_status bbox(Ctx* c, const double* locs, int64_t n, const double* extra, int64_t n_extra, double out[4]) {
  const int nb = 120;
  double4* part = static_cast<double4*>(c->arena.alloc(sizeof(double4) * 2 * nb));
  if (!part) return fail(c, VL_ERR_OOM, "workspace exhausted (bbox)");
  int used = 0;
  if (n > 0) {
    minmax_kernel<<<nb, 256, 0, VL_STREAM(c)>>>(reinterpret_cast<const double2*>(locs), (int)n, part);
    used += nb;
  }
  if (n_extra > 0) {
    minmax_kernel<<<nb, 256, 0, VL_STREAM(c)>>>(reinterpret_cast<const double2*>(extra), (int)n_extra, part + used);
    used += nb;
  }
  std::vector<double4> h(used);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && used)
    e = cudaMemcpyAsync(h.data(), part, sizeof(double4) * used, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  c->arena.release(part);
  if (e != cudaSuccess) return cuda_fail(c, e, "bbox");
  out[0] = out[2] = INFINITY;
  out[1] = out[3] = -INFINITY;
  for (auto& v : h) {
    out[0] = std::min(out[0], v.x);
    out[1] = std::max(out[1], v.y);
    out[2] = std::min(out[2], v.z);
    out[3] = std::max(out[3], v.w);
  }
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]) || !std::isfinite(out[2]) || !std::isfinite(out[3]))
    return fail(c, VL_ERR_INVALID_ARG, "locations contain NaN or infinity");
  return VL_OK;
}

// ----------------------------------------------------------------------------- grid build
__global__ void cell_keys_kernel(const double2* __restrict__ p, int n, double x0, double y0, double inv_h,
                                 int gx, int gy, int* __restrict__ key, int* __restrict__ val,
                                 int* __restrict__ count) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = cell_of(p[i].y, y0, inv_h, gy) * gx + cell_of(p[i].x, x0, inv_h, gx);
  key[i] = c;
  val[i] = i;
  atomicAdd(&count[c], 1);
}

__global__ void gather_pts_kernel(const double2* __restrict__ p, const int* __restrict__ idx, int n,
                                  double2* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = p[idx[i]];
}

namespace {
struct GridMem {
  Ctx* c;
  std::vector<void*> blocks;
  void* get(size_t b) {
    void* p = c->arena.alloc(b + 16);
    if (p) blocks.push_back(p);
    return p;
  }
  ~GridMem() {
    for (void* p : blocks) c->arena.release(p);
  }
};
}  // namespace

// Builds the grid over `pts` (n points). bb = {xmin, xmax, ymin, ymax} covering all
// queries and points.
static vl_status build_grid(Ctx* c, GridMem& gm, const double2* pts, int n, const double bb[4], Grid& G) {
  double W = bb[1] - bb[0], H = bb[3] - bb[2];
  double cells = std::max(1.0, n / 2.0);
  double h;
  if (W > 0 && H > 0) h = std::sqrt(W * H / cells);
  else if (W > 0 || H > 0) h = std::max(W, H) / cells;
  else h = 1.0;
  long long gx = std::max(1LL, (long long)std::ceil(W / h));
  long long gy = std::max(1LL, (long long)std::ceil(H / h));
  while (gx * gy > (1LL << 26)) {
    h *= 1.5;
    gx = std::max(1LL, (long long)std::ceil(W / h));
    gy = std::max(1LL, (long long)std::ceil(H / h));
  }
  G.x0 = bb[0];
  G.y0 = bb[2];
  G.h = h;
  G.inv_h = 1.0 / h;
  G.gx = (int)gx;
  G.gy = (int)gy;
  const int ncell = (int)(gx * gy);
  int* key = (int*)gm.get(sizeof(int) * n);
  int* val = (int*)gm.get(sizeof(int) * n);
  int* key2 = (int*)gm.get(sizeof(int) * n);
  int* val2 = (int*)gm.get(sizeof(int) * n);
  int* count = (int*)gm.get(sizeof(int) * (ncell + 1));
  int* start = (int*)gm.get(sizeof(int) * (ncell + 1));
  double2* cpts = (double2*)gm.get(sizeof(double2) * n);
  if (!key || !val || !key2 || !val2 || !count || !start || !cpts)
    return fail(c, VL_ERR_OOM, "workspace exhausted (kNN grid)");
  VL_CUDA(c, cudaMemsetAsync(count, 0, sizeof(int) * (ncell + 1), c->stream));
  const int T = 256;
  if (n > 0)
    cell_keys_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(pts, n, G.x0, G.y0, G.inv_h, G.gx, G.gy, key, val, count);
  VL_CUDA(c, cudaGetLastError());
  size_t tb1 = 0, tb2 = 0;
  int bits = 1;
  while ((1LL << bits) < ncell + 1) ++bits;
  cub::DeviceRadixSort::SortPairs(nullptr, tb1, key, key2, val, val2, n, 0, bits, c->stream);
  cub::DeviceScan::ExclusiveSum(nullptr, tb2, count, start, ncell + 1, c->stream);
  void* tmp = gm.get(std::max(tb1, tb2));
  if (!tmp) return fail(c, VL_ERR_OOM, "workspace exhausted (kNN sort)");
  VL_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tb1, key, key2, val, val2, n, 0, bits, c->stream));
  VL_CUDA(c, cub::DeviceScan::ExclusiveSum(tmp, tb2, count, start, ncell + 1, c->stream));
  if (n > 0) gather_pts_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(pts, val2, n, cpts);
  VL_CUDA(c, cudaGetLastError());
  G.cell_start = start;
  G.cell_idx = val2;
  G.cell_pts = cpts;
  return VL_OK;
}

vl_status knn_prev_dev(Ctx* c, const double* locs_v, int64_t n, int m, int32_t* N_out) {
  if (m < 0 || m > kMaxM) return fail(c, VL_ERR_INVALID_ARG, "m must be in [0, 64]");
  if (n <= 0 || m == 0) {
    if (n > 0 && m > 0) VL_CUDA(c, cudaMemsetAsync(N_out, 0xff, sizeof(int32_t) * n * m, c->stream));
    return VL_OK;
  }
  double bb[4];
  VL_TRY(bbox(c, locs_v, n, nullptr, 0, bb));
  GridMem gm{c};
  Grid G;
  VL_TRY(build_grid(c, gm, reinterpret_cast<const double2*>(locs_v), (int)n, bb, G));
  const int T = 128;
  ProfScope ps(c, "knn", m);
  knn_prev_kernel<<<(int)((n + T - 1) / T), T, 0, VL_STREAM(c)>>>(reinterpret_cast<const double2*>(locs_v), (int)n, m, G, N_out);
  VL_CUDA(c, cudaGetLastError());
  VL_CUDA(c, cudaStreamSynchronize(c->stream));  // the grid lives in scratch
  return VL_OK;
}

vl_status knn_cross_dev(Ctx* c, const double* train, int64_t n, const double* test, int64_t np, int m,
                        int32_t* N_out) {
  if (m < 0 || m > kMaxM) return fail(c, VL_ERR_INVALID_ARG, "m must be in [0, 64]");
  if (np <= 0 || m == 0) return VL_OK;
  if (n <= 0) {
    VL_CUDA(c, cudaMemsetAsync(N_out, 0xff, sizeof(int32_t) * np * m, c->stream));
    return VL_OK;
  }
  double bb[4];
  VL_TRY(bbox(c, train, n, test, np, bb));
  GridMem gm{c};
  Grid G;
  VL_TRY(build_grid(c, gm, reinterpret_cast<const double2*>(train), (int)n, bb, G));
  const int T = 128;
  knn_cross_kernel<<<(int)((np + T - 1) / T), T, 0, VL_STREAM(c)>>>(reinterpret_cast<const double2*>(test), (int)np,
                                                                   (int)n, m, G, N_out);
  VL_CUDA(c, cudaGetLastError());
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

// ----------------------------------------------------------------------------- Morton order
__device__ __forceinline__ uint32_t spread16(uint32_t v) {
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

__global__ void morton_kernel(const double2* __restrict__ p, int n, double x0, double sx, double y0, double sy,
                              uint32_t* __restrict__ key, int* __restrict__ val) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double fx = (p[i].x - x0) * sx, fy = (p[i].y - y0) * sy;
  uint32_t qx = (uint32_t)fmin(fmax(fx, 0.0), 65535.0);
  uint32_t qy = (uint32_t)fmin(fmax(fy, 0.0), 65535.0);
  key[i] = (spread16(qy) << 1) | spread16(qx);
  val[i] = i;
}

// perm_out[s] = index (into locs) of the s-th point in Morton order; ties keep
// ascending index order.
vl_status morton_perm(Ctx* c, const double* locs, int64_t n, int32_t* perm_out) {
  double bb[4];
  VL_TRY(bbox(c, locs, n, nullptr, 0, bb));
  double W = bb[1] - bb[0], H = bb[3] - bb[2];
  double sx = W > 0 ? 65535.0 / W : 0.0, sy = H > 0 ? 65535.0 / H : 0.0;
  GridMem gm{c};
  uint32_t* key = (uint32_t*)gm.get(sizeof(uint32_t) * n);
  uint32_t* key2 = (uint32_t*)gm.get(sizeof(uint32_t) * n);
  int* val = (int*)gm.get(sizeof(int) * n);
  if (!key || !key2 || !val) return fail(c, VL_ERR_OOM, "workspace exhausted (Morton)");
  const int T = 256;
  morton_kernel<<<(int)((n + T - 1) / T), T, 0, VL_STREAM(c)>>>(reinterpret_cast<const double2*>(locs), (int)n, bb[0], sx,
                                                            bb[2], sy, key, val);
  VL_CUDA(c, cudaGetLastError());
  size_t tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, key, key2, val, perm_out, (int)n, 0, 32, c->stream);
  void* tmp = gm.get(tb);
  if (!tmp) return fail(c, VL_ERR_OOM, "workspace exhausted (Morton sort)");
  VL_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tb, key, key2, val, perm_out, (int)n, 0, 32, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

}  // namespace vl
