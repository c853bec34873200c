// Sparsity pattern of B in storage order, its transpose, and level schedules.
//
// Rows are stored in Morton order of the locations (a relabelling only; the
// Vecchia order still defines N(i) and the triangular structure), so that the
// neighbours a row gathers sit close to it in memory.
//
// Levels of the unit lower-triangular B:
//   forward  lev(i)  = 0 if N(i) is empty, else 1 + max_{j in N(i)} lev(j)
//   backward levT(j) = 0 if no row lists j, else 1 + max_{i: j in N(i)} levT(i)
// They are computed by a sync-free cooperative kernel that walks the Vecchia
// order (a topological order of the dependency graph): each warp takes rows
// w, w + W, w + 2W, ... and waits, with a bounded spin, on the rows it depends on.
// With every warp resident (cooperative launch) the earliest unfinished row always
// has its inputs ready, so the walk cannot deadlock.
#include <cooperative_groups.h>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <vector>

#include "vl_device.cuh"

namespace vl {

__global__ void storage_maps_kernel(int n, int m, const int32_t* __restrict__ perm, const int32_t* __restrict__ order,
                                    const double* __restrict__ locs_v, int32_t* __restrict__ s2v,
                                    int32_t* __restrict__ v2s, int32_t* __restrict__ s2u, int32_t* __restrict__ u2s,
                                    double* __restrict__ locs_s) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int v = perm[s];
  s2v[s] = v;
  v2s[v] = s;
  int u = order ? order[v] : v;
  s2u[s] = u;
  u2s[u] = s;
  locs_s[2 * s] = locs_v[2 * v];
  locs_s[2 * s + 1] = locs_v[2 * v + 1];
}

__global__ void translate_nbr_kernel(int n, int m, const int32_t* __restrict__ s2v, const int32_t* __restrict__ v2s,
                                     const int32_t* __restrict__ N_v, int32_t* __restrict__ nbr,
                                     unsigned long long* __restrict__ tkey, int32_t* __restrict__ tval,
                                     int32_t* __restrict__ count) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * m) return;
  int s = (int)(e / m), c = (int)(e % m);
  int jv = N_v[(int64_t)s2v[s] * m + c];
  int j = jv >= 0 ? v2s[jv] : -1;
  nbr[e] = j;
  if (j >= 0) {
    tkey[e] = ((unsigned long long)(unsigned)j << 32) | (unsigned)s;
    atomicAdd(&count[j], 1);
  } else {
    tkey[e] = ~0ULL;
  }
  tval[e] = (int32_t)e;
}

__global__ void unpack_transpose_kernel(int64_t nnz, const unsigned long long* __restrict__ key,
                                        int32_t* __restrict__ colT) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) colT[p] = (int32_t)(key[p] & 0xffffffffULL);
}

__global__ void gather_vals_kernel(int64_t nnz, const int32_t* __restrict__ permT, const double* __restrict__ A64,
                                   double* __restrict__ valT64, float* __restrict__ valT32, int64_t nm,
                                   float* __restrict__ A32) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nnz) {
    double a = A64[permT[p]];
    valT64[p] = a;
    valT32[p] = (float)a;
  }
  if (p < nm) A32[p] = (float)A64[p];
}

__global__ void levels_fwd_kernel(int n, int m, const int32_t* __restrict__ nbr, const int32_t* __restrict__ v2s,
                                  int* lev, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int k = warp; k < n; k += nw) {
    const int s = v2s[k];
    int mx = -1;
    for (int c = lane; c < m; c += 32) {
      const int j = nbr[(int64_t)s * m + c];
      if (j >= 0) {
        int v = -1;
        bounded_wait([&] { v = ld_acquire(&lev[j]); return v >= 0; }, st, k);
        mx = max(mx, v);
      }
    }
    mx = warp_max(mx);
    if (lane == 0) st_release(&lev[s], mx + 1);
  }
}

__global__ void levels_bwd_kernel(int n, const int32_t* __restrict__ rowptrT, const int32_t* __restrict__ colT,
                                  const int32_t* __restrict__ v2s, int* levT, DevStatus* st) {
  const int lane = threadIdx.x & 31;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int kk = warp; kk < n; kk += nw) {
    const int s = v2s[n - 1 - kk];
    int mx = -1;
    for (int e = rowptrT[s] + lane; e < rowptrT[s + 1]; e += 32) {
      const int i = colT[e];
      int v = -1;
      bounded_wait([&] { v = ld_acquire(&levT[i]); return v >= 0; }, st, n - 1 - kk);
      mx = max(mx, v);
    }
    mx = warp_max(mx);
    if (lane == 0) st_release(&levT[s], mx + 1);
  }
}

// work[lev(s)] += number of dependencies of row s
__global__ void level_work_kernel(int n, int m, const int* __restrict__ lev, const int32_t* __restrict__ nbr,
                                  const int32_t* __restrict__ rowptrT, unsigned long long* __restrict__ work) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int d = 0;
  if (nbr) {
    for (int c = 0; c < m; ++c) d += nbr[(int64_t)s * m + c] >= 0;
  } else {
    d = rowptrT[s + 1] - rowptrT[s];
  }
  atomicAdd(&work[lev[s]], (unsigned long long)d);
}

// Sort key (level, light, s): inside a level, rows with more than kHeavyDeps
// dependencies come first (the solve gives each of them a whole block).
constexpr int kHeavyDeps = 48;

__device__ __forceinline__ int row_deps(int s, int m, const int32_t* nbr, const int32_t* rowptrT) {
  if (nbr) {
    int d = 0;
    for (int c = 0; c < m; ++c) d += nbr[(int64_t)s * m + c] >= 0;
    return d;
  }
  return rowptrT[s + 1] - rowptrT[s];
}

__global__ void level_keys_kernel(int n, int m, const int* __restrict__ lev, const int32_t* __restrict__ nbr,
                                  const int32_t* __restrict__ rowptrT, unsigned long long* __restrict__ key,
                                  unsigned* __restrict__ hcnt) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const bool heavy = row_deps(s, m, nbr, rowptrT) > kHeavyDeps;
  key[s] = ((unsigned long long)(unsigned)lev[s] << 32) | ((unsigned long long)(heavy ? 0u : 1u) << 31) | (unsigned)s;
  if (heavy) atomicAdd(&hcnt[lev[s]], 1u);
}

__global__ void unpack_tasks_kernel(int n, const unsigned long long* __restrict__ key, int32_t* __restrict__ task,
                                    int32_t* __restrict__ lptr) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  task[p] = (int32_t)(key[p] & 0x7fffffffULL);
  const int l = (int)(key[p] >> 32);
  // levels are dense (0..nlev-1), so each level starts where the key's level changes
  if (p == 0 || (int)(key[p - 1] >> 32) != l) lptr[l] = p;
  if (p == n - 1) lptr[l + 1] = n;
}

namespace {
struct Scratch {
  Ctx* c;
  std::vector<void*> blocks;
  void* get(size_t b) {
    void* p = c->arena.alloc(b + 16);
    if (p) blocks.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void* p : blocks) c->arena.release(p);
  }
};

vl_status launch_coop(Ctx* c, const void* fn, int want_blocks, int block, void** args) {
  int maxb = resident_blocks(c, fn, block, 0);
  int grid = std::max(1, std::min(want_blocks, maxb));
  ++c->launches;
    VL_CUDA(c, cudaLaunchCooperativeKernel(fn, grid, block, args, 0, c->stream));
  return VL_OK;
}

vl_status task_order(Ctx* c, Scratch& S, int n, int m, const int* lev, const int32_t* nbr, const int32_t* rowptrT,
                     int32_t* task, int* nlev, int32_t** lptr, std::vector<int32_t>& h_lptr, int32_t** hptr,
                     std::vector<int32_t>& h_hptr, Owned& own) {
  auto* k1 = (unsigned long long*)S.get(sizeof(unsigned long long) * n);
  auto* k2 = (unsigned long long*)S.get(sizeof(unsigned long long) * n);
  auto* hc = (unsigned*)S.get(sizeof(unsigned) * (n + 1));
  if (!k1 || !k2 || !hc) return fail(c, VL_ERR_OOM, "workspace exhausted (task order)");
  const int T = 256;
  VL_CUDA(c, cudaMemsetAsync(hc, 0, sizeof(unsigned) * (n + 1), c->stream));
  level_keys_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(n, m, lev, nbr, rowptrT, k1, hc);
  VL_CUDA(c, cudaGetLastError());
  size_t tb = 0;
  cub::DeviceRadixSort::SortKeys(nullptr, tb, k1, k2, n, 0, 64, c->stream);
  void* tmp = S.get(tb);
  if (!tmp) return fail(c, VL_ERR_OOM, "workspace exhausted (task sort)");
  VL_CUDA(c, cub::DeviceRadixSort::SortKeys(tmp, tb, k1, k2, n, 0, 64, c->stream));
  unsigned long long last = 0;
  VL_CUDA(c, cudaMemcpyAsync(&last, k2 + (n - 1), sizeof(last), cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  *nlev = (int)(last >> 32) + 1;
  *lptr = own.get<int32_t>(*nlev + 1);
  if (!*lptr) return fail(c, VL_ERR_OOM, "workspace exhausted (level pointers)");
  unpack_tasks_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(n, k2, task, *lptr);
  VL_CUDA(c, cudaGetLastError());
  h_lptr.resize(*nlev + 1);
  std::vector<unsigned> h_hc(*nlev);
  VL_CUDA(c, cudaMemcpyAsync(h_lptr.data(), *lptr, sizeof(int32_t) * (*nlev + 1), cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaMemcpyAsync(h_hc.data(), hc, sizeof(unsigned) * (*nlev), cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  // hptr[l] = end of the heavy rows of level l (they lead the level)
  h_hptr.resize(*nlev);
  for (int l = 0; l < *nlev; ++l) h_hptr[l] = h_lptr[l] + (int32_t)h_hc[l];
  *hptr = own.get<int32_t>(*nlev);
  if (!*hptr) return fail(c, VL_ERR_OOM, "workspace exhausted (level pointers)");
  VL_CUDA(c, cudaMemcpyAsync(*hptr, h_hptr.data(), sizeof(int32_t) * (*nlev), cudaMemcpyHostToDevice, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}
}  // namespace

// Builds storage maps, ELL neighbours, transpose pattern, levels and task orders
// from the Vecchia-order neighbour table N_v (device, n x m) and the Vecchia-order
// locations already in f->locs_s (overwritten with storage-order locations).
vl_status build_graph_impl(Factor* f, const int32_t* N_v, const double* locs_v, const int32_t* order_dev) {
  Ctx* c = f->ctx;
  const int n = (int)f->n, m = f->m;
  const int64_t nm = (int64_t)n * m;
  Scratch S{c};
  int32_t* perm = (int32_t*)S.get(sizeof(int32_t) * n);
  if (!perm) return fail(c, VL_ERR_OOM, "workspace exhausted (graph)");
  VL_TRY(morton_perm(c, locs_v, n, perm));
  const int T = 256;
  storage_maps_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(n, m, perm, order_dev, locs_v, f->s2v, f->v2s, f->s2u,
                                                              f->u2s, f->locs_s);
  VL_CUDA(c, cudaGetLastError());
  f->nnz = 0;
  for (int64_t k = 0; k < n; ++k) f->nnz += std::min<int64_t>(k, m);   // |N(k)| = min(k, m)
  const int64_t nnz = f->nnz;
  f->rowptrT = f->mem.get<int32_t>(n + 1);
  f->colT = f->mem.get<int32_t>(std::max<int64_t>(nnz, 1));
  f->permT = f->mem.get<int32_t>(std::max<int64_t>(nnz, 1));
  f->valT64 = f->mem.get<double>(std::max<int64_t>(nnz, 1));
  f->valT32 = f->mem.get<float>(std::max<int64_t>(nnz, 1));
  if (!f->rowptrT || !f->colT || !f->permT || !f->valT64 || !f->valT32)
    return fail(c, VL_ERR_OOM, "workspace exhausted (transpose)");
  int32_t* count = (int32_t*)S.get(sizeof(int32_t) * (n + 1));
  if (!count) return fail(c, VL_ERR_OOM, "workspace exhausted (graph)");
  VL_CUDA(c, cudaMemsetAsync(count, 0, sizeof(int32_t) * (n + 1), c->stream));
  if (m > 0) {
    auto* tk = (unsigned long long*)S.get(sizeof(unsigned long long) * nm);
    auto* tk2 = (unsigned long long*)S.get(sizeof(unsigned long long) * nm);
    int32_t* tv = (int32_t*)S.get(sizeof(int32_t) * nm);
    int32_t* tv2 = (int32_t*)S.get(sizeof(int32_t) * nm);
    if (!tk || !tk2 || !tv || !tv2) return fail(c, VL_ERR_OOM, "workspace exhausted (transpose sort)");
    translate_nbr_kernel<<<(int)((nm + T - 1) / T), T, 0, VL_STREAM(c)>>>(n, m, f->s2v, f->v2s, N_v, f->nbr, tk, tv,
                                                                        count);
    VL_CUDA(c, cudaGetLastError());
    size_t tb = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tb, tk, tk2, tv, tv2, (int)nm, 0, 64, c->stream);
    void* tmp = S.get(tb);
    if (!tmp) return fail(c, VL_ERR_OOM, "workspace exhausted (transpose sort)");
    VL_CUDA(c, cub::DeviceRadixSort::SortPairs(tmp, tb, tk, tk2, tv, tv2, (int)nm, 0, 64, c->stream));
    if (nnz > 0) {
      unpack_transpose_kernel<<<(int)((nnz + T - 1) / T), T, 0, VL_STREAM(c)>>>(nnz, tk2, f->colT);
      VL_CUDA(c, cudaMemcpyAsync(f->permT, tv2, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, c->stream));
    }
  }
  {
    size_t tb = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, count, f->rowptrT, n + 1, c->stream);
    void* tmp = S.get(tb);
    if (!tmp) return fail(c, VL_ERR_OOM, "workspace exhausted (scan)");
    VL_CUDA(c, cub::DeviceScan::ExclusiveSum(tmp, tb, count, f->rowptrT, n + 1, c->stream));
  }
  // levels
  VL_CUDA(c, cudaMemsetAsync(f->lev_fwd, 0xff, sizeof(int) * n, c->stream));
  VL_CUDA(c, cudaMemsetAsync(f->lev_bwd, 0xff, sizeof(int) * n, c->stream));
  VL_CUDA(c, status_clear(c));
  {
    int nn = n, mm = m;
    const int32_t* a1 = f->nbr;
    const int32_t* a2 = f->v2s;
    int* a3 = f->lev_fwd;
    DevStatus* a4 = c->dstatus;
    void* args[] = {&nn, &mm, &a1, &a2, &a3, &a4};
    VL_TRY(launch_coop(c, (const void*)levels_fwd_kernel, (n + 7) / 8, 256, args));
  }
  {
    int nn = n;
    const int32_t* a1 = f->rowptrT;
    const int32_t* a2 = f->colT;
    const int32_t* a3 = f->v2s;
    int* a4 = f->lev_bwd;
    DevStatus* a5 = c->dstatus;
    void* args[] = {&nn, &a1, &a2, &a3, &a4, &a5};
    VL_TRY(launch_coop(c, (const void*)levels_bwd_kernel, (n + 7) / 8, 256, args));
  }
  VL_TRY(check_dev_status(c, "level schedule"));
  VL_TRY(task_order(c, S, n, m, f->lev_fwd, f->nbr, nullptr, f->task_fwd, &f->nlev_fwd, &f->lptr_fwd, f->h_lptr_fwd,
                    &f->hptr_fwd, f->h_hptr_fwd, f->mem));
  VL_TRY(task_order(c, S, n, m, f->lev_bwd, nullptr, f->rowptrT, f->task_bwd, &f->nlev_bwd, &f->lptr_bwd,
                    f->h_lptr_bwd, &f->hptr_bwd, f->h_hptr_bwd, f->mem));
  for (int dir = 0; dir < 2; ++dir) {
    const int nl = dir == 0 ? f->nlev_fwd : f->nlev_bwd;
    auto* w = (unsigned long long*)S.get(sizeof(unsigned long long) * nl);
    if (!w) return fail(c, VL_ERR_OOM, "workspace exhausted (level work)");
    VL_CUDA(c, cudaMemsetAsync(w, 0, sizeof(unsigned long long) * nl, c->stream));
    level_work_kernel<<<(n + T - 1) / T, T, 0, VL_STREAM(c)>>>(n, m, dir == 0 ? f->lev_fwd : f->lev_bwd,
                                                              dir == 0 ? f->nbr : nullptr, f->rowptrT, w);
    VL_CUDA(c, cudaGetLastError());
    std::vector<int64_t>& hw = dir == 0 ? f->h_lwork_fwd : f->h_lwork_bwd;
    hw.resize(nl);
    VL_CUDA(c, cudaMemcpyAsync(hw.data(), w, sizeof(int64_t) * nl, cudaMemcpyDeviceToHost, c->stream));
  }
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status refresh_transpose_values(Factor* f) {
  Ctx* c = f->ctx;
  const int64_t nm = f->n * (int64_t)f->m;
  const int64_t work = std::max<int64_t>(std::max<int64_t>(f->nnz, nm), 1);
  const int T = 256;
  gather_vals_kernel<<<(int)((work + T - 1) / T), T, 0, VL_STREAM(c)>>>(f->nnz, f->permT, f->A64, f->valT64,
                                                                     f->valT32, nm, f->A32);
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

}  // namespace vl
