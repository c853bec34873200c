// Krylov engine: the operators of Eqs. pcls1/pcls2 and the preconditioners of
// Section 3.1 on a block of t right-hand sides, and the PCG loop of the appendix
// algorithm with per-column freezing and Lanczos T extraction.
#pragma once

#include "tile_plan.h"
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "lrac_tc.cuh"

namespace vl {

struct Scratch {
  Ctx* c = nullptr;
  std::vector<void*> blocks;
  explicit Scratch(Ctx* ctx) : c(ctx) {}
  Scratch(const Scratch&) = delete;
  template <typename T>
  T* get(size_t count) {
    void* p = c->arena.alloc(count * sizeof(T) + 16);
    if (p) blocks.push_back(p);
    return static_cast<T*>(p);
  }
  ~Scratch() {
    for (void* p : blocks) c->arena.release(p);
  }
};

// ----------------------------------------------------------------------------- small kernels
template <typename T>
__global__ void diag_prep_kernel(int n, int prec, const double* __restrict__ W, const double* __restrict__ D,
                                 T* __restrict__ Wt, T* __restrict__ Dinv, T* __restrict__ dsc, T* __restrict__ Dt,
                                 T* __restrict__ Winv) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double w = W ? W[s] : 0.0, d = D[s];
    Wt[s] = (T)w;
    Dinv[s] = (T)(1.0 / d);
    Dt[s] = (T)d;
    // VADU: (W + D^{-1})^{-1}; LVA: D; LRAC uses W^{-1} and Sigma_tilde = B^{-1} D B^{-T}
    dsc[s] = (prec == VL_PREC_VADU) ? (T)(1.0 / (w + 1.0 / d)) : (T)d;
    Winv[s] = (T)(W ? 1.0 / w : 0.0);
  }
}

template <typename T>
__global__ void fill_kernel(int64_t total, T v, T* __restrict__ x) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    x[e] = v;
}

// Z = Y + w o X  (row scale)
template <typename T>
__global__ void add_diag_kernel(int n, int t, int ld, const T* __restrict__ Y, const T* __restrict__ w,
                                const T* __restrict__ X, T* __restrict__ Z) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    if (c < t) Z[e] = Y[e] + w[s] * X[e];
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(int64_t total, const TI* __restrict__ a, TO* __restrict__ b) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = (TO)a[e];
}

// x += y (mixed types)
template <typename TX, typename TY>
__global__ void accumulate_kernel(int64_t total, TX* __restrict__ x, const TY* __restrict__ y) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    x[e] += (TX)y[e];
}

// r = b - r (in place on r holding A x)
static __global__ void residual_kernel(int64_t total, const double* __restrict__ b, double* __restrict__ r) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    r[e] = b[e] - r[e];
}

// Calls f(LPV, NV, UNR) (as integral constants) for the row-gather shape that
// covers ld columns: LPV lanes per row, NV vector words per lane, UNR dependency
// rows in flight per lane.
template <typename T, typename F>
vl_status with_shape(int ld, F&& f) {
  using I8 = std::integral_constant<int, 8>;
  using I16 = std::integral_constant<int, 16>;
  using I32 = std::integral_constant<int, 32>;
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  using I4 = std::integral_constant<int, 4>;
  const int nvec = ld / VecT<T>::n;
  if (nvec <= 8) return f(I8{}, I1{}, I8{});
  if (nvec <= 16) return f(I16{}, I1{}, I8{});
  if (nvec <= 32) return f(I32{}, I1{}, I8{});
  if (nvec <= 64) return f(I32{}, I2{}, I4{});
  return f(I32{}, I4{}, I2{});
}

// Sets a kernel's dynamic shared-memory limit once per device (the value is the
// kernel's fixed maximum, so repeating it would only cost a driver call per launch).
inline vl_status smem_limit_once(Ctx* c, const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({c->device, fn})) return VL_OK;
  VL_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  done.insert({c->device, fn});
  return VL_OK;
}

// Largest system the t = 1 solve keeps in shared memory (one block).
constexpr size_t kSmemSolveBytes = 200 * 1024;

// A triangular solve runs in one thread-block cluster (hardware cluster barrier,
// part of the device) rather than on the whole grid (software grid barrier) while
// the widest level needs at most this many rounds of the largest cluster's teams.
// Problems up to kSharedRows rows are the ones served side by side (batched and
// serving forms): for them the cluster is kept even for wide levels, since a grid
// solve needs the whole device; measured on the serving mix this raised throughput
// by half. Larger problems usually own the device, where the grid solve is faster.
constexpr int64_t kSharedRows = 262144;
#ifndef VL_T1_CLUSTER_ROUNDS
#define VL_T1_CLUSTER_ROUNDS 8
#endif
#ifndef VL_BLOCK_CLUSTER_ROUNDS
#define VL_BLOCK_CLUSTER_ROUNDS 4
#endif
#ifndef VL_SHARED_CLUSTER_ROUNDS
#define VL_SHARED_CLUSTER_ROUNDS 32
#endif

inline vl_status cuda_ok(Ctx* c, cudaError_t e) { return e == cudaSuccess ? VL_OK : cuda_fail(c, e, "kernel launch"); }

inline int grid_for(Ctx* c, int64_t work, int block = 256) {
  int64_t g = (work + block - 1) / block;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)c->num_sms * 16));
}

// Heavy rows (task[lptr[l] .. hptr[l])) of the levels that have more of them than
// min_rows, cut into chunks of at most ch dependencies, with level-local partial slots and
// row counters (see HeavyChunk); other levels keep a whole block per heavy row. Built once
// per factor, direction and chunk size from host copies of the task list and row lengths.
inline vl_status chunk_plan(Ctx* c, Factor* f, bool fwd, int ch, const Factor::ChunkPlan** out) {
  auto key = std::make_pair(fwd ? 1 : 0, ch);
  auto it = f->chunk_plans.find(key);
  if (it != f->chunk_plans.end()) {
    *out = &it->second;
    return VL_OK;
  }
  const int n = (int)f->n, m = f->m;
  const int min_rows = 4 * c->num_sms;   // about two rounds of the grid's blocks
  const std::vector<int32_t>& lp = fwd ? f->h_lptr_fwd : f->h_lptr_bwd;
  const std::vector<int32_t>& hp = fwd ? f->h_hptr_fwd : f->h_hptr_bwd;
  const int nlev = (int)lp.size() - 1;
  int64_t nheavy = 0;
  for (int l = 0; l < nlev; ++l) nheavy += hp[l] - lp[l];
  std::vector<HeavyChunk> items;
  std::vector<int32_t> cptr(nlev + 1, 0);
  Factor::ChunkPlan plan;
  if (nheavy > 0) {
    // heavy rows are at most a few percent of the rows: copy only what is needed
    std::vector<int32_t> task(n), rp;
    VL_CUDA(c, cudaMemcpyAsync(task.data(), fwd ? f->task_fwd : f->task_bwd, sizeof(int32_t) * n,
                               cudaMemcpyDeviceToHost, c->stream));
    if (!fwd) {
      rp.resize(n + 1);
      VL_CUDA(c, cudaMemcpyAsync(rp.data(), f->rowptrT, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int l = 0; l < nlev; ++l) {
      cptr[l] = (int32_t)items.size();
      int slot = 0, row = 0;
      if (hp[l] - lp[l] <= min_rows) continue;
      for (int p = lp[l]; p < hp[l]; ++p, ++row) {
        const int s = task[p];
        const int beg = fwd ? s * m : rp[s], end = fwd ? s * m + m : rp[s + 1];
        const int nch = std::max(1, (end - beg + ch - 1) / ch);
        for (int k = 0; k < nch; ++k)
          items.push_back(HeavyChunk{p, beg + k * ch, std::min(end, beg + (k + 1) * ch), slot + k, slot, nch, row, 0});
        slot += nch;
      }
      plan.max_slots = std::max(plan.max_slots, slot);
      plan.max_rows = std::max(plan.max_rows, row);
    }
  }
  cptr[nlev] = (int32_t)items.size();
  plan.cptr = f->mem.get<int32_t>(nlev + 1);
  plan.chunk = f->mem.get<HeavyChunk>(std::max<size_t>(items.size(), 1));
  if (!plan.cptr || !plan.chunk) return fail(c, VL_ERR_OOM, "workspace exhausted (heavy-row chunks)");
  VL_CUDA(c, cudaMemcpyAsync(plan.cptr, cptr.data(), sizeof(int32_t) * (nlev + 1), cudaMemcpyHostToDevice, c->stream));
  if (!items.empty())
    VL_CUDA(c, cudaMemcpyAsync(plan.chunk, items.data(), sizeof(HeavyChunk) * items.size(), cudaMemcpyHostToDevice,
                               c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = &(f->chunk_plans[key] = plan);
  return VL_OK;
}

// out[p * m + c] = nbr[task[p] * m + c] for the first `rows` task positions
static __global__ void head_nbr_kernel(int rows, int m, const int32_t* __restrict__ task, const int32_t* __restrict__ nbr,
                                       int32_t* __restrict__ out) {
  const int64_t total = (int64_t)rows * m;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / m), c = (int)(e % m);
    out[e] = nbr[(int64_t)task[p] * m + c];
  }
}

// Dependencies of the forward head's rows (levels [0, l_head)) as task positions; unusable if a
// dependency lay outside the head (it cannot: a row depends only on rows of earlier levels).
// Plan of the tiled solve in one direction over G tiles (tile_plan.h), built on the host from
// the task list and the dependency lists, and kept on the device.
inline vl_status tile_plan(Ctx* c, Factor* f, bool fwd, int G, int first, const Factor::TilePlan** out) {
  const std::tuple<int, int, int> key{fwd ? 1 : 0, G, first};
  auto it = f->tile_plans.find(key);
  if (it != f->tile_plans.end()) {
    *out = &it->second;
    return VL_OK;
  }
  const int n = (int)f->n, m = f->m;
  std::vector<int32_t> task(n), nbr, rp, col;
  VL_CUDA(c, cudaMemcpyAsync(task.data(), fwd ? f->task_fwd : f->task_bwd, sizeof(int32_t) * n,
                             cudaMemcpyDeviceToHost, c->stream));
  if (fwd) {
    nbr.resize((size_t)n * m);
    if (m > 0)
      VL_CUDA(c, cudaMemcpyAsync(nbr.data(), f->nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, c->stream));
  } else {
    rp.resize(n + 1);
    col.resize(std::max<int64_t>(f->nnz, 1));
    VL_CUDA(c, cudaMemcpyAsync(rp.data(), f->rowptrT, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, c->stream));
    if (f->nnz > 0)
      VL_CUDA(c, cudaMemcpyAsync(col.data(), f->colT, sizeof(int32_t) * f->nnz, cudaMemcpyDeviceToHost, c->stream));
  }
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  const TilePlanHost H = build_tile_plan(n, G, task.data(), m, fwd ? nbr.data() : nullptr,
                                         fwd ? nullptr : rp.data(), fwd ? nullptr : col.data(), first);
  Factor::TilePlan plan;
  plan.G = G;
  plan.R = H.R;
  auto up = [&](const void* h, size_t bytes, void** d) -> vl_status {
    *d = f->mem.get<uint8_t>(std::max<size_t>(bytes, 16));
    if (!*d) return fail(c, VL_ERR_OOM, "workspace exhausted (tile plan)");
    if (bytes) VL_CUDA(c, cudaMemcpyAsync(*d, h, bytes, cudaMemcpyHostToDevice, c->stream));
    return VL_OK;
  };
  VL_TRY(up(H.ttask.data(), sizeof(int32_t) * H.ttask.size(), (void**)&plan.ttask));
  VL_TRY(up(H.toff.data(), sizeof(int32_t) * H.toff.size(), (void**)&plan.toff));
  VL_TRY(up(H.exported.data(), H.exported.size(), (void**)&plan.exported));
  plan.flag = f->mem.get<int>(std::max(n, 1));
  if (!plan.flag) return fail(c, VL_ERR_OOM, "workspace exhausted (tile plan)");
  VL_CUDA(c, cudaMemsetAsync(plan.flag, 0, sizeof(int) * std::max(n, 1), c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  *out = &(f->tile_plans[key] = plan);
  return VL_OK;
}

// Shared memory a staged product block uses for its rows (two blocks of 256 threads per SM).
constexpr size_t kHaloBytes = 96 * 1024;

// Plan of the staged products in one direction for rows of row_bytes bytes (build_halo_plan).
inline vl_status halo_plan(Ctx* c, Factor* f, bool fwd, int row_bytes, const Factor::HaloPlan** out) {
  const std::pair<int, int> key{fwd ? 1 : 0, row_bytes};
  auto it = f->halo_plans.find(key);
  if (it != f->halo_plans.end()) {
    *out = &it->second;
    return VL_OK;
  }
  const int n = (int)f->n, m = f->m;
  std::vector<int32_t> nbr, rp, col;
  if (fwd) {
    nbr.resize((size_t)n * m);
    if (m > 0)
      VL_CUDA(c, cudaMemcpyAsync(nbr.data(), f->nbr, sizeof(int32_t) * nbr.size(), cudaMemcpyDeviceToHost, c->stream));
  } else {
    rp.resize(n + 1);
    col.resize(std::max<int64_t>(f->nnz, 1));
    VL_CUDA(c, cudaMemcpyAsync(rp.data(), f->rowptrT, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost, c->stream));
    if (f->nnz > 0)
      VL_CUDA(c, cudaMemcpyAsync(col.data(), f->colT, sizeof(int32_t) * f->nnz, cudaMemcpyDeviceToHost, c->stream));
  }
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  Factor::HaloPlan plan;
  plan.ucap = std::min<int>(65535, (int)(kHaloBytes / row_bytes));
  const HaloPlanHost H = build_halo_plan(n, m, fwd ? nbr.data() : nullptr, fwd ? nullptr : rp.data(),
                                         fwd ? nullptr : col.data(), plan.ucap, 512);
  if (H.ok && n > 0) {
    plan.nb = (int)H.brow.size() - 1;
    auto up = [&](const void* h, size_t bytes, void** d) -> vl_status {
      *d = f->mem.get<uint8_t>(std::max<size_t>(bytes, 16));
      if (!*d) return fail(c, VL_ERR_OOM, "workspace exhausted (staged product plan)");
      if (bytes) VL_CUDA(c, cudaMemcpyAsync(*d, h, bytes, cudaMemcpyHostToDevice, c->stream));
      return VL_OK;
    };
    VL_TRY(up(H.brow.data(), sizeof(int32_t) * H.brow.size(), (void**)&plan.brow));
    VL_TRY(up(H.uoff.data(), sizeof(int32_t) * H.uoff.size(), (void**)&plan.uoff));
    VL_TRY(up(H.ulist.data(), sizeof(int32_t) * H.ulist.size(), (void**)&plan.ulist));
    VL_TRY(up(H.lidx.data(), sizeof(uint16_t) * H.lidx.size(), (void**)&plan.lidx));
    VL_TRY(up(H.lself.data(), sizeof(uint16_t) * H.lself.size(), (void**)&plan.lself));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    plan.usable = true;
  }
  *out = &(f->halo_plans[key] = plan);
  return VL_OK;
}

inline vl_status head_plan(Ctx* c, Factor* f, int l_head, const Factor::HeadPlan** out) {
  auto it = f->head_plans.find(l_head);
  if (it != f->head_plans.end()) {
    *out = &it->second;
    return VL_OK;
  }
  Factor::HeadPlan plan;
  const int H = f->h_lptr_fwd[l_head], m = f->m;
  plan.rows = H;
  if (H > 0 && m > 0) {
    Scratch S(c);
    int32_t* dn = S.get<int32_t>((size_t)H * m);
    if (!dn) return fail(c, VL_ERR_OOM, "workspace exhausted (head plan)");
    head_nbr_kernel<<<grid_for(c, (int64_t)H * m), 256, 0, VL_STREAM(c)>>>(H, m, f->task_fwd, f->nbr, dn);
    VL_CUDA(c, cudaGetLastError());
    std::vector<int32_t> hn((size_t)H * m), task(H);
    VL_CUDA(c, cudaMemcpyAsync(hn.data(), dn, sizeof(int32_t) * hn.size(), cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(task.data(), f->task_fwd, sizeof(int32_t) * H, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    std::map<int32_t, int32_t> pos;
    for (int p = 0; p < H; ++p) pos[task[p]] = p;
    bool ok = true;
    for (int32_t& j : hn) {
      if (j < 0) continue;
      auto q = pos.find(j);
      if (q == pos.end()) {
        ok = false;
        break;
      }
      j = q->second;
    }
    if (ok) {
      plan.hpos = f->mem.get<int32_t>(hn.size());
      if (!plan.hpos) return fail(c, VL_ERR_OOM, "workspace exhausted (head plan)");
      VL_CUDA(c, cudaMemcpyAsync(plan.hpos, hn.data(), sizeof(int32_t) * hn.size(), cudaMemcpyHostToDevice, c->stream));
      VL_CUDA(c, cudaStreamSynchronize(c->stream));
      plan.usable = true;
    }
  }
  *out = &(f->head_plans[l_head] = plan);
  return VL_OK;
}

// ----------------------------------------------------------------------------- launch tuner
// Launch parameters that do not change any result (blocks per SM of a grid solve, dependency
// rows in flight per lane, lanes per row of a block product) are tuned at first use: every
// candidate is run on the live call and timed with CUDA events, and the fastest is kept for
// later calls of the same key (kernel class and direction, value size, row width, size bucket).
struct TuneKey {
  int device, cls, vbytes, ld, nbucket;
  bool operator<(const TuneKey& o) const {
    return std::tie(device, cls, vbytes, ld, nbucket) < std::tie(o.device, o.cls, o.vbytes, o.ld, o.nbucket);
  }
};

inline int log2_bucket(int64_t n) {
  int b = 0;
  while ((1LL << (b + 1)) <= n) ++b;
  return b;
}

struct Tuner {
  std::mutex mu;
  std::map<TuneKey, int> best;          // key -> candidate
  std::map<TuneKey, std::vector<float>> times;
};
inline Tuner& tuner() {
  static Tuner t;
  return t;
}

// Runs candidate `best` of key (tuning it first when the context allows and no choice is
// cached): run(cand) launches candidate cand on the context's stream.
template <typename Run>
vl_status tuned_call(Ctx* c, const TuneKey& key, int ncand, Run run) {
  if (!c->autotune || ncand < 2) return run(0);   // the defaults
  int choice = -1;
  {
    std::lock_guard<std::mutex> lk(tuner().mu);
    auto it = tuner().best.find(key);
    if (it != tuner().best.end()) choice = it->second;
  }
  if (choice >= 0) return run(choice);
  cudaEvent_t a = nullptr, b = nullptr;
  VL_CUDA(c, cudaEventCreate(&a));
  VL_CUDA(c, cudaEventCreate(&b));
  // one untimed run first (first-use work such as building a solve's chunk plan must not
  // count against a candidate), then the best of two timed runs of each candidate
  vl_status st = run(0);
  std::vector<float> ms(ncand, 0.f);
  for (int k = 0; k < ncand && st == VL_OK; ++k) {
    float best = 0.f;
    for (int rep = 0; rep < 2 && st == VL_OK; ++rep) {
      cudaEventRecord(a, c->stream);
      st = run(k);
      cudaEventRecord(b, c->stream);
      if (cudaEventSynchronize(b) != cudaSuccess) st = cuda_fail(c, cudaGetLastError(), "tuning");
      float x = 0.f;
      cudaEventElapsedTime(&x, a, b);
      best = rep == 0 ? x : std::min(best, x);
    }
    ms[k] = best;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  VL_TRY(st);
  const int pick = (int)(std::min_element(ms.begin(), ms.end()) - ms.begin());
  {
    std::lock_guard<std::mutex> lk(tuner().mu);
    tuner().best[key] = pick;
    tuner().times[key] = ms;
  }
  // every candidate computed the same result; the last run stands
  return VL_OK;
}

// ----------------------------------------------------------------------------- engine
template <typename T>
struct Engine {
  Ctx* c = nullptr;
  Factor* f = nullptr;
  int n = 0, m = 0, t = 0, ld = 0, prec = VL_PREC_VADU;
  Scratch mem;
  const T* Aval = nullptr;
  const T* valT = nullptr;
  T *W = nullptr, *Dinv = nullptr, *dsc = nullptr, *Dt = nullptr, *Winv = nullptr;
  T *u = nullptr, *r = nullptr, *z = nullptr, *h = nullptr, *v = nullptr, *y = nullptr, *sv = nullptr;
  double *partial = nullptr, *red = nullptr, *red2 = nullptr;
  int nblk = 1, rpb = 1;
  int nseg = 1, ncol = 1;          // segments (problems of a batch) and nseg * t scalar columns
  BlockRows br{};                  // reduction blocks (segment-aligned)
  std::vector<int32_t> h_blk_seg;  // segment of each reduction block (batches; empty: all 0)
  unsigned* done = nullptr;        // arrival counter of the fused reductions
  dim3 cb;
  size_t csh = 0;
  PcgScalars S{};
  int lmax = 0;
  int* d_count = nullptr;
  int* h_count = nullptr;
  // LRAC (Section 3.1.2): L (factor-owned), C = I + L^T W L, its Cholesky factor,
  // R^{-1} and C^{-1} (rebuilt lazily after W changes), the rank-k blocks of one apply
  int kr = 0;
  const T* Lk = nullptr;
  double *Cm = nullptr, *Rinv = nullptr, *Cinv = nullptr, *lpart = nullptr, *Gk = nullptr, *Vk = nullptr;
  double* dlogdet = nullptr;
  int* lbad = nullptr;
  int nch_g = 1, rows_g = 0, nch_a = 1, rows_a = 0, nch_tc = 1, rows_tc = 0;
  bool use_tc = false;   // float32 blocks of 2..64 columns with k <= 512: tensor-core products
  float* Vt = nullptr;   // split image of V for the tensor-core product
  bool lr_dirty = true;
  double logdetC = 0.0;
  T* b2 = nullptr;
  // partial rows and row counters of the heavy-row chunks (grid solves), grown on demand
  T* chunk_part = nullptr;
  int* chunk_cnt = nullptr;
  int part_slots = 0, cnt_len = 0;

  explicit Engine(Ctx* ctx) : c(ctx), mem(ctx) {}

  template <typename Run>
  vl_status tuned(const TuneKey& key, int ncand, Run run) {
    return tuned_call(c, key, ncand, run);
  }

  // Whether cooperative launches in thread-block clusters are accepted on this process
  // (cleared after the first refusal).
  static bool& cluster_grid_ok() {
    static bool ok = true;
    return ok;
  }
  // Most clusters of csize blocks (config cfg) co-resident, cached per (device, kernel, smem).
  int cluster_capacity(const void* fn, const cudaLaunchConfig_t& cfg, int csize) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t, int>, int> cache;
    const auto key = std::make_tuple(c->device, fn, cfg.dynamicSmemBytes, csize);
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) return it->second;
    }
    cudaLaunchConfig_t q = cfg;
    q.gridDim = dim3(csize);
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, fn, &q) != cudaSuccess) {
      cudaGetLastError();
      ncl = 0;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = ncl;
    return ncl;
  }

  // Heavy-row chunk plan of a grid solve, with partial slots and zeroed counters.
  vl_status chunk_setup(bool fwd, int ch, LevelPlan& L) {
    const Factor::ChunkPlan* pl = nullptr;
    VL_TRY(chunk_plan(c, f, fwd, ch, &pl));
    const int w = t == 1 ? 1 : ld;
    if (pl->max_slots > part_slots) {
      chunk_part = mem.get<T>((size_t)pl->max_slots * w);
      if (!chunk_part) return fail(c, VL_ERR_OOM, "workspace exhausted (heavy-row partials)");
      part_slots = pl->max_slots;
    }
    if (pl->max_rows > cnt_len) {
      chunk_cnt = mem.get<int>(pl->max_rows);
      if (!chunk_cnt) return fail(c, VL_ERR_OOM, "workspace exhausted (heavy-row counters)");
      cnt_len = pl->max_rows;
    }
    if (cnt_len > 0) VL_CUDA(c, cudaMemsetAsync(chunk_cnt, 0, sizeof(int) * cnt_len, c->stream));
    L.chunk = static_cast<const HeavyChunk*>(pl->chunk);
    L.cptr = pl->cptr;
    L.part = chunk_part;
    L.cnt = chunk_cnt;
    return VL_OK;
  }

  // Leading dimension: 1 for a single column, else a multiple of 8 (the same for
  // float32 and float64 blocks, so mixed-precision refinement converts in place).
  static int lead(int t_) { return t_ == 1 ? 1 : (t_ + 7) / 8 * 8; }

  // ops_only: only the operators (opA, opA2, opSigma, opB, opBt, coldot) are used, so only
  // their intermediate blocks are made; no Krylov vectors, no PCG state, no LRAC inverse.
  vl_status init(Factor* fac, int t_, int prec_, const double* W64, int lmax_, bool ops_only = false) {
    f = fac;
    n = (int)f->n;
    m = f->m;
    t = t_;
    prec = prec_;
    if (t < 1 || t > 256) return fail(c, VL_ERR_INVALID_ARG, "block width t must be in [1, 256]");
    ld = lead(t);
    Aval = std::is_same<T, double>::value ? (const T*)f->A64 : (const T*)f->A32;
    valT = std::is_same<T, double>::value ? (const T*)f->valT64 : (const T*)f->valT32;
    W = mem.get<T>(n);
    Dinv = mem.get<T>(n);
    dsc = mem.get<T>(n);
    Dt = mem.get<T>(n);
    Winv = mem.get<T>(n);
    if (!W || !Dinv || !dsc || !Dt || !Winv) return fail(c, VL_ERR_OOM, "workspace exhausted (engine diagonals)");
    diag_prep_kernel<T><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, prec, W64, f->D64, W, Dinv, dsc, Dt, Winv);
    VL_CUDA(c, cudaGetLastError());
    const size_t vec = (size_t)n * ld;
    T** vs[] = {&u, &r, &z, &h, &v, &y, &sv};
    for (T** p : vs) {
      if (ops_only && p != &y && !(p == &sv && prec == VL_PREC_LRAC)) continue;
      *p = mem.get<T>(vec);
      if (!*p) return fail(c, VL_ERR_OOM, "workspace exhausted (Krylov vectors)");
      VL_CUDA(c, cudaMemsetAsync(*p, 0, sizeof(T) * vec, c->stream));
    }
    // column sweeps: 1024-thread blocks (cx lanes over the columns, a power of two), at most
    // two per SM, so that the last block's final sums read few partials
    const int cx = (t == 1) ? 1 : (t <= 32 ? 32 : (t <= 64 ? 64 : (t <= 128 ? 128 : 256)));
    cb = dim3(cx, 1024 / cx);
    csh = sizeof(double) * 1024;
    nseg = std::max(1, f->nseg);
    ncol = nseg * t;
    const int64_t want = (n + (int64_t)cb.y * 8 - 1) / ((int64_t)cb.y * 8);
    nblk = (int)std::max<int64_t>(1, std::min<int64_t>(want, 2LL * c->num_sms));
    rpb = (n + nblk - 1) / nblk;
    br = BlockRows{n, rpb, nblk, 1, nullptr, nullptr, nullptr, nullptr};
    if (nseg > 1) VL_TRY(segment_blocks());
    partial = mem.get<double>((size_t)nblk * std::max(t, 2));
    red = mem.get<double>(ncol);
    red2 = mem.get<double>(ncol);
    done = mem.get<unsigned>(1);
    if (!partial || !red || !red2 || !done) return fail(c, VL_ERR_OOM, "workspace exhausted (reductions)");
    VL_CUDA(c, cudaMemsetAsync(done, 0, sizeof(unsigned), c->stream));
    lmax = lmax_;
    if (lmax > 0) {
      double** ds[] = {&S.rz, &S.rz0, &S.alpha, &S.beta, &S.alpha_prev, &S.beta_prev, &S.bnorm2, &S.rnorm2, &S.relres};
      for (double** p : ds) {
        *p = mem.get<double>(ncol);
        if (!*p) return fail(c, VL_ERR_OOM, "workspace exhausted (PCG scalars)");
      }
      S.tol2 = nullptr;
      S.active = mem.get<int>(ncol);
      S.stop = mem.get<int>(ncol);
      S.iters = mem.get<int>(ncol);
      S.Tdiag = mem.get<double>((size_t)ncol * lmax);
      S.Toff = mem.get<double>((size_t)ncol * lmax);
      d_count = mem.get<int>(1);
      S.count = d_count;
      S.lmax = lmax;
      if (!S.active || !S.stop || !S.iters || !S.Tdiag || !S.Toff || !d_count)
        return fail(c, VL_ERR_OOM, "workspace exhausted (PCG state)");
      VL_CUDA(c, cudaMemsetAsync(S.Tdiag, 0, sizeof(double) * ncol * lmax, c->stream));
      VL_CUDA(c, cudaMemsetAsync(S.Toff, 0, sizeof(double) * ncol * lmax, c->stream));
    }
    h_count = reinterpret_cast<int*>(c->pinned);
    if (prec == VL_PREC_LRAC) {
      if (!ops_only) VL_TRY(lrac_init());
      else if (f->lrac_k >= 1 && std::is_same<T, double>::value) {   // probes L r1 need L only
        kr = f->lrac_k;
        Lk = (const T*)f->L64;
      }
    }
    return VL_OK;
  }

  // New W (float64, storage order): the diagonals and, for LRAC, C on next use.
  vl_status set_W(const double* W64) {
    diag_prep_kernel<T><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, prec, W64, f->D64, W, Dinv, dsc, Dt, Winv);
    VL_CUDA(c, cudaGetLastError());
    lr_dirty = true;
    return VL_OK;
  }

  // ------------------------------------------------------------------ LRAC
  static int chunks_for(int64_t rows, int64_t tiles, int target) {
    const int64_t want = std::max<int64_t>(1, (target + tiles - 1) / tiles);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (rows + 255) / 256));
  }

  vl_status lrac_init() {
    if (f->lrac_k < 1 || !f->L64) return fail(c, VL_ERR_STATE, "LRAC factor not built");
    if (!std::is_same<T, double>::value) VL_TRY(lrac_float(f));
    kr = f->lrac_k;
    Lk = std::is_same<T, double>::value ? (const T*)f->L64 : (const T*)f->L32;
    const int64_t kk = (int64_t)kr * kr;
    const int tq = (kr + 63) / 64;
    nch_g = chunks_for(n, (int64_t)tq * (tq + 1) / 2, 2 * c->num_sms);
    rows_g = (int)(((n + nch_g - 1) / nch_g + 31) / 32 * 32);
    nch_g = (n + rows_g - 1) / rows_g;
    if (t == 1)
      nch_a = chunks_for(n, (kr + 7) / 8, 4 * c->num_sms);
    else
      nch_a = chunks_for(n, (int64_t)tq * ((t + 63) / 64), 2 * c->num_sms);
    rows_a = (int)(((n + nch_a - 1) / nch_a + 511) / 512 * 512);
    nch_a = (n + rows_a - 1) / rows_a;
    use_tc = std::is_same<T, float>::value && t > 1 && t <= kTcN && kr <= kTcMaxRank;
    if (use_tc) {
      nch_tc = std::max(1, std::min(c->num_sms, (n + 15) / 16));
      rows_tc = ((n + nch_tc - 1) / nch_tc + 15) / 16 * 16;
      nch_tc = (n + rows_tc - 1) / rows_tc;
      Vt = mem.get<float>((size_t)((kr + 31) / 32) * 4096);
      if (!Vt) return fail(c, VL_ERR_OOM, "workspace exhausted (LRAC tensor-core operands)");
      VL_CUDA(c, cudaFuncSetAttribute(lrac_tn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTnSmem));
      VL_CUDA(c, cudaFuncSetAttribute(lrac_nn_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kNnSmem));
    }
    Cm = mem.get<double>(kk);
    Rinv = mem.get<double>(kk);
    Cinv = mem.get<double>(kk);
    lpart = mem.get<double>(std::max<int64_t>((int64_t)nch_g * kk, (int64_t)std::max(nch_a, nch_tc) * kr * t));
    Gk = mem.get<double>((size_t)kr * t);
    Vk = mem.get<double>((size_t)kr * t);
    dlogdet = mem.get<double>(1);
    lbad = mem.get<int>(1);
    b2 = mem.get<T>((size_t)n * ld);
    if (!Cm || !Rinv || !Cinv || !lpart || !Gk || !Vk || !dlogdet || !lbad || !b2)
      return fail(c, VL_ERR_OOM, "workspace exhausted (LRAC)");
    VL_CUDA(c, cudaMemsetAsync(b2, 0, sizeof(T) * (size_t)n * ld, c->stream));
    lr_dirty = true;
    return VL_OK;
  }

  // C = I + L^T W L, its blocked Cholesky factor (log det C), R^{-1} and C^{-1}.
  vl_status lrac_prepare() {
    if (!lr_dirty) return VL_OK;
    const int k = kr;
    {
      ProfScope ps(c, "lrac_gram", k);
      const int tq = (k + 63) / 64;
      lrac_tn_kernel<T><<<dim3(tq, tq, nch_g), 256, 0, VL_STREAM(c)>>>(n, k, k, rows_g, Lk, Lk, 1, n, W, 1, lpart);
      lrac_sum_chunks_kernel<<<grid_for(c, (int64_t)k * k), 256, 0, VL_STREAM(c)>>>(nch_g, (int64_t)k * k, lpart, Cm, k);
    }
    {
      ProfScope ps(c, "lrac_kxk", k);
      VL_CUDA(c, cudaMemsetAsync(dlogdet, 0, sizeof(double), c->stream));
      VL_CUDA(c, cudaMemsetAsync(lbad, 0, sizeof(int), c->stream));
      for (int J = 0; J < k; J += kCholNB) {
        const int b = std::min(kCholNB, k - J), rest = k - J - b;
        lrac_chol_panel_kernel<<<std::max(1, (rest + 127) / 128), 128, 0, VL_STREAM(c)>>>(k, J, Cm, dlogdet, lbad);
        if (rest > 0) {
          const int nt = (rest + 31) / 32;
          lrac_chol_update_kernel<<<dim3(nt, nt), 256, 0, VL_STREAM(c)>>>(k, J, Cm);
        }
      }
      const size_t smem = sizeof(double) * ((size_t)k * 16 + 256);
      const size_t smem_max = sizeof(double) * ((size_t)kMaxRank * 16 + 256);   // fixed: see cluster_size
      VL_CUDA(c, cudaFuncSetAttribute(lrac_trinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
      lrac_trinv_kernel<<<(k + 15) / 16, 256, smem, VL_STREAM(c)>>>(k, Cm, Rinv);
      lrac_cinv_kernel<<<dim3((k + 127) / 128, k), 128, 0, VL_STREAM(c)>>>(k, Rinv, Cinv);
    }
    VL_CUDA(c, cudaGetLastError());
    double* hld = reinterpret_cast<double*>(c->pinned + 64);
    int* hb = reinterpret_cast<int*>(c->pinned + 128);
    VL_CUDA(c, cudaMemcpyAsync(hld, dlogdet, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(hb, lbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*hb) return fail(c, VL_ERR_NOT_SPD, "LRAC: I + L^T W L is not numerically positive definite");
    logdetC = *hld;
    lr_dirty = false;
    return VL_OK;
  }

  // Z = (W - W L C^{-1} L^T W) R      (Woodbury form of P_LRAC^{-1})
  vl_status opPinv_lrac(const T* R, T* Zo) {
    VL_TRY(lrac_prepare());
    ProfScope ps(c, "woodbury", t);
    const int k = kr;
    if (t == 1) {
      lrac_tn1_kernel<T><<<dim3((k + 7) / 8, nch_a), 256, 0, VL_STREAM(c)>>>(n, k, rows_a, Lk, R, W, lpart);
      lrac_sum_chunks_kernel<<<grid_for(c, k), 256, 0, VL_STREAM(c)>>>(nch_a, k, lpart, Gk, 0);
      lrac_cinv_apply1_kernel<<<(k + 7) / 8, 256, 0, VL_STREAM(c)>>>(k, Cinv, Gk, Vk);
      lrac_nn1_kernel<T><<<(n + 255) / 256, 256, sizeof(T) * k, VL_STREAM(c)>>>(n, k, Lk, Vk, R, W, W, T(-1), Zo);
    } else if (use_tc) {
      if constexpr (std::is_same<T, float>::value) {
        lrac_tn_tc_kernel<<<nch_tc, 256, kTnSmem, VL_STREAM(c)>>>(n, k, t, ld, rows_tc, Lk, R, W, lpart, c->dstatus);
        lrac_sum_chunks_kernel<<<grid_for(c, (int64_t)k * t), 256, 0, VL_STREAM(c)>>>(nch_tc, (int64_t)k * t, lpart, Gk,
                                                                                     0);
        lrac_cinv_apply_kernel<<<dim3((t + 63) / 64, k), 64, 0, VL_STREAM(c)>>>(k, t, Cinv, Gk, Vk);
        VL_TRY(nn_tc(Vk, R, W, W, -1.f, Zo));
      }
    } else {
      const int tq = (k + 63) / 64, tt = (t + 63) / 64;
      lrac_tn_kernel<T><<<dim3(tq, tt, nch_a), 256, 0, VL_STREAM(c)>>>(n, k, t, rows_a, Lk, R, ld, 1, W, 0, lpart);
      lrac_sum_chunks_kernel<<<grid_for(c, (int64_t)k * t), 256, 0, VL_STREAM(c)>>>(nch_a, (int64_t)k * t, lpart, Gk, 0);
      lrac_cinv_apply_kernel<<<dim3((t + 63) / 64, k), 64, 0, VL_STREAM(c)>>>(k, t, Cinv, Gk, Vk);
      lrac_nn_kernel<T><<<dim3((n + 63) / 64, tt), 256, 0, VL_STREAM(c)>>>(n, k, t, ld, Lk, Vk, R, W, W, T(-1), Zo);
    }
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  // Z = a o Y + beta b o (L V) on the tensor cores (float32 blocks; V k x t float64).
  vl_status nn_tc(const double* V, const T* Y, const T* a, const T* b, float beta, T* Zo) {
    if constexpr (std::is_same<T, float>::value) {
      const int k = kr, nkc = (k + 31) / 32;
      lrac_vprep_kernel<<<grid_for(c, (int64_t)nkc * 32 * kTcN), 256, 0, VL_STREAM(c)>>>(k, t, nkc, V, Vt);
      const int tiles = (n + 127) / 128;
      lrac_nn_tc_kernel<<<std::max(1, std::min(tiles, 2 * c->num_sms)), 128, kNnSmem, VL_STREAM(c)>>>(
          n, k, t, ld, Lk, Vt, Y, a, b, beta, Zo, c->dstatus);
      VL_CUDA(c, cudaGetLastError());
      return VL_OK;
    } else {
      return fail(c, VL_ERR_STATE, "tensor-core LRAC path is float32 only");
    }
  }

  // Z = a o Y + L V with V (k x t, float64, device): the LRAC probe z = W^{-1/2} r2 + L r1.
  vl_status lrac_lowrank_plus(const double* V, const T* Y, const T* a, T* Zo) {
    const int k = kr;
    if (use_tc) {
      ProfScope ps(c, "woodbury", t);
      return nn_tc(V, Y, a, nullptr, 1.f, Zo);
    }
    if (t == 1)
      lrac_nn1_kernel<T><<<(n + 255) / 256, 256, sizeof(T) * k, VL_STREAM(c)>>>(n, k, Lk, V, Y, a, nullptr, T(1), Zo);
    else
      lrac_nn_kernel<T><<<dim3((n + 63) / 64, (t + 63) / 64), 256, 0, VL_STREAM(c)>>>(n, k, t, ld, Lk, V, Y, a, nullptr,
                                                                                   T(1), Zo);
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  // Segment-aligned reduction blocks of about rpb rows: each problem of a batch gets
  // ceil(rows / rpb) blocks of its own.
  vl_status segment_blocks() {
    const std::vector<int64_t>& r0 = f->seg_row0;
    if ((int)r0.size() != nseg + 1) return fail(c, VL_ERR_STATE, "batch segments missing");
    std::vector<int32_t> b0, b1, bs, sb(nseg + 1, 0);
    for (int k = 0; k < nseg; ++k) {
      sb[k] = (int32_t)b0.size();
      for (int64_t a = r0[k]; a < r0[k + 1]; a += rpb) {
        b0.push_back((int32_t)a);
        b1.push_back((int32_t)std::min<int64_t>(r0[k + 1], a + rpb));
        bs.push_back(k);
      }
    }
    sb[nseg] = (int32_t)b0.size();
    nblk = std::max(1, (int)b0.size());
    int32_t* d = mem.get<int32_t>((size_t)3 * nblk + nseg + 1);
    if (!d) return fail(c, VL_ERR_OOM, "workspace exhausted (reduction blocks)");
    std::vector<int32_t> all;
    all.insert(all.end(), b0.begin(), b0.end());
    all.insert(all.end(), b1.begin(), b1.end());
    all.insert(all.end(), bs.begin(), bs.end());
    all.insert(all.end(), sb.begin(), sb.end());
    VL_CUDA(c, cudaMemcpyAsync(d, all.data(), sizeof(int32_t) * all.size(), cudaMemcpyHostToDevice, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    br = BlockRows{n, rpb, nblk, nseg, d, d + nblk, d + 2 * nblk, d + 3 * nblk};
    h_blk_seg = bs;
    return VL_OK;
  }

  ReduceTail tail(int epi, double* out = nullptr, double tol2 = 0.0, int max_iter = 0) const {
    return ReduceTail{epi, out, S, tol2, max_iter, done};
  }

  // ------------------------------------------------------------------ primitives
  // out[k * t + c] = sum over segment k's rows of w_s X[s,c] Y[s,c]
  vl_status coldot(const T* X, const T* Y, const T* w, double* out) {
    ProfScope ps(c, "coldot", t);
    if (vec_sweeps())
      coldot_vec_kernel<T><<<nblk, 1024, vsh(), VL_STREAM(c)>>>(br, t, ld, X, Y, w, partial, tail(EPI_NONE, out));
    else
      coldot_kernel<T><<<nblk, cb, csh, VL_STREAM(c)>>>(br, t, ld, X, Y, w, partial, tail(EPI_NONE, out));
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  int spmv_grid() const { return std::max(1, std::min((n + 7) / 8, c->num_sms * 8)); }
  // blocks of the contiguous-range products: per_sm blocks per SM, at least 64 rows each
  int spmv_chunks(int per_sm) const { return std::max(1, std::min((n + 63) / 64, c->num_sms * per_sm)); }

  // Y = ys o (B X)
  vl_status opB(const T* X, const T* ys, T* Yo) {
    ProfScope ps(c, "spmv_B", t);
    if (t == 1) {
      spmv_B_t1_kernel<T, 8><<<spmv_grid(), 256, 0, VL_STREAM(c)>>>(n, m, f->nbr, Aval, X, ys, Yo);
    } else {
      // candidates (the same numbers): teams interleaved over the grid, or one contiguous range
      // of rows per block with 4 or 8 blocks per SM
      const Factor::HaloPlan* hp = nullptr;
      VL_TRY(halo_plan(c, f, true, ld * (int)sizeof(T), &hp));
      return tuned(TuneKey{c->device, 4, (int)sizeof(T), ld, log2_bucket(n)}, hp->usable ? 4 : 3, [&](int cand) {
        return with_shape<T>(ld, [&](auto L, auto N, auto U) {
          constexpr int LPV = decltype(L)::value, NV = decltype(N)::value, UNR = decltype(U)::value;
          if (cand == 3 && hp->usable) {   // staged: the block's rows in shared memory
            const void* fn = (const void*)spmv_B_staged_kernel<T, LPV, NV>;
            VL_TRY(smem_limit_once(c, fn, kHaloBytes));
            HaloArgs H{hp->brow, hp->uoff, hp->ulist, hp->lidx, hp->lself};
            spmv_B_staged_kernel<T, LPV, NV><<<hp->nb, 256, (size_t)hp->ucap * ld * sizeof(T), VL_STREAM(c)>>>(
                H, m, f->nbr, Aval, X, ld, ys, Yo);
            return cuda_ok(c, cudaGetLastError());
          }
          if (cand == 0)
            spmv_B_kernel<T, LPV, NV, UNR, 0><<<spmv_grid(), 256, 0, VL_STREAM(c)>>>(n, m, f->nbr, Aval, X, ld, ys, Yo);
          else
            spmv_B_kernel<T, LPV, NV, UNR, 1><<<spmv_chunks(cand == 1 ? 4 : 8), 256, 0, VL_STREAM(c)>>>(
                n, m, f->nbr, Aval, X, ld, ys, Yo);
          return cuda_ok(c, cudaGetLastError());
        });
      });
    }
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }
  // Z = wx o X + B^T (ys o Y)
  vl_status opBt(const T* Y, const T* ys, const T* X, const T* wx, T* Zo) {
    ProfScope ps(c, "spmv_Bt", t);
    if (t == 1) {
      spmv_Bt_t1_kernel<T, 8><<<spmv_grid(), 256, 0, VL_STREAM(c)>>>(n, f->rowptrT, f->colT, valT, Y, ys, X, wx, Zo);
    } else {
      const Factor::HaloPlan* hp = nullptr;
      VL_TRY(halo_plan(c, f, false, ld * (int)sizeof(T), &hp));
      return tuned(TuneKey{c->device, 5, (int)sizeof(T), ld, log2_bucket(n)}, hp->usable ? 4 : 3, [&](int cand) {
        return with_shape<T>(ld, [&](auto L, auto N, auto U) {
          constexpr int LPV = decltype(L)::value, NV = decltype(N)::value, UNR = decltype(U)::value;
          if (cand == 3 && hp->usable) {   // staged: the block's rows in shared memory
            const void* fn = (const void*)spmv_Bt_staged_kernel<T, LPV, NV>;
            VL_TRY(smem_limit_once(c, fn, kHaloBytes));
            HaloArgs H{hp->brow, hp->uoff, hp->ulist, hp->lidx, hp->lself};
            spmv_Bt_staged_kernel<T, LPV, NV><<<hp->nb, 256, (size_t)hp->ucap * ld * sizeof(T), VL_STREAM(c)>>>(
                H, f->rowptrT, f->colT, valT, Y, ys, X, wx, ld, Zo);
            return cuda_ok(c, cudaGetLastError());
          }
          if (cand == 0)
            spmv_Bt_kernel<T, LPV, NV, UNR, 0><<<spmv_grid(), 256, 0, VL_STREAM(c)>>>(n, f->rowptrT, f->colT, valT,
                                                                                    Y, ys, X, wx, ld, Zo);
          else
            spmv_Bt_kernel<T, LPV, NV, UNR, 1><<<spmv_chunks(cand == 1 ? 4 : 8), 256, 0, VL_STREAM(c)>>>(
                n, f->rowptrT, f->colT, valT, Y, ys, X, wx, ld, Zo);
          return cuda_ok(c, cudaGetLastError());
        });
      });
    }
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }
  // A X = W X + B^T D^{-1} B X      (Eq. pcls1 operator)
  vl_status opA(const T* X, T* Z) {
    VL_TRY(opB(X, Dinv, y));
    return opBt(y, nullptr, X, W, Z);
  }

  // Head/tail cut of the level profile: leading and trailing levels whose gathers
  // (rows + dependencies, in vector words) fit one block's round of loads run in
  // block 0 alone; the rest use the whole grid with a barrier per level.
  static void level_cut(const std::vector<int32_t>& lp, const std::vector<int32_t>& hp,
                        const std::vector<int64_t>& work, int words, int* l_head, int* l_tail) {
    const int nlev = (int)lp.size() - 1;
    const int64_t cap = 4096;   // vector loads one 512-thread block issues in ~one round trip
    // block 0 runs heavy rows one after another, so a level with more than two goes to the grid
    auto narrow = [&](int l) {
      return (work[l] + (lp[l + 1] - lp[l])) * (int64_t)words <= cap && hp[l] - lp[l] <= 2;
    };
    int h = 0;
    while (h < nlev && narrow(h)) ++h;
    int tl = nlev;
    while (tl > h && narrow(tl - 1)) --tl;
    *l_head = h;
    *l_tail = tl;
  }

  // Largest cluster (<= 16 blocks of 1024 threads, smem bytes of dynamic shared
  // memory each) the device can co-schedule for fn. Function attributes are
  // process-wide and other threads may launch fn concurrently with another size, so
  // the shared-memory bound is always set to the kernel's fixed maximum smem_max.
  // The answer depends only on (device, kernel, smem) and is cached: a solve of a small
  // problem is short enough for a driver query per call to show up in its latency.
  int cluster_size(const void* fn, size_t smem = 0, size_t smem_max = 0) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void*, size_t>, int> cache;
    const auto key = std::make_tuple(c->device, fn, smem);
    {
      std::lock_guard<std::mutex> lk(mu);
      auto it = cache.find(key);
      if (it != cache.end()) return it->second;
    }
    const int cs = cluster_size_query(fn, smem, smem_max);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = cs;
    return cs;
  }

  int cluster_size_query(const void* fn, size_t smem, size_t smem_max) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (smem_max > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 1;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(16);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 0;
    int cs = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&cs, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return std::min(cs, 16);
  }

  // Smallest power-of-two cluster (<= cs_max blocks) whose teams cover the widest
  // level in two rounds: narrow problems take a few SMs and leave the rest of the
  // device to other streams.
  static int fit_cluster(int widest, int cta_teams, int cs_max) {
    int cs = 1;
    while (cs < cs_max && widest > 2 * cs * cta_teams) cs *= 2;
    return std::min(cs, cs_max);
  }

  template <bool FWD>
  vl_status solve_launch(const T* rhs, const T* q, T* x) {
    const std::vector<int32_t>& hl = FWD ? f->h_lptr_fwd : f->h_lptr_bwd;
    const std::vector<int64_t>& hw = FWD ? f->h_lwork_fwd : f->h_lwork_bwd;
    const std::vector<int32_t>& hh = FWD ? f->h_hptr_fwd : f->h_hptr_bwd;
    LevelPlan L{FWD ? f->task_fwd : f->task_bwd, FWD ? f->lptr_fwd : f->lptr_bwd, FWD ? f->hptr_fwd : f->hptr_bwd, 0, 0,
                (int)hl.size() - 1, c->gbar, c->dstatus, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
    const char* cls = FWD ? "sptrsv_fwd" : "sptrsv_bwd";
    // form: chosen from n, t and the widest level, or forced by vl_ctx_set_solve_form
    // (VL_SOLVE_SHARED concerns single-column solves; block solves keep the automatic choice)
    const int form = (c->solve_form == VL_SOLVE_SHARED && t > 1) ? VL_SOLVE_AUTO : c->solve_form;
    if (c->prof.trace) {
      if (c->prof.dtrace_len < hl.size()) {
        if (c->prof.dtrace) c->arena.release(c->prof.dtrace);
        c->prof.dtrace = static_cast<long long*>(c->arena.alloc(sizeof(long long) * hl.size()));
        c->prof.dtrace_len = c->prof.dtrace ? hl.size() : 0;
      }
      L.trace = c->prof.dtrace;
    }
    int mm = m, l = ld;
    const int32_t* idx = FWD ? f->nbr : f->colT;
    const T* val = FWD ? Aval : valT;
    const int32_t* rp = FWD ? nullptr : f->rowptrT;
    auto launch = [&](const void* fn, void** args, int lpv, int bps, int csize = 0) -> vl_status {
      // the grid barriers start from a zeroed arrival counter and generation word in every
      // launch (the tuner launches one solve several times)
      VL_CUDA(c, cudaMemsetAsync(c->gbar, 0, 2 * sizeof(unsigned), c->stream));
      const int tpb = 16 * (32 / lpv);   // row teams per 512-thread block
      // heavy rows of the grid body in chunks: one round of loads of a team
      // (t = 1: lpv lanes x 4 loads; blocks: 16 dependency rows, whatever the row shape)
      VL_TRY(chunk_setup(FWD, t == 1 ? lpv * 4 : 16, L));
      const size_t smem = sizeof(T) * (size_t)tpb * (t == 1 ? 1 : ld);   // heavy-row partials
      level_cut(hl, hh, hw, t == 1 ? 1 : ld / VecT<T>::n, &L.l_head, &L.l_tail);
      if (form == VL_SOLVE_GRID_ALL) {   // forced: every level on the whole grid (no single-block head / tail)
        L.l_head = 0;
        L.l_tail = L.nlev;
      }
      L.head_done = 0;
      ProfScope ps(c, cls, t);
      if (t == 1 && FWD && L.l_head > 0 && (size_t)hl[L.l_head] * sizeof(T) <= kSmemSolveBytes) {
        // the narrow leading levels in one block with x in shared memory, then the grid from l_head
        const Factor::HeadPlan* hp = nullptr;
        VL_TRY(head_plan(c, f, L.l_head, &hp));
        if (hp->usable) {
          auto hfn = sptrsv_t1_head_kernel<T, 8>;
          VL_TRY(smem_limit_once(c, (const void*)hfn, kSmemSolveBytes));
          hfn<<<1, 1024, sizeof(T) * (size_t)hp->rows, VL_STREAM(c)>>>(L, m, hp->hpos, val, rhs, q, x);
          VL_CUDA(c, cudaGetLastError());
          L.head_done = 1;
        }
      }
      const int body_rows = hl[L.l_tail] - hl[L.l_head];
      // at most bps blocks per SM: fewer arrivals per grid barrier
      const int maxb = std::min(resident_blocks(c, fn, 512, smem), bps * c->num_sms);
      const int grid = std::max(1, std::min(maxb, (body_rows + tpb - 1) / tpb));
      ++c->launches;
      if (csize > 0 && cluster_grid_ok()) {
        // thread-block clusters of csize blocks, cooperative: as many whole clusters as can be
        // co-resident and the body needs; a configuration the device refuses falls back to
        // the plain cooperative launch below (a refused launch changes nothing)
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = csize;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cfg.blockDim = dim3(512);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        const int ncl = cluster_capacity(fn, cfg, csize);
        const int want = std::max(1, (grid + csize - 1) / csize);
        if (ncl >= 1) {
          cfg.gridDim = dim3(csize * std::min(ncl, want));
          if (cudaLaunchKernelExC(&cfg, fn, args) == cudaSuccess) return VL_OK;
          cudaGetLastError();
          cluster_grid_ok() = false;
        }
      }
      VL_CUDA(c, cudaLaunchCooperativeKernel(fn, grid, 512, args, smem, c->stream));
      if (L.trace) {
        std::vector<long long>& h = c->prof.traces[{cls, t}];
        h.resize(hl.size());
        VL_CUDA(c, cudaMemcpyAsync(h.data(), L.trace, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost, c->stream));
        VL_CUDA(c, cudaStreamSynchronize(c->stream));
        c->prof.cuts[{cls, t}] = {L.l_head, L.l_tail};
      }
      return VL_OK;
    };
    // the automatic choice takes the tiled walk for backward scalar solves of large systems
    // (n = 1e6 grid: 1.07 ms against 1.94 ms for the grid walk); forward scalar solves keep the
    // grid walk with its one-block head (1.05 ms against 1.20 ms), block solves keep the grid
    // walk (their rows wait on 224-byte gathers: 8.9 / 16.2 ms tiled against 2.9 / 4.5 ms)
    const bool auto_tile = form == VL_SOLVE_AUTO && t == 1 && !FWD && n > kSharedRows && x != rhs;
    if (form == VL_SOLVE_TILE || auto_tile) {
      // storage-row tiles, each row waiting only for its own dependencies (see TileArgs)
      if (x == rhs) return fail(c, VL_ERR_STATE, "tiled solve in place");
      auto args_of = [&](const Factor::TilePlan* tp) {
        return TileArgs{tp->ttask, tp->toff, tp->exported, tp->flag, c->dstatus, n, tp->R, tp->epoch};
      };
      if (t == 1) {
        constexpr int LPVT = 16;   // forward rows too: 1.20 ms against 1.33 ms with 8 lanes (n = 1e6)
        const void* fn = (const void*)sptrsv_tile1_kernel<T, FWD, LPVT>;
        VL_TRY(smem_limit_once(c, fn, kSmemSolveBytes));
        for (int bps = 1; bps <= 2; ++bps) {
          const int G = bps * c->num_sms;
          const size_t smem = sizeof(T) * (size_t)((n + G - 1) / G);
          if (smem > kSmemSolveBytes || resident_blocks(c, fn, 1024, smem) < G) continue;
          // forward: the narrow leading levels first by one block with x in shared memory (their
          // rows depend on rows far apart, which would make every link a cross-tile hand-off)
          int first = 0;
          const Factor::HeadPlan* hp = nullptr;
          if (FWD) {
            int l_tail = 0;
            level_cut(hl, hh, hw, 1, &L.l_head, &l_tail);
            if (L.l_head > 0 && (size_t)hl[L.l_head] * sizeof(T) <= kSmemSolveBytes) {
              VL_TRY(head_plan(c, f, L.l_head, &hp));
              if (hp->usable) first = hl[L.l_head];
            }
          }
          Factor::TilePlan* tp = nullptr;
          VL_TRY(tile_plan(c, f, FWD, G, first, (const Factor::TilePlan**)&tp));
          TileArgs A = args_of(tp);
          void* args[] = {&A, &mm, &idx, &val, &rp, &rhs, &q, &x};
          // every value starts "unsolved" (all bits set): it is its own ready flag
          VL_CUDA(c, cudaMemsetAsync(x, 0xff, sizeof(T) * (size_t)n, c->stream));
          ProfScope ps(c, cls, t);
          if (first > 0) {
            auto hfn = sptrsv_t1_head_kernel<T, 8>;
            VL_TRY(smem_limit_once(c, (const void*)hfn, kSmemSolveBytes));
            hfn<<<1, 1024, sizeof(T) * (size_t)hp->rows, VL_STREAM(c)>>>(L, m, hp->hpos, val, rhs, q, x);
            VL_CUDA(c, cudaGetLastError());
          }
          ++c->launches;
          return cuda_ok(c, cudaLaunchCooperativeKernel(fn, G, 1024, args, smem, c->stream));
        }
        if (form == VL_SOLVE_TILE)
          return fail(c, VL_ERR_INVALID_ARG, "solve form VL_SOLVE_TILE: a tile of x does not fit shared memory");
      }
    }
    if (form == VL_SOLVE_TILE) {
      auto args_of = [&](const Factor::TilePlan* tp) {
        return TileArgs{tp->ttask, tp->toff, tp->exported, tp->flag, c->dstatus, n, tp->R, tp->epoch};
      };
      if (ld % 8 != 0) return fail(c, VL_ERR_STATE, "block solve with a row width that is not a multiple of 8");
      // candidates (all give the same numbers: a row's sum does not depend on its tile or team):
      // tiles of 512 threads, 2 or 1 per SM, x the shape's UNR or twice it
      return tuned(TuneKey{c->device, FWD ? 2 : 3, (int)sizeof(T), ld, log2_bucket(n)}, 4, [&](int cand) {
        return with_shape<T>(ld, [&](auto Lc, auto N, auto U) {
          constexpr int LPV = decltype(Lc)::value, NV = decltype(N)::value, UNR = decltype(U)::value;
          const void* fn = (cand & 2) ? (const void*)sptrsv_tile_kernel<T, FWD, LPV, NV, 2 * UNR>
                                      : (const void*)sptrsv_tile_kernel<T, FWD, LPV, NV, UNR>;
          VL_TRY(smem_limit_once(c, fn, kSmemSolveBytes));
          // 2 or 1 tiles per SM, fewer when the shape's registers or the flags do not allow them
          int G = 0;
          size_t smem = 0;
          for (int per_sm = (cand & 1) ? 1 : 2; per_sm >= 1 && G == 0; --per_sm) {
            const int g = per_sm * c->num_sms;
            const size_t sm = sizeof(int) * (size_t)((n + g - 1) / g);
            if (sm <= kSmemSolveBytes && resident_blocks(c, fn, 512, sm) >= g) {
              G = g;
              smem = sm;
            }
          }
          if (G == 0)
            return fail(c, VL_ERR_INVALID_ARG, "solve form VL_SOLVE_TILE: the tiles do not fit the device");
          Factor::TilePlan* tp = nullptr;
          VL_TRY(tile_plan(c, f, FWD, G, 0, (const Factor::TilePlan**)&tp));
          if (tp->epoch == 0x7fffffff) {   // flags of earlier launches hold older epochs
            VL_CUDA(c, cudaMemsetAsync(tp->flag, 0, sizeof(int) * (size_t)std::max(n, 1), c->stream));
            tp->epoch = 0;
          }
          ++tp->epoch;
          TileArgs A = args_of(tp);
          void* args[] = {&A, &mm, &idx, &val, &rp, &rhs, &q, &x, &l};
          ++c->launches;
          ProfScope ps(c, cls, t);
          return cuda_ok(c, cudaLaunchCooperativeKernel(fn, G, 512, args, smem, c->stream));
        });
      });
    }
    int widest = 0;
    for (size_t lv = 0; lv + 1 < hl.size(); ++lv) widest = std::max(widest, hl[lv + 1] - hl[lv]);
    const bool smem_fits = t == 1 && (size_t)n * sizeof(T) <= kSmemSolveBytes;
    if (form == VL_SOLVE_SHARED && !smem_fits)
      return fail(c, VL_ERR_INVALID_ARG, "solve form VL_SOLVE_SHARED needs n * sizeof(value) <= 200 KiB");
    if (smem_fits && (form == VL_SOLVE_AUTO || form == VL_SOLVE_SHARED)) {
      // small system: one block with x in shared memory (see sptrsv_t1_smem_kernel)
      constexpr int LPV1 = FWD ? 8 : 16;
      auto fn = sptrsv_t1_smem_kernel<T, FWD, LPV1>;
      const size_t smem = (size_t)n * sizeof(T);
      VL_TRY(smem_limit_once(c, (const void*)fn, kSmemSolveBytes));
      L.l_head = 0;
      L.l_tail = L.nlev;
      int nn = n;
      {
        ProfScope ps(c, cls, t);
        fn<<<1, 1024, smem, VL_STREAM(c)>>>(L, nn, mm, idx, val, rp, rhs, q, x);
        VL_CUDA(c, cudaGetLastError());
      }
      if (L.trace) {
        std::vector<long long>& h = c->prof.traces[{cls, t}];
        h.resize(hl.size());
        VL_CUDA(c, cudaMemcpyAsync(h.data(), L.trace, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost, c->stream));
        VL_CUDA(c, cudaStreamSynchronize(c->stream));
        c->prof.cuts[{cls, t}] = {L.l_head, L.l_tail};
      }
      return VL_OK;
    }
    if (t > 1 && form != VL_SOLVE_GRID && form != VL_SOLVE_GRID_ALL) {
      // narrow level profile: one thread-block cluster (see sptrsv_cluster_kernel)
      vl_status out = VL_OK;
      bool done = false;
      VL_TRY(with_shape<T>(ld, [&](auto Lc, auto N, auto U) {
        constexpr int LPV = decltype(Lc)::value, NV = decltype(N)::value;
        if constexpr (NV > 2) {
          // very wide blocks stay on the grid kernel (register budget of 1024-thread blocks)
          return form == VL_SOLVE_CLUSTER ? fail(c, VL_ERR_INVALID_ARG, "solve form VL_SOLVE_CLUSTER covers float64 "
                                                                         "blocks of at most 128 columns")
                                          : VL_OK;
        } else {
        auto fn = sptrsv_cluster_kernel<T, FWD, LPV, NV, decltype(U)::value>;
        const int tpb = 32 * (32 / LPV);
        const size_t smem = sizeof(T) * (size_t)tpb * ld;
        const size_t smem_max = sizeof(T) * (size_t)tpb * (LPV * NV * VecT<T>::n);   // widest row this shape covers
        const int cs_max = cluster_size((const void*)fn, smem, smem_max);
        const int rounds = n <= kSharedRows ? VL_SHARED_CLUSTER_ROUNDS : VL_BLOCK_CLUSTER_ROUNDS;
        if (cs_max < 1)
          return form == VL_SOLVE_CLUSTER ? fail(c, VL_ERR_INVALID_ARG, "no thread-block cluster fits this solve")
                                          : VL_OK;
        if (form == VL_SOLVE_AUTO && widest > rounds * cs_max * tpb) return VL_OK;
        const int cs = fit_cluster(widest, tpb, cs_max);
        L.l_head = 0;
        L.l_tail = L.nlev;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        {
          ProfScope ps(c, cls, t);
          ++c->launches;
          out = cuda_ok(c, cudaLaunchKernelEx(&cfg, fn, L, mm, idx, val, rp, rhs, q, x, l));
        }
        done = true;
        return out;
        }
      }));
      if (done) {
        if (L.trace) {
          std::vector<long long>& h = c->prof.traces[{cls, t}];
          h.resize(hl.size());
          VL_CUDA(c, cudaMemcpyAsync(h.data(), L.trace, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost,
                                     c->stream));
          VL_CUDA(c, cudaStreamSynchronize(c->stream));
          c->prof.cuts[{cls, t}] = {L.l_head, L.l_tail};
        }
        return VL_OK;
      }
    }
    if (t == 1) {
      // one thread-block cluster walks all levels (see sptrsv_t1_cluster_kernel)
      constexpr int LPV1 = FWD ? 8 : 16;   // backward rows can list hundreds of dependents
      auto fn = sptrsv_t1_cluster_kernel<T, FWD, LPV1>;
      const int cs_max = cluster_size((const void*)fn);
      // one cluster only pays off while every level fits a few rounds of its teams;
      // the widest levels of large problems need the whole grid
      const int cta_teams = (1024 / 32) * (32 / LPV1);
      const int rounds = n <= kSharedRows ? VL_SHARED_CLUSTER_ROUNDS : VL_T1_CLUSTER_ROUNDS;
      if (form == VL_SOLVE_CLUSTER && cs_max < 1)
        return fail(c, VL_ERR_INVALID_ARG, "no thread-block cluster fits this solve");
      if (form != VL_SOLVE_GRID && form != VL_SOLVE_GRID_ALL && ((form == VL_SOLVE_CLUSTER && cs_max >= 1) ||
                                    (form == VL_SOLVE_AUTO && cs_max >= 2 && widest <= rounds * cs_max * cta_teams))) {
        const int cs = fit_cluster(widest, cta_teams, cs_max);
        L.l_head = 0;
        L.l_tail = L.nlev;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        {
          ProfScope ps(c, cls, t);
          ++c->launches;
          VL_CUDA(c, cudaLaunchKernelEx(&cfg, fn, L, mm, idx, val, rp, rhs, q, x));
        }
        if (L.trace) {
          std::vector<long long>& h = c->prof.traces[{cls, t}];
          h.resize(hl.size());
          VL_CUDA(c, cudaMemcpyAsync(h.data(), L.trace, sizeof(long long) * h.size(), cudaMemcpyDeviceToHost,
                                     c->stream));
          VL_CUDA(c, cudaStreamSynchronize(c->stream));
          c->prof.cuts[{cls, t}] = {L.l_head, L.l_tail};
        }
        return VL_OK;
      }
      void* args[] = {&L, &mm, &idx, &val, &rp, &rhs, &q, &x};
      // backward rows list up to 48 light dependents: 16 lanes keep them to one round of loads
      constexpr int LPVG = FWD ? 8 : 16;
      const void* fn1 = (const void*)sptrsv_t1_kernel<T, FWD, LPVG>;
      const void* fn1c = (const void*)sptrsv_t1_kernel<T, FWD, LPVG, 2>;
      // candidates: 2 or 1 blocks per SM with the counter barrier; clusters of 8 blocks with
      // the two-stage barrier
      return tuned(TuneKey{c->device, FWD ? 0 : 1, (int)sizeof(T), 1, log2_bucket(n)}, 3, [&](int cand) {
        return cand == 2 ? launch(fn1c, args, LPVG, 1, 8) : launch(fn1, args, LPVG, cand == 0 ? 2 : 1);
      });
    }
    // block kernels read rows as float4 / double2 words: ld must be a multiple of 8
    if (ld % 8 != 0) return fail(c, VL_ERR_STATE, "block solve with a row width that is not a multiple of 8");
    void* args[] = {&L, &mm, &idx, &val, &rp, &rhs, &q, &x, &l};
    // candidates (all give the same numbers): dependency rows in flight per lane (the shape's
    // UNR or twice it) x blocks per SM (2 or 1); clusters of 8 blocks; L2 prefetch of the next
    // rows' dependencies before each level barrier, 2 or 1 blocks per SM
    return tuned(TuneKey{c->device, FWD ? 0 : 1, (int)sizeof(T), ld, log2_bucket(n)}, 7, [&](int cand) {
      return with_shape<T>(ld, [&](auto Lc, auto N, auto U) {
        constexpr int LPV = decltype(Lc)::value, NV = decltype(N)::value, UNR = decltype(U)::value;
        if (cand == 4)   // clusters of 8 blocks with the two-stage barrier
          return launch((const void*)sptrsv_kernel<T, FWD, LPV, NV, 2 * UNR, 2>, args, LPV, 1, 8);
        if (cand >= 5)
          return launch((const void*)sptrsv_kernel<T, FWD, LPV, NV, UNR, 0, 1>, args, LPV, cand == 5 ? 2 : 1);
        const int bps = (cand & 1) ? 1 : 2;
        if (cand & 2) return launch((const void*)sptrsv_kernel<T, FWD, LPV, NV, 2 * UNR>, args, LPV, bps);
        return launch((const void*)sptrsv_kernel<T, FWD, LPV, NV, UNR>, args, LPV, bps);
      });
    });
  }
  // x = B^{-1} (q o rhs)
  vl_status solveB(const T* rhs, const T* q, T* x) { return solve_launch<true>(rhs, q, x); }
  // x = B^{-T} (q o rhs)
  vl_status solveBt(const T* rhs, const T* q, T* x) { return solve_launch<false>(rhs, q, x); }
  // P^{-1} R. VADU / LVA: B^{-1} dsc B^{-T} R (Section 3.1.1); LRAC: Woodbury.
  vl_status opPinv(const T* R, T* Zo) {
    if (prec == VL_PREC_LRAC) return opPinv_lrac(R, Zo);
    VL_TRY(solveBt(R, nullptr, sv));
    return solveB(sv, dsc, Zo);
  }
  // Sigma_tilde X = B^{-1} D B^{-T} X
  vl_status opSigma(const T* X, T* Zo) {
    VL_TRY(solveBt(X, nullptr, sv));
    return solveB(sv, Dt, Zo);
  }
  // (Sigma_tilde + W^{-1}) X       (Eq. pcls2 operator)
  vl_status opA2(const T* X, T* Zo) {
    VL_TRY(opSigma(X, y));
    add_diag_kernel<T><<<grid_for(c, (int64_t)n * ld), 256, 0, VL_STREAM(c)>>>(n, t, ld, y, Winv, X, Zo);
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  // ------------------------------------------------------------------ PCG
  // The system operator of the preconditioner's form: W + B^T D^{-1} B (Eq. pcls1) for
  // VADU and LVA, Sigma_tilde + W^{-1} (Eq. pcls2) for LRAC.
  vl_status opSys(const T* X, T* Zo) { return prec == VL_PREC_LRAC ? opA2(X, Zo) : opA(X, Zo); }

  // Solves (W + Sigma_tilde^{-1}) D = Rm. VADU / LVA: PCG on form 1. LRAC: PCG on
  // form 2, (Sigma_tilde + W^{-1}) X = Sigma_tilde Rm, then D = W^{-1} X.
  vl_status solve_A1(const T* Rm, T* Dm, double tol, int max_iter, int* iters_used, const double* tol2v = nullptr) {
    if (prec != VL_PREC_LRAC) return pcg(Rm, Dm, tol, max_iter, iters_used, tol2v);
    VL_TRY(opSigma(Rm, b2));
    VL_TRY(pcg(b2, Dm, tol, max_iter, iters_used, tol2v));
    scale_rows_kernel<T><<<grid_for(c, (int64_t)n * ld), 256, 0, VL_STREAM(c)>>>(n, t, ld, Winv, Dm);
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  // Solves S U = Bm (S = opSys) column by column (u_0 = 0), stopping a column when
  // ||r|| <= tol ||b||; records T (Lanczos) per column.
  // One PCG iteration (Appendix, PCG algorithm) on every active column: v = S h; alpha
  // (fused into the h^T v reduction); u += alpha h, r -= alpha v with the stopping test
  // (fused into the ||r||^2 reduction); z = P^{-1} r; beta, T entries and freezing (fused into
  // the r^T z reduction); h = z + beta h.
  // block vectors use the 16-byte-word sweeps (VecSweep) when a row has at most 64 words
  bool vec_sweeps() const { return t > 1 && ld % 8 == 0 && ld / VecT<T>::n <= 64; }
  size_t vsh() const { return sizeof(double) * 1024 * VecT<T>::n; }

  vl_status pcg_step(T* U, double tol2, int max_iter) {
    VL_TRY(opSys(h, v));
    {
      ProfScope ps(c, "coldot", t);
      if (vec_sweeps())
        coldot_vec_kernel<T><<<nblk, 1024, vsh(), VL_STREAM(c)>>>(br, t, ld, h, v, nullptr, partial, tail(EPI_ALPHA));
      else
        coldot_kernel<T><<<nblk, cb, csh, VL_STREAM(c)>>>(br, t, ld, h, v, nullptr, partial, tail(EPI_ALPHA));
    }
    {
      ProfScope ps(c, "pcg_update", t);
      if (vec_sweeps())
        pcg_update1_vec_kernel<T><<<nblk, 1024, vsh(), VL_STREAM(c)>>>(br, t, ld, U, r, h, v, partial,
                                                                        tail(EPI_STOP, nullptr, tol2));
      else
        pcg_update1_kernel<T><<<nblk, cb, csh, VL_STREAM(c)>>>(br, t, ld, U, r, h, v, partial,
                                                                tail(EPI_STOP, nullptr, tol2));
    }
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(opPinv(r, z));
    {
      ProfScope ps(c, "coldot", t);
      if (vec_sweeps())
        coldot_vec_kernel<T><<<nblk, 1024, vsh(), VL_STREAM(c)>>>(br, t, ld, r, z, nullptr, partial,
                                                                   tail(EPI_BETA, nullptr, 0.0, max_iter));
      else
        coldot_kernel<T><<<nblk, cb, csh, VL_STREAM(c)>>>(br, t, ld, r, z, nullptr, partial,
                                                           tail(EPI_BETA, nullptr, 0.0, max_iter));
    }
    {
      ProfScope ps(c, "pcg_update", t);
      if (vec_sweeps())
        pcg_update2_vec_kernel<T><<<nblk, 1024, 0, VL_STREAM(c)>>>(br, t, ld, S.beta, S.active, z, h);
      else
        pcg_update2_kernel<T><<<nblk, cb, 0, VL_STREAM(c)>>>(br, t, ld, S.beta, S.active, z, h);
    }
    VL_CUDA(c, cudaGetLastError());
    return VL_OK;
  }

  // Solves S U = Bm (S = opSys) column by column (u_0 = 0), stopping a column when
  // ||r|| <= tol ||b|| (or per column sqrt(tol2[q]) when tol2 is given, device, ncol entries);
  // records T (Lanczos) per column. Finished columns are frozen on the device.
  vl_status pcg(const T* Bm, T* U, double tol, int max_iter, int* iters_used, const double* tol2v = nullptr) {
    const int64_t vec = (int64_t)n * ld;
    VL_CUDA(c, cudaMemsetAsync(U, 0, sizeof(T) * vec, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(r, Bm, sizeof(T) * vec, cudaMemcpyDeviceToDevice, c->stream));
    VL_TRY(opPinv(r, z));
    VL_CUDA(c, cudaMemcpyAsync(h, z, sizeof(T) * vec, cudaMemcpyDeviceToDevice, c->stream));
    VL_TRY(coldot(r, z, nullptr, S.rz));
    VL_TRY(coldot(Bm, Bm, nullptr, S.bnorm2));
    S.tol2 = tol2v;
    pcg_init_kernel<<<1, 256, 0, VL_STREAM(c)>>>(ncol, S);
    VL_CUDA(c, cudaGetLastError());
    const double tol2 = tol * tol;
    // The host stays one iteration ahead: it issues iteration i + 1, then waits for the
    // active count (and device status) of iteration i, so the GPU never waits for the host;
    // at most one iteration runs after the last column finished, and it changes nothing.
    int* ring = reinterpret_cast<int*>(c->pinned + 256);   // {count, status} x 2
    cudaEvent_t ev[2] = {c->ev_ring[0], c->ev_ring[1]};
    bool stop = false;
    for (int it = 0; it < max_iter && !stop; ++it) {
      VL_TRY(pcg_step(U, tol2, max_iter));
      const int k = it & 1;
      VL_CUDA(c, cudaMemcpyAsync(ring + 2 * k, d_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      VL_CUDA(c, cudaMemcpyAsync(ring + 2 * k + 1, &c->dstatus->code, sizeof(int), cudaMemcpyDeviceToHost,
                                 c->stream));
      VL_CUDA(c, cudaEventRecord(ev[k], c->stream));
      if (it > 0) {
        VL_CUDA(c, cudaEventSynchronize(ev[k ^ 1]));
        stop = ring[2 * (k ^ 1)] == 0 || ring[2 * (k ^ 1) + 1] != 0;
      }
    }
    VL_TRY(check_dev_status(c, "PCG"));
    S.tol2 = nullptr;
    // iterations actually taken: the most any column took
    if (iters_used) {
      std::vector<int> its(ncol);
      VL_CUDA(c, cudaMemcpyAsync(its.data(), S.iters, sizeof(int) * ncol, cudaMemcpyDeviceToHost, c->stream));
      VL_CUDA(c, cudaStreamSynchronize(c->stream));
      *iters_used = its.empty() ? 0 : *std::max_element(its.begin(), its.end());
    }
    return VL_OK;
  }



  // Host copies of per-column results.
  vl_status column_stats(std::vector<int>& iters, std::vector<double>& relres) {
    iters.resize(ncol);
    relres.resize(ncol);
    VL_CUDA(c, cudaMemcpyAsync(iters.data(), S.iters, sizeof(int) * ncol, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(relres.data(), S.relres, sizeof(double) * ncol, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    return VL_OK;
  }
};

}  // namespace vl
