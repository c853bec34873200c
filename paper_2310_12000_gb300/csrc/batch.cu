// Batched form: independent problems merged into one block-diagonal system.
//
// The rows of every member factor are concatenated (problem k owns the storage rows
// [row0_k, row0_k + n_k)), B stays block diagonal, and the level sets of the triangular
// solves merge level by level: level l of the batch is level l of every problem, so one
// level walk, one product and one reduction launch serve all problems, and the number of
// levels is the largest of any problem, not their sum. Reductions are per problem and the
// Newton and PCG scalars per (problem, column), so each problem follows its own iteration
// (laplace.cuh); the probes of a problem are numbered by its own caller indices, so a problem
// draws the same probes in a batch as alone.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <numeric>
#include <vector>

#include "laplace.cuh"

struct vl_factor : vl::Factor {};   // the same definition as in api.cu

namespace vl {

void ctx_retain(Ctx* c);
void ctx_release_ref(Ctx* c);
vl_status pred_from_rows(State* st, const vl_opts* o, int64_t np, int m, const int32_t* Np, const double* Ap,
                         const double* Dp, const double* dF, double* dmean, double* dvar, vl_stats* loc);

struct Batch {
  Ctx* ctx = nullptr;
  std::vector<Factor*> members;
  std::vector<int64_t> row0, nnz0;
  Factor merged;
  State state;
  bool has_state = false;
  std::vector<vl_stats> mode_stats;
  std::vector<char> conv;
  std::vector<double> gammas;   // last vl_batch_log_marglik: nprob x t
  int last_t = 0;
};

namespace {

// ELL rows of one member into the merged ELL of width mm (indices shifted by off, -1 and 0
// padding); values only when nbr_out is null.
__global__ void merge_ell_kernel(int n, int m, int mm, int32_t off, const int32_t* __restrict__ nbr,
                                 const double* __restrict__ A64, const float* __restrict__ A32,
                                 int32_t* __restrict__ nbr_out, double* __restrict__ A64_out, float* __restrict__ A32_out) {
  const int64_t total = (int64_t)n * mm;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / mm), c = (int)(e % mm);
    const int64_t src = (int64_t)s * m + c;
    const int64_t dst = (int64_t)(off + s) * mm + c;
    const bool in = c < m;
    if (nbr_out) {
      const int j = in ? nbr[src] : -1;
      nbr_out[dst] = j >= 0 ? j + off : -1;
    }
    A64_out[dst] = in ? A64[src] : 0.0;
    A32_out[dst] = in ? A32[src] : 0.f;
  }
}

// out[i] = in[i] + add for i < count
__global__ void shift_kernel(int64_t count, const int32_t* __restrict__ in, int32_t add, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] + add;
}

__global__ void fill_int_kernel(int64_t count, int32_t v, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}

// Xs[s] = Xu[s2u[s]] (one column, float64)
__global__ void gather_rows_kernel(int n, const int32_t* __restrict__ s2u, const double* __restrict__ Xu,
                                   double* __restrict__ Xs) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) Xs[s] = Xu[s2u[s]];
}
__global__ void scatter_rows_kernel(int n, const int32_t* __restrict__ s2u, const double* __restrict__ Xs,
                                    double* __restrict__ Xu) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) Xu[s2u[s]] = Xs[s];
}

// Test-point rows of one member into the merged rows of width mm: neighbour Vecchia indices
// of the member -> member storage rows (v2s) for its own factor rows (Nloc), and -> merged
// storage rows (+ off) with -1 / 0 padding (Nm, Am).
__global__ void pred_rows_local_kernel(int64_t total, const int32_t* __restrict__ v2s, int32_t* __restrict__ N) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    N[e] = N[e] >= 0 ? v2s[N[e]] : -1;
}
__global__ void pred_rows_merge_kernel(int np, int m, int mm, int32_t off, const int32_t* __restrict__ Nloc,
                                       const double* __restrict__ Aloc, int32_t* __restrict__ Nm,
                                       double* __restrict__ Am) {
  const int64_t total = (int64_t)np * mm;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / mm), c = (int)(e % mm);
    const int j = c < m ? Nloc[(int64_t)p * m + c] : -1;
    Nm[e] = j >= 0 ? j + off : -1;
    Am[e] = j >= 0 ? Aloc[(int64_t)p * m + c] : 0.0;
  }
}

// Where a caller's pointer lives: *dev is set for memory that kernels on the context's device
// may use directly; another GPU's memory is refused (VL_ERR_INVALID_ARG).
vl_status locate(Ctx* c, const void* p, bool* dev) {
  *dev = false;
  if (!p) return VL_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return VL_OK;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (!device_memory_usable(a.type, a.device, c->device))
      return fail(c, VL_ERR_INVALID_ARG, "a device pointer is not on the context's device");
    *dev = true;
  }
  return VL_OK;
}

// Copies values (A, D, B^T values) of every member into the merged arrays.
vl_status merge_values(Batch* b) {
  Ctx* c = b->ctx;
  Factor& M = b->merged;
  for (size_t k = 0; k < b->members.size(); ++k) {
    Factor* f = b->members[k];
    const int n = (int)f->n;
    const int32_t off = (int32_t)b->row0[k];
    if (f->m > 0 || M.m > 0)
      merge_ell_kernel<<<grid_for(c, (int64_t)n * std::max(M.m, 1)), 256, 0, VL_STREAM(c)>>>(
          n, f->m, M.m, off, f->nbr, f->A64, f->A32, nullptr, M.A64, M.A32);
    VL_CUDA(c, cudaMemcpyAsync(M.D64 + off, f->D64, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    if (f->nnz > 0) {
      VL_CUDA(c, cudaMemcpyAsync(M.valT64 + b->nnz0[k], f->valT64, sizeof(double) * f->nnz, cudaMemcpyDeviceToDevice,
                                 c->stream));
      VL_CUDA(c, cudaMemcpyAsync(M.valT32 + b->nnz0[k], f->valT32, sizeof(float) * f->nnz, cudaMemcpyDeviceToDevice,
                                 c->stream));
    }
  }
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

// Task lists of the merged level walk: level l lists the heavy rows of every problem (problem
// order), then the light rows of every problem, each problem's rows in its own task order.
vl_status merge_levels(Batch* b, bool fwd) {
  Ctx* c = b->ctx;
  Factor& M = b->merged;
  const int P = (int)b->members.size();
  int nlev = 0;
  for (Factor* f : b->members) nlev = std::max(nlev, fwd ? f->nlev_fwd : f->nlev_bwd);
  std::vector<std::vector<int32_t>> task(P);
  for (int k = 0; k < P; ++k) {
    Factor* f = b->members[k];
    task[k].resize(f->n);
    VL_CUDA(c, cudaMemcpyAsync(task[k].data(), fwd ? f->task_fwd : f->task_bwd, sizeof(int32_t) * f->n,
                               cudaMemcpyDeviceToHost, c->stream));
  }
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<int32_t> out;
  out.reserve(M.n);
  std::vector<int32_t> lptr(nlev + 1, 0), hptr(nlev, 0);
  std::vector<int64_t> work(nlev, 0);
  for (int l = 0; l < nlev; ++l) {
    lptr[l] = (int32_t)out.size();
    for (int pass = 0; pass < 2; ++pass) {   // heavy rows of all problems, then light rows
      for (int k = 0; k < P; ++k) {
        Factor* f = b->members[k];
        const std::vector<int32_t>& lp = fwd ? f->h_lptr_fwd : f->h_lptr_bwd;
        const std::vector<int32_t>& hp = fwd ? f->h_hptr_fwd : f->h_hptr_bwd;
        if (l + 1 >= (int)lp.size()) continue;
        const int a = pass == 0 ? lp[l] : hp[l], e = pass == 0 ? hp[l] : lp[l + 1];
        for (int p = a; p < e; ++p) out.push_back(task[k][p] + (int32_t)b->row0[k]);
      }
      if (pass == 0) hptr[l] = (int32_t)out.size();
    }
    for (Factor* f : b->members) {
      const std::vector<int64_t>& w = fwd ? f->h_lwork_fwd : f->h_lwork_bwd;
      if (l < (int)w.size()) work[l] += w[l];
    }
  }
  lptr[nlev] = (int32_t)out.size();
  if ((int64_t)out.size() != M.n) return fail(c, VL_ERR_STATE, "batch: merged task list has the wrong length");
  int32_t* dtask = fwd ? M.task_fwd : M.task_bwd;
  int32_t* dl = M.mem.get<int32_t>(nlev + 1);
  int32_t* dh = M.mem.get<int32_t>(std::max(nlev, 1));
  if (!dl || !dh) return fail(c, VL_ERR_OOM, "workspace exhausted (batch levels)");
  VL_TRY(to_device(c, dtask, out));
  VL_TRY(to_device(c, dl, lptr));
  VL_TRY(to_device(c, dh, hptr));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (fwd) {
    M.nlev_fwd = nlev;
    M.lptr_fwd = dl;
    M.hptr_fwd = dh;
    M.h_lptr_fwd = lptr;
    M.h_hptr_fwd = hptr;
    M.h_lwork_fwd = work;
  } else {
    M.nlev_bwd = nlev;
    M.lptr_bwd = dl;
    M.hptr_bwd = dh;
    M.h_lptr_bwd = lptr;
    M.h_hptr_bwd = hptr;
    M.h_lwork_bwd = work;
  }
  return VL_OK;
}

vl_status batch_build(Batch* b) {
  Ctx* c = b->ctx;
  Factor& M = b->merged;
  const int P = (int)b->members.size();
  M.ctx = c;
  M.mem.ctx = c;
  b->row0.assign(P + 1, 0);
  b->nnz0.assign(P + 1, 0);
  int mm = 0;
  for (int k = 0; k < P; ++k) {
    Factor* f = b->members[k];
    b->row0[k + 1] = b->row0[k] + f->n;
    b->nnz0[k + 1] = b->nnz0[k] + f->nnz;
    mm = std::max(mm, f->m);
  }
  const int64_t n = b->row0[P], nnz = b->nnz0[P];
  if (n > (1LL << 30)) return fail(c, VL_ERR_INVALID_ARG, "batch: more than 2^30 rows in all");
  M.n = n;
  M.m = mm;
  M.nnz = nnz;
  M.nseg = P;
  M.seg_row0 = b->row0;
  M.nbr = M.mem.get<int32_t>(std::max<int64_t>(n * mm, 1));
  M.A64 = M.mem.get<double>(std::max<int64_t>(n * mm, 1));
  M.A32 = M.mem.get<float>(std::max<int64_t>(n * mm, 1));
  M.D64 = M.mem.get<double>(n);
  M.rowptrT = M.mem.get<int32_t>(n + 1);
  M.colT = M.mem.get<int32_t>(std::max<int64_t>(nnz, 1));
  M.valT64 = M.mem.get<double>(std::max<int64_t>(nnz, 1));
  M.valT32 = M.mem.get<float>(std::max<int64_t>(nnz, 1));
  M.s2u = M.mem.get<int32_t>(n);
  M.s2u_loc = M.mem.get<int32_t>(n);
  M.row_seg = M.mem.get<int32_t>(n);
  M.task_fwd = M.mem.get<int32_t>(n);
  M.task_bwd = M.mem.get<int32_t>(n);
  if (!M.nbr || !M.A64 || !M.A32 || !M.D64 || !M.rowptrT || !M.colT || !M.valT64 || !M.valT32 || !M.s2u ||
      !M.s2u_loc || !M.row_seg || !M.task_fwd || !M.task_bwd)
    return fail(c, VL_ERR_OOM, "workspace exhausted (batch)");
  for (int k = 0; k < P; ++k) {
    Factor* f = b->members[k];
    const int nk = (int)f->n;
    const int32_t off = (int32_t)b->row0[k];
    if (mm > 0)
      merge_ell_kernel<<<grid_for(c, (int64_t)nk * mm), 256, 0, VL_STREAM(c)>>>(nk, f->m, mm, off, f->nbr, f->A64,
                                                                              f->A32, M.nbr, M.A64, M.A32);
    shift_kernel<<<grid_for(c, nk), 256, 0, VL_STREAM(c)>>>(nk, f->rowptrT, (int32_t)b->nnz0[k], M.rowptrT + off);
    if (f->nnz > 0)
      shift_kernel<<<grid_for(c, f->nnz), 256, 0, VL_STREAM(c)>>>(f->nnz, f->colT, off, M.colT + b->nnz0[k]);
    shift_kernel<<<grid_for(c, nk), 256, 0, VL_STREAM(c)>>>(nk, f->s2u, off, M.s2u + off);
    VL_CUDA(c, cudaMemcpyAsync(M.s2u_loc + off, f->s2u, sizeof(int32_t) * nk, cudaMemcpyDeviceToDevice, c->stream));
    fill_int_kernel<<<grid_for(c, nk), 256, 0, VL_STREAM(c)>>>(nk, k, M.row_seg + off);
  }
  const int32_t last = (int32_t)nnz;
  VL_CUDA(c, cudaMemcpyAsync(M.rowptrT + n, &last, sizeof(int32_t), cudaMemcpyHostToDevice, c->stream));
  VL_CUDA(c, cudaGetLastError());
  VL_TRY(merge_values(b));
  VL_TRY(merge_levels(b, true));
  VL_TRY(merge_levels(b, false));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status batch_opts(Ctx* c, const vl_opts* o) {
  if (!o) return fail(c, VL_ERR_INVALID_ARG, "opts is NULL");
  if (o->precision != VL_FP64 && o->precision != VL_FP32_REFINE) return fail(c, VL_ERR_INVALID_ARG, "unknown precision");
  if (o->precond != VL_PREC_VADU && o->precond != VL_PREC_LVA)
    return fail(c, VL_ERR_INVALID_ARG, "batches support the VADU and LVA preconditioners");
  if (o->t < 1 || o->t > 256 || !(o->cg_tol > 0) || o->cg_max_iter < 1 || o->newton_max_iter < 1)
    return fail(c, VL_ERR_INVALID_ARG, "invalid option value");
  return VL_OK;
}

}  // namespace
}  // namespace vl

using namespace vl;

struct vl_batch : Batch {};

extern "C" {

vl_status vl_batch_create(vl_ctx* ctx, int nprob, vl_factor* const* factors, vl_batch** out) {
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!c) return VL_ERR_INVALID_ARG;
  if (!out || nprob < 1 || !factors) return fail(c, VL_ERR_INVALID_ARG, "vl_batch_create: invalid argument");
  for (int k = 0; k < nprob; ++k)
    if (!factors[k] || factors[k]->ctx != c || factors[k]->nseg != 1)
      return fail(c, VL_ERR_INVALID_ARG, "vl_batch_create: every factor must be a problem made on this context");
  *out = nullptr;
  vl_batch* b = new vl_batch();
  b->ctx = c;
  for (int k = 0; k < nprob; ++k) b->members.push_back(factors[k]);
  const vl_status s = batch_build(b);
  if (s != VL_OK) {
    b->merged.mem.free_all();
    delete b;
    return s;
  }
  ctx_retain(c);
  *out = b;
  return VL_OK;
}

vl_status vl_batch_refresh(vl_batch* b) {
  if (!b) return VL_ERR_INVALID_ARG;
  VL_TRY(merge_values(b));
  VL_CUDA(b->ctx, cudaStreamSynchronize(b->ctx->stream));
  return VL_OK;
}

vl_status vl_batch_info(const vl_batch* b, int64_t* n_total, int* nlev_fwd, int* nlev_bwd) {
  if (!b) return VL_ERR_INVALID_ARG;
  if (n_total) *n_total = b->merged.n;
  if (nlev_fwd) *nlev_fwd = b->merged.nlev_fwd;
  if (nlev_bwd) *nlev_bwd = b->merged.nlev_bwd;
  return VL_OK;
}

vl_status vl_batch_find_mode(vl_batch* b, const int* lik, const double* y, const double* F, const vl_opts* opts,
                             double* mode_out, vl_stats* stats) {
  if (!b) return VL_ERR_INVALID_ARG;
  Ctx* c = b->ctx;
  VL_TRY(batch_opts(c, opts));
  const int P = (int)b->members.size();
  if (!lik || !y) return fail(c, VL_ERR_INVALID_ARG, "vl_batch_find_mode: lik and y are required");
  for (int k = 0; k < P; ++k)
    if (lik[k] != VL_LIK_BERNOULLI_LOGIT && lik[k] != VL_LIK_POISSON_LOG && lik[k] != VL_LIK_GAMMA_LOG)
      return fail(c, VL_ERR_INVALID_ARG, "vl_batch_find_mode: unknown likelihood");
  if (!(opts->lik_shape > 0.0 && std::isfinite(opts->lik_shape)))
    return fail(c, VL_ERR_INVALID_ARG, "vl_batch_find_mode: the gamma shape must be > 0");
  Factor& M = b->merged;
  const int n = (int)M.n;
  State& st = b->state;
  if (!b->has_state) {
    st.f = &M;
    st.ctx = c;
    st.mem.ctx = c;
    st.y = st.mem.get<double>(n);
    st.F = st.mem.get<double>(n);
    st.b = st.mem.get<double>(n);
    st.W = st.mem.get<double>(n);
    st.d_seg_lik = st.mem.get<int>(P);
    st.d_seg_shape = st.mem.get<double>(P);
    if (!st.y || !st.F || !st.b || !st.W || !st.d_seg_lik || !st.d_seg_shape) {
      st.mem.free_all();
      return fail(c, VL_ERR_OOM, "workspace exhausted (batch state)");
    }
    b->has_state = true;
  }
  std::vector<int> hl(lik, lik + P);
  std::vector<double> hs(P);
  for (int k = 0; k < P; ++k) hs[k] = lik[k] == VL_LIK_GAMMA_LOG ? opts->lik_shape : 1.0;
  VL_TRY(to_device(c, st.d_seg_lik, hl));
  VL_TRY(to_device(c, st.d_seg_shape, hs));
  {
    Scratch S(c);
    const double *dy = y, *dF = F;
    bool y_dev, F_dev;
    VL_TRY(locate(c, y, &y_dev));
    VL_TRY(locate(c, F, &F_dev));
    if (!y_dev) {
      double* t = S.get<double>(n);
      if (!t) return fail(c, VL_ERR_OOM, "workspace exhausted (staging y)");
      VL_CUDA(c, cudaMemcpyAsync(t, y, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      dy = t;
    }
    if (F && !F_dev) {
      double* t = S.get<double>(n);
      if (!t) return fail(c, VL_ERR_OOM, "workspace exhausted (staging F)");
      VL_CUDA(c, cudaMemcpyAsync(t, F, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
      dF = t;
    }
    gather_rows_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, M.s2u, dy, st.y);
    if (dF)
      gather_rows_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, M.s2u, dF, st.F);
    else
      VL_CUDA(c, cudaMemsetAsync(st.F, 0, sizeof(double) * n, c->stream));
    VL_CUDA(c, cudaMemsetAsync(st.b, 0, sizeof(double) * n, c->stream));
    int* bad = S.get<int>(1);
    if (!bad) return fail(c, VL_ERR_OOM, "workspace exhausted (input check)");
    VL_CUDA(c, cudaMemsetAsync(bad, 0x7f, sizeof(int), c->stream));
    check_inputs_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, lik_spec(&st), st.y, st.F, bad);
    VL_CUDA(c, cudaGetLastError());
    std::vector<int> hb;
    VL_TRY(to_host(c, hb, (const int*)bad, 1));
    if (hb[0] >= 0 && hb[0] < n) {
      std::vector<int32_t> seg, loc;
      VL_TRY(to_host(c, seg, (const int32_t*)M.row_seg + hb[0], 1));
      VL_TRY(to_host(c, loc, (const int32_t*)M.s2u_loc + hb[0], 1));
      char buf[200];
      snprintf(buf, sizeof buf, "vl_batch_find_mode: problem %d, y[%d] is not a finite value in the support of its "
               "likelihood (or its offset is not finite)", seg[0], loc[0]);
      return fail(c, VL_ERR_INVALID_ARG, buf);
    }
  }
  VL_TRY(newton_run(&st, opts, b->mode_stats, b->conv));
  if (mode_out) {
    bool out_dev;
    VL_TRY(locate(c, mode_out, &out_dev));
    if (out_dev) {
      scatter_rows_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, M.s2u, st.b, mode_out);
    } else {
      Scratch S(c);
      double* t = S.get<double>(n);
      if (!t) return fail(c, VL_ERR_OOM, "workspace exhausted (mode out)");
      scatter_rows_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, M.s2u, st.b, t);
      VL_CUDA(c, cudaMemcpyAsync(mode_out, t, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    }
    VL_CUDA(c, cudaGetLastError());
  }
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  if (stats)
    for (int k = 0; k < P; ++k) stats[k] = b->mode_stats[k];
  for (int k = 0; k < P; ++k)
    if (!b->conv[k]) return fail(c, VL_ERR_NOT_CONVERGED, "Newton reached newton_max_iter on a problem of the batch");
  return VL_OK;
}

vl_status vl_batch_log_marglik(vl_batch* b, const vl_opts* o, double* lml, double* logdet, vl_stats* stats) {
  if (!b) return VL_ERR_INVALID_ARG;
  Ctx* c = b->ctx;
  VL_TRY(batch_opts(c, o));
  if (!lml) return fail(c, VL_ERR_INVALID_ARG, "lml is NULL");
  if (!b->has_state) return fail(c, VL_ERR_STATE, "vl_batch_log_marglik: call vl_batch_find_mode first");
  const int P = (int)b->members.size(), t = o->t;
  SlqOut q;
  if (o->precision == VL_FP64)
    VL_TRY(slq_run<double>(&b->state, o, q));
  else
    VL_TRY(slq_run<float>(&b->state, o, q));
  LmlOut L;
  VL_TRY(lml_assemble(&b->state, o, q, L));
  b->gammas = q.gam;
  b->last_t = t;
  for (int k = 0; k < P; ++k) {
    lml[k] = L.lml[k];
    if (logdet) logdet[k] = L.logdet[k];
    if (stats) {
      vl_stats& s = stats[k];
      s = vl_stats{};
      s.cg_calls = 1;
      for (int j = 0; j < t; ++j) {
        s.cg_iters_max = std::max(s.cg_iters_max, q.iters[k * t + j]);
        s.cg_iters_total += q.iters[k * t + j];
        s.cg_relres_max = std::max(s.cg_relres_max, q.relres[k * t + j]);
      }
      s.true_relres_max = q.true_rel[k];
      s.probe_relres_max = q.true_rel[k];
      s.probe_refine_steps = q.passes[k];
      s.slq_mean = L.mean[k];
      s.slq_stderr = L.se[k];
      s.logdet = L.logdet[k];
    }
  }
  return VL_OK;
}

vl_status vl_batch_pred_var(vl_batch* b, const int64_t* np, const double* test_locs, const double* Fp,
                            const vl_opts* o, double* mean, double* var) {
  if (!b) return VL_ERR_INVALID_ARG;
  Ctx* c = b->ctx;
  VL_TRY(batch_opts(c, o));
  if (!np || o->s < 1) return fail(c, VL_ERR_INVALID_ARG, "vl_batch_pred_var: invalid argument");
  if (!b->has_state) return fail(c, VL_ERR_STATE, "vl_batch_pred_var: call vl_batch_find_mode first");
  const int P = (int)b->members.size();
  Factor& M = b->merged;
  std::vector<int64_t> p0(P + 1, 0);
  for (int k = 0; k < P; ++k) {
    if (np[k] < 0) return fail(c, VL_ERR_INVALID_ARG, "vl_batch_pred_var: negative test count");
    p0[k + 1] = p0[k] + np[k];
  }
  const int64_t ntot = p0[P];
  if (ntot == 0) return VL_OK;
  if (!test_locs || ntot > (1LL << 30)) return fail(c, VL_ERR_INVALID_ARG, "vl_batch_pred_var: invalid argument");
  const int mm = std::max(M.m, 1);
  Scratch S(c);
  const double* dq = test_locs;
  const double* dF = Fp;
  bool q_dev, F_dev, mean_dev, var_dev;
  VL_TRY(locate(c, test_locs, &q_dev));
  VL_TRY(locate(c, Fp, &F_dev));
  VL_TRY(locate(c, mean, &mean_dev));
  VL_TRY(locate(c, var, &var_dev));
  if (!q_dev) {
    double* t = S.get<double>((size_t)ntot * 2);
    if (!t) return fail(c, VL_ERR_OOM, "workspace exhausted (staging test locations)");
    VL_CUDA(c, cudaMemcpyAsync(t, test_locs, sizeof(double) * ntot * 2, cudaMemcpyHostToDevice, c->stream));
    dq = t;
  }
  if (Fp && !F_dev) {
    double* t = S.get<double>(ntot);
    if (!t) return fail(c, VL_ERR_OOM, "workspace exhausted (staging Fp)");
    VL_CUDA(c, cudaMemcpyAsync(t, Fp, sizeof(double) * ntot, cudaMemcpyHostToDevice, c->stream));
    dF = t;
  }
  int32_t* Nm = S.get<int32_t>((size_t)ntot * mm);
  double* Am = S.get<double>((size_t)ntot * mm);
  double* Dp = S.get<double>(ntot);
  double* dmean = S.get<double>(ntot);
  double* dvar = S.get<double>(ntot);
  if (!Nm || !Am || !Dp || !dmean || !dvar) return fail(c, VL_ERR_OOM, "workspace exhausted (batch prediction)");
  // each problem's test points condition on its own m nearest training points (Section 4.1)
  for (int k = 0; k < P; ++k) {
    const int64_t npk = np[k];
    if (npk == 0) continue;
    Factor* f = b->members[k];
    const int m = f->m;
    Scratch T(c);
    int32_t* Nl = T.get<int32_t>((size_t)npk * std::max(m, 1));
    double* Al = T.get<double>((size_t)npk * std::max(m, 1));
    if (!Nl || !Al) return fail(c, VL_ERR_OOM, "workspace exhausted (batch prediction rows)");
    const double* q = dq + 2 * p0[k];
    if (m > 0) {
      VL_TRY(knn_cross_dev(c, f->locs_v, f->n, q, npk, m, Nl));
      pred_rows_local_kernel<<<grid_for(c, npk * m), 256, 0, VL_STREAM(c)>>>(npk * m, f->v2s, Nl);
      VL_CUDA(c, cudaGetLastError());
    }
    VL_CUDA(c, status_clear(c));
    VL_TRY(factor_rows(c, npk, m, q, f->locs_s, Nl, f->cov, f->sigma2, f->rho, f->nugget, Al, Dp + p0[k], nullptr));
    VL_TRY(check_dev_status(c, "batch prediction rows"));
    pred_rows_merge_kernel<<<grid_for(c, npk * mm), 256, 0, VL_STREAM(c)>>>((int)npk, m, mm, (int32_t)b->row0[k], Nl,
                                                                           Al, Nm + p0[k] * mm, Am + p0[k] * mm);
    VL_CUDA(c, cudaGetLastError());
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  VL_TRY(pred_from_rows(&b->state, o, ntot, mm, Nm, Am, Dp, dF, dmean, var ? dvar : nullptr, nullptr));
  if (mean)
    VL_CUDA(c, cudaMemcpyAsync(mean, dmean, sizeof(double) * ntot,
                               mean_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  if (var)
    VL_CUDA(c, cudaMemcpyAsync(var, dvar, sizeof(double) * ntot,
                               var_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status vl_batch_gammas(const vl_batch* b, double* gammas, int t) {
  if (!b) return VL_ERR_INVALID_ARG;
  if (!gammas || t != b->last_t || b->gammas.empty())
    return fail(b->ctx, VL_ERR_STATE, "vl_batch_gammas: no SLQ result of that width");
  std::copy(b->gammas.begin(), b->gammas.end(), gammas);
  return VL_OK;
}

void vl_batch_destroy(vl_batch* b) {
  if (!b) return;
  Ctx* c = b->ctx;
  cudaStreamSynchronize(c->stream);
  b->state.mem.free_all();
  b->merged.mem.free_all();
  delete b;
  ctx_release_ref(c);
}

}  // extern "C"
