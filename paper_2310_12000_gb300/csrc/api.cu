// extern "C" entry points of libvl (include/vl.h) and the orchestration of the
// Newton, SLQ and prediction steps. Every arithmetic step runs in the kernels of
// kernels.cuh / factor.cu / knn.cu / graph.cu; the host only sequences launches,
// reads back scalars and makes the stopping decisions.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "lanczos.cuh"

namespace vl {

// ----------------------------------------------------------------------------- small kernels
__global__ void gather2_kernel(int n, const double* __restrict__ in, const int32_t* __restrict__ idx,
                               double* __restrict__ out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) {
    int u = idx ? idx[k] : k;
    out[2 * k] = in[2 * (int64_t)u];
    out[2 * k + 1] = in[2 * (int64_t)u + 1];
  }
}

template <typename T>
__global__ void to_storage_kernel(int n, int t, int ld, const int32_t* __restrict__ s2u, const double* __restrict__ Xu,
                                  T* __restrict__ Xs) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    Xs[e] = (c < t) ? (T)Xu[(int64_t)s2u[s] * t + c] : T(0);
  }
}

template <typename T>
__global__ void from_storage_kernel(int n, int t, int ld, const int32_t* __restrict__ s2u, const T* __restrict__ Xs,
                                    double* __restrict__ Xu) {
  const int64_t total = (int64_t)n * t;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / t), c = (int)(e % t);
    Xu[(int64_t)s2u[s] * t + c] = (double)Xs[(int64_t)s * ld + c];
  }
}

__global__ void export_kernel(int n, int m, const int32_t* __restrict__ s2v, const int32_t* __restrict__ nbr,
                              const double* __restrict__ A, const double* __restrict__ D, const int32_t* __restrict__ lf,
                              const int32_t* __restrict__ lb, int32_t* __restrict__ N_out, double* __restrict__ A_out,
                              double* __restrict__ D_out, int32_t* __restrict__ lf_out, int32_t* __restrict__ lb_out) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int k = s2v[s];
  for (int c = 0; c < m; ++c) {
    const int j = nbr[(int64_t)s * m + c];
    if (N_out) N_out[(int64_t)k * m + c] = j >= 0 ? s2v[j] : -1;
    if (A_out) A_out[(int64_t)k * m + c] = A[(int64_t)s * m + c];
  }
  if (D_out) D_out[k] = D[s];
  if (lf_out) lf_out[k] = lf[s];
  if (lb_out) lb_out[k] = lb[s];
}

// out[b] = partial sums of x (one column) or of log D etc., combined with reduce_partials.
__global__ void sum_kernel(int n, int mode, const double* __restrict__ a, const double* __restrict__ b,
                           double* __restrict__ partial) {
  double acc = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double v;
    if (mode == 0) v = a[s];                          // sum a
    else if (mode == 1) v = log(a[s]);                // sum log a
    else v = log(b[s] + 1.0 / a[s]);                  // sum log(W + 1/D), a = D, b = W
    acc += v;
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < blockDim.x; ++i) s += sh[i];
    partial[blockIdx.x] = s;
  }
}

__global__ void absmax_kernel(int n, const double* __restrict__ a, const double* __restrict__ b,
                              double* __restrict__ partial) {
  double m1 = 0.0, m2 = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    m1 = fmax(m1, fabs(a[s] - (b ? b[s] : 0.0)));
    m2 = fmax(m2, fabs(a[s]));
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = m1;
  s2[threadIdx.x] = m2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < blockDim.x; ++i) {
      x = fmax(x, s1[i]);
      y = fmax(y, s2[i]);
    }
    partial[2 * blockIdx.x] = x;
    partial[2 * blockIdx.x + 1] = y;
  }
}

__global__ void set_wait_limit_kernel(DevStatus* st, long long cycles) { st->limit = cycles; }

// One bounded wait on a flag that nothing sets (the library's timeout path).
__global__ void wait_probe_kernel(const int* flag, DevStatus* st) {
  if (threadIdx.x == 0) bounded_wait([&] { return ld_acquire(flag) != 0; }, st, -1);
}

// Prediction: mean_p = Fp + sum_c Ap[p,c] b[nbr_p,c];  var_p = Dp + mean_k z4[p,k]^2 with
// z4[p,k] = -sum_c Ap[p,c] U[nbr_p,c][k]. One warp per test point, lanes over columns.
template <typename T>
__global__ void pred_kernel(int np, int m, const int32_t* __restrict__ nbr, const double* __restrict__ Ap,
                            const double* __restrict__ Dp, const double* __restrict__ Fp, const double* __restrict__ b,
                            const T* __restrict__ U, int s_cols, int ld, double* __restrict__ mean,
                            double* __restrict__ var_acc) {
  const int lane = threadIdx.x & 31;
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= np) return;
  double mu = 0.0;
  for (int c = lane; c < m; c += 32) {
    const int j = nbr[(int64_t)p * m + c];
    if (j >= 0) mu += Ap[(int64_t)p * m + c] * b[j];
  }
  mu = warp_sum(mu);
  double sq = 0.0;
  if (U) {
    for (int col = lane; col < s_cols; col += 32) {
      double z4 = 0.0;
      for (int c = 0; c < m; ++c) {
        const int j = nbr[(int64_t)p * m + c];
        if (j < 0) break;
        z4 -= Ap[(int64_t)p * m + c] * (double)U[(int64_t)j * ld + col];
      }
      sq += z4 * z4;
    }
    sq = warp_sum(sq);
  }
  if (lane == 0) {
    if (mean) mean[p] = (Fp ? Fp[p] : 0.0) + mu;
    if (var_acc) var_acc[p] += sq;
  }
}

__global__ void pred_finish_kernel(int np, const double* __restrict__ Dp, double inv_s, double* __restrict__ var) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < np) var[p] = Dp[p] + var[p] * inv_s;
}

// L_out[s2u[s] * k + j] = L[j * n + s]  (column-major storage rows -> caller rows)
__global__ void lrac_export_kernel(int n, int k, const int32_t* __restrict__ s2u, const double* __restrict__ L,
                                   double* __restrict__ out) {
  const int64_t total = (int64_t)n * k;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), s = (int)(e % n);
    out[(int64_t)s2u[s] * k + j] = L[e];
  }
}

__global__ void translate_kernel(int64_t total, const int32_t* __restrict__ map, int32_t* __restrict__ idx) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    idx[e] = idx[e] >= 0 ? map[idx[e]] : -1;
}

// ----------------------------------------------------------------------------- pointer staging
static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory that kernels on the context's device may not use (another GPU's memory).
static bool foreign_device_ptr(Ctx* c, const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && !device_memory_usable(a.type, a.device, c->device);
}

template <typename T>
static vl_status stage_in(Ctx* c, Scratch& S, const T* p, size_t count, const T** out) {
  if (!p || count == 0) {
    *out = p;
    return VL_OK;
  }
  if (foreign_device_ptr(c, p)) return fail(c, VL_ERR_INVALID_ARG, "a device pointer is not on the context's device");
  if (is_device_ptr(p)) {
    *out = p;
    return VL_OK;
  }
  T* d = S.get<T>(count);
  if (!d) return fail(c, VL_ERR_OOM, "workspace exhausted (staging input)");
  VL_CUDA(c, cudaMemcpyAsync(d, p, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
  *out = d;
  return VL_OK;
}

template <typename T>
static vl_status stage_out(Ctx* c, const T* dev, T* p, size_t count) {
  if (!p || count == 0) return VL_OK;
  if (foreign_device_ptr(c, p)) return fail(c, VL_ERR_INVALID_ARG, "a device pointer is not on the context's device");
  const bool d = is_device_ptr(p);
  VL_CUDA(c, cudaMemcpyAsync(p, dev, sizeof(T) * count, d ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
  if (!d) VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

static double read_scalar(Ctx* c, const double* dev, vl_status* st) {
  double v = 0.0;
  cudaError_t e = cudaMemcpyAsync(&v, dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) *st = cuda_fail(c, e, "read back");
  return v;
}

static vl_status check_opts(Ctx* c, const vl_opts* o) {
  if (!o) return fail(c, VL_ERR_INVALID_ARG, "opts is NULL");
  if (o->precision != VL_FP64 && o->precision != VL_FP32_REFINE)
    return fail(c, VL_ERR_INVALID_ARG, "unknown precision");
  if (o->precond < 0 || o->precond > 2) return fail(c, VL_ERR_INVALID_ARG, "unknown preconditioner");
  if (o->precond == VL_PREC_LRAC && (o->k < 1 || o->k > kMaxRank))
    return fail(c, VL_ERR_INVALID_ARG, "LRAC rank k must be in [1, " + std::to_string(kMaxRank) + "]");
  if (o->t < 1 || o->t > 256 || o->s < 1 || !(o->cg_tol > 0) || o->cg_max_iter < 1 || o->newton_max_iter < 1)
    return fail(c, VL_ERR_INVALID_ARG, "invalid option value");
  return VL_OK;
}

// The LRAC factor L_k of Sigma (built once per covariance parameters and k).
static vl_status ensure_precond(Factor* f, const vl_opts* o) {
  if (o->precond != VL_PREC_LRAC) return VL_OK;
  return lrac_build(f, o->k);
}

// VL_ERR_NOT_CONVERGED when a column of the engine's last PCG run stopped at cg_max_iter
// above cg_tol.
template <typename T>
static vl_status cg_converged(Engine<T>& E, const vl_opts* o, const char* what) {
  std::vector<int> iters;
  std::vector<double> rel;
  VL_TRY(E.column_stats(iters, rel));
  for (int k = 0; k < E.ncol; ++k)
    if (rel[k] > o->cg_tol && iters[k] >= o->cg_max_iter)
      return fail(E.c, VL_ERR_NOT_CONVERGED, std::string(what) + ": PCG reached cg_max_iter above cg_tol");
  return VL_OK;
}

}  // namespace vl

namespace vl {

__global__ void repack_kernel(int64_t total, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[e];
}

// U = (W + Sigma_tilde^{-1})^{-1} z3 for simulation columns [col0, col0 + sc),
// z3 = W^{1/2} z1 + B^T D^{-1/2} z2 (Algorithm simAlgo). U: n x ld float64 (storage).
static vl_status sim_block(State* st, const vl_opts* o, Engine<double>& E64, int sc, int col0, double* U,
                           vl_stats* stats) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n, ld = E64.ld;
  const int64_t vec = (int64_t)n * ld;
  Scratch S(c);
  double* z1 = S.get<double>(vec);
  double* z2 = S.get<double>(vec);
  double* z3 = S.get<double>(vec);
  double* sW = S.get<double>(n);
  double* sD = S.get<double>(n);
  if (!z1 || !z2 || !z3 || !sW || !sD) return fail(c, VL_ERR_OOM, "workspace exhausted (simulation)");
  gaussian_kernel<<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, sc, ld, col0, f->s2u_probe(), o->seed, 1, z1);
  gaussian_kernel<<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, sc, ld, col0, f->s2u_probe(), o->seed, 2, z2);
  diag_fn_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 2, st->W, f->D64, sW);
  diag_fn_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 1, st->W, f->D64, sD);
  VL_CUDA(c, cudaGetLastError());
  VL_TRY(E64.opBt(z2, sD, z1, sW, z3));
  int used = 0;
  if (o->precision == VL_FP64) {
    VL_TRY(E64.solve_A1(z3, U, o->cg_tol, o->cg_max_iter, &used));
    if (stats) {
      stats->cg_calls++;
      stats->cg_iters_total += used;
      stats->cg_iters_max = used;
    }
    return cg_converged(E64, o, "simulation solves");
  }
  Engine<float> E32(c);
  VL_TRY(E32.init(f, sc, o->precond, st->W, o->cg_max_iter + 1));
  double* res = S.get<double>(vec);
  float* r32 = S.get<float>(vec);
  float* d32 = S.get<float>(vec);
  if (!res || !r32 || !d32) return fail(c, VL_ERR_OOM, "workspace exhausted (simulation refinement)");
  VL_CUDA(c, cudaMemsetAsync(res, 0, sizeof(double) * vec, c->stream));
  VL_CUDA(c, cudaMemsetAsync(U, 0, sizeof(double) * vec, c->stream));
  // per (problem, column) norms: a batch has nseg * sc columns
  const int ncol = E64.ncol;
  VL_TRY(E64.coldot(z3, z3, nullptr, E64.red2));
  std::vector<double> bn(ncol), rn(ncol);
  VL_CUDA(c, cudaMemcpyAsync(bn.data(), E64.red2, sizeof(double) * ncol, cudaMemcpyDeviceToHost, c->stream));
  double worst = 1.0;
  for (int pass = 0; pass < 12; ++pass) {
    VL_TRY(E64.opA(U, res));
    residual_kernel<<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, z3, res);
    VL_TRY(E64.coldot(res, res, nullptr, E64.red));
    VL_CUDA(c, cudaMemcpyAsync(rn.data(), E64.red, sizeof(double) * ncol, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    worst = 0.0;
    for (int k = 0; k < ncol; ++k) worst = std::max(worst, bn[k] > 0 ? std::sqrt(rn[k] / bn[k]) : 0.0);
    if (worst <= o->cg_tol) break;
    repack_kernel<<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, res, r32);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(E32.solve_A1(r32, d32, std::max(o->cg_tol, 1e-4), o->cg_max_iter, &used));
    accumulate_kernel<double, float><<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, U, d32);
    VL_CUDA(c, cudaGetLastError());
    if (stats) {
      stats->cg_calls++;
      stats->cg_iters_total += used;
      stats->cg_iters_max = used;
      stats->refine_steps++;
    }
  }
  if (stats) stats->true_relres_max = std::max(stats->true_relres_max, worst);
  if (worst > o->cg_tol) return fail(c, VL_ERR_NOT_CONVERGED, "simulation solves: refinement did not reach cg_tol");
  return VL_OK;
}

// Predictive mean and simulated variances at np test points whose neighbours (storage rows of
// st->f, -1 padding, m per point), weights Ap and conditional variances Dp are given (Eq.
// latentpostpredictive, Algorithm simAlgo); mean/var device arrays of np. Shared by single
// problems and batches.
vl_status pred_from_rows(State* st, const vl_opts* o, int64_t np, int m, const int32_t* Np, const double* Ap,
                         const double* Dp, const double* dF, double* dmean, double* dvar, vl_stats* loc) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n;
  Scratch S(c);
  const int pg = (int)((np * 32 + 255) / 256);
  if (dmean) {
    pred_kernel<double><<<pg, 256, 0, VL_STREAM(c)>>>((int)np, m, Np, Ap, Dp, dF, st->b, nullptr, 0, 1, dmean, nullptr);
    VL_CUDA(c, cudaGetLastError());
  }
  if (!dvar) return VL_OK;
  VL_CUDA(c, cudaMemsetAsync(dvar, 0, sizeof(double) * np, c->stream));
  if (o->precond == VL_PREC_LRAC) VL_TRY(lrac_build(f, o->k));
  for (int col0 = 0; col0 < o->s; col0 += 128) {
    const int sc = std::min(128, o->s - col0);
    Engine<double> E64(c);
    VL_TRY(E64.init(f, sc, o->precond, st->W, o->precision == VL_FP64 ? o->cg_max_iter + 1 : 0));
    double* U = S.get<double>((size_t)n * E64.ld);
    if (!U) return fail(c, VL_ERR_OOM, "workspace exhausted (simulation)");
    VL_TRY(sim_block(st, o, E64, sc, col0, U, loc));
    pred_kernel<double><<<pg, 256, 0, VL_STREAM(c)>>>((int)np, m, Np, Ap, Dp, nullptr, st->b, U, sc, E64.ld, nullptr, dvar);
    VL_CUDA(c, cudaGetLastError());
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    c->arena.release(U);
    S.blocks.erase(std::find(S.blocks.begin(), S.blocks.end(), (void*)U));
  }
  pred_finish_kernel<<<(int)((np + 255) / 256), 256, 0, VL_STREAM(c)>>>((int)np, Dp, 1.0 / o->s, dvar);
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

template <typename T>
static vl_status apply_op(State* st, int op, const double* Xd, int t, const vl_opts* o, double* Yd) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n;
  Engine<T> E(c);
  VL_TRY(ensure_precond(f, o));
  VL_TRY(E.init(f, t, o->precond, st->W, 0));
  to_storage_kernel<T><<<grid_for(c, (int64_t)n * E.ld), 256, 0, VL_STREAM(c)>>>(n, t, E.ld, f->s2u, Xd, E.u);
  VL_CUDA(c, cudaGetLastError());
  switch (op) {
    case VL_OP_A: VL_TRY(E.opA(E.u, E.v)); break;
    case VL_OP_PINV: VL_TRY(E.opPinv(E.u, E.v)); break;
    case VL_OP_B: VL_TRY(E.opB(E.u, nullptr, E.v)); break;
    case VL_OP_BT: VL_TRY(E.opBt(E.u, nullptr, nullptr, nullptr, E.v)); break;
    case VL_OP_BINV: VL_TRY(E.solveB(E.u, nullptr, E.v)); break;
    case VL_OP_BTINV: VL_TRY(E.solveBt(E.u, nullptr, E.v)); break;
    case VL_OP_SIGMA: VL_TRY(E.opSigma(E.u, E.v)); break;
    case VL_OP_A2: VL_TRY(E.opA2(E.u, E.v)); break;
    default: return fail(c, VL_ERR_INVALID_ARG, "vl_apply: unknown op");
  }
  from_storage_kernel<T><<<grid_for(c, (int64_t)n * t), 256, 0, VL_STREAM(c)>>>(n, t, E.ld, f->s2u, E.v, Yd);
  VL_CUDA(c, cudaGetLastError());
  return check_dev_status(c, "vl_apply");
}

template <typename T>
static vl_status pcg_op(State* st, const double* Rd, int t, const vl_opts* o, double* Ud, int lmax, double* Td,
                        double* To, int* iters, double* relres) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n;
  Engine<T> E(c);
  VL_TRY(ensure_precond(f, o));
  VL_TRY(E.init(f, t, o->precond, st->W, o->cg_max_iter + 1));
  Scratch S(c);
  T* Bm = S.get<T>((size_t)n * E.ld);
  T* Um = S.get<T>((size_t)n * E.ld);
  if (!Bm || !Um) return fail(c, VL_ERR_OOM, "workspace exhausted (vl_pcg_solve)");
  VL_CUDA(c, cudaMemsetAsync(Bm, 0, sizeof(T) * n * E.ld, c->stream));
  to_storage_kernel<T><<<grid_for(c, (int64_t)n * E.ld), 256, 0, VL_STREAM(c)>>>(n, t, E.ld, f->s2u, Rd, Bm);
  VL_CUDA(c, cudaGetLastError());
  int used = 0;
  VL_TRY(E.pcg(Bm, Um, o->cg_tol, o->cg_max_iter, &used));
  from_storage_kernel<T><<<grid_for(c, (int64_t)n * t), 256, 0, VL_STREAM(c)>>>(n, t, E.ld, f->s2u, Um, Ud);
  VL_CUDA(c, cudaGetLastError());
  std::vector<int> it;
  std::vector<double> rel;
  VL_TRY(E.column_stats(it, rel));
  if (iters) std::copy(it.begin(), it.end(), iters);
  if (relres) std::copy(rel.begin(), rel.end(), relres);
  if (lmax > 0 && (Td || To)) {
    std::vector<double> hd((size_t)t * E.lmax), ho((size_t)t * E.lmax);
    VL_CUDA(c, cudaMemcpyAsync(hd.data(), E.S.Tdiag, sizeof(double) * t * E.lmax, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(ho.data(), E.S.Toff, sizeof(double) * t * E.lmax, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < t; ++k)
      for (int l = 0; l < lmax; ++l) {
        const bool in = l < E.lmax;
        if (Td) Td[(size_t)k * lmax + l] = in ? hd[(size_t)k * E.lmax + l] : 0.0;
        if (To) To[(size_t)k * lmax + l] = in ? ho[(size_t)k * E.lmax + l] : 0.0;
      }
  }
  return VL_OK;
}

}  // namespace vl

using namespace vl;

struct vl_ctx : Ctx {};
struct vl_factor : Factor {};
struct vl_state : State {};

// ============================================================================== C ABI
extern "C" {

const char* vl_version(void) { return "vl 0.1.0 sm_103a"; }

void vl_opts_default(vl_opts* o) {
  if (!o) return;
  o->precision = VL_FP64;
  o->precond = VL_PREC_VADU;
  o->t = 50;
  o->k = 50;
  o->s = 100;
  o->cg_tol = 1e-6;
  o->cg_max_iter = 1000;
  o->newton_tol = 1e-9;
  o->newton_max_iter = 100;
  o->nugget = -1.0;
  o->seed = 1;
  o->lik_shape = 1.0;
  o->newton_eta_max = 0.1;
}

vl_status vl_ctx_create(int device, void* cuda_stream, void* workspace, size_t ws_bytes, vl_ctx** out) {
  if (!out || ws_bytes < (1u << 20)) return VL_ERR_INVALID_ARG;
  *out = nullptr;
  vl_ctx* c = new vl_ctx();
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  auto bail = [&](vl_status s) {
    if (c->owns_ws && c->ws) cudaFree(c->ws);
    if (c->pinned) cudaFreeHost(c->pinned);
    delete c;
    return s;
  };
  if (cudaSetDevice(device) != cudaSuccess) return bail(VL_ERR_CUDA);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return bail(VL_ERR_CUDA);
  c->num_sms = prop.multiProcessorCount;
  if (workspace) {
    c->ws = static_cast<char*>(workspace);
  } else {
    if (cudaMalloc(&c->ws, ws_bytes) != cudaSuccess) {
      cudaGetLastError();
      return bail(VL_ERR_OOM);
    }
    c->owns_ws = true;
  }
  c->arena.init(c->ws, ws_bytes);
  c->pinned_bytes = 1 << 16;
  if (cudaMallocHost(&c->pinned, c->pinned_bytes) != cudaSuccess) return bail(VL_ERR_CUDA);
  c->hstatus = reinterpret_cast<DevStatus*>(c->pinned + 1024);
  c->dstatus = static_cast<DevStatus*>(c->arena.alloc(sizeof(DevStatus)));
  c->gbar = static_cast<unsigned*>(c->arena.alloc(2 * sizeof(unsigned)));
  if (!c->dstatus || !c->gbar) return bail(VL_ERR_OOM);
  if (cudaMemsetAsync(c->dstatus, 0, sizeof(DevStatus), c->stream) != cudaSuccess) return bail(VL_ERR_CUDA);
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return bail(VL_ERR_CUDA);
  for (cudaEvent_t& e : c->ev_ring)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(VL_ERR_CUDA);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(VL_ERR_CUDA);
  *out = c;
  return VL_OK;
}

// A context lives until it has been destroyed and every factor, state and batch made on
// it has been destroyed too, in whatever order those calls come.
static void ctx_release(Ctx* cc);

}  // extern "C"
namespace vl {
void ctx_retain(Ctx* c) { ++c->refs; }
void ctx_release_ref(Ctx* c) { ctx_release(c); }
}  // namespace vl
extern "C" {

static void ctx_release(Ctx* cc) {
  if (--cc->refs > 0) return;
  vl_ctx* c = static_cast<vl_ctx*>(cc);
  cudaStreamSynchronize(c->stream);
  prof_release(c);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  for (cudaEvent_t e : c->ev_ring)
    if (e) cudaEventDestroy(e);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  if (c->pinned) cudaFreeHost(c->pinned);
  delete c;
}

void vl_ctx_destroy(vl_ctx* c) {
  if (!c || c->closed) return;
  c->closed = true;
  ctx_release(c);
}

const char* vl_last_error(const vl_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

vl_status vl_ctx_synchronize(vl_ctx* c) {
  if (!c) return VL_ERR_INVALID_ARG;
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status vl_profile_enable(vl_ctx* c, int enable) {
  if (!c) return VL_ERR_INVALID_ARG;
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  prof_drain(c);
  c->prof.on = enable != 0;
  c->prof.trace = enable >= 2;
  return VL_OK;
}

vl_status vl_profile_trace(vl_ctx* c, const char* cls, int t, long long* out, int cap, int* len, int* l_head,
                           int* l_tail) {
  if (!c || !cls) return VL_ERR_INVALID_ARG;
  auto it = c->prof.traces.find({cls, t});
  if (it == c->prof.traces.end()) {
    if (len) *len = 0;
    return VL_OK;
  }
  const int n = (int)it->second.size();
  if (len) *len = n;
  if (out)
    for (int i = 0; i < std::min(n, cap); ++i) out[i] = it->second[i];
  auto ct = c->prof.cuts[{cls, t}];
  if (l_head) *l_head = ct.first;
  if (l_tail) *l_tail = ct.second;
  return VL_OK;
}

vl_status vl_profile_read(vl_ctx* c, const char* cls, int t, double* ms, int64_t* launches, int reset) {
  if (!c) return VL_ERR_INVALID_ARG;
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  prof_drain(c);
  double tot = 0.0;
  int64_t cnt = 0;
  if (cls && std::string(cls) == "all") {
    cnt = c->launches;
  } else if (cls) {
    for (auto& kv : c->prof.acc) {
      if (kv.first.first == cls && (t == 0 || kv.first.second == t)) {
        tot += kv.second.ms;
        cnt += kv.second.launches;
      }
    }
  }
  if (ms) *ms = tot;
  if (launches) *launches = cnt;
  if (reset) {
    c->prof.acc.clear();
    c->launches = 0;
  }
  return VL_OK;
}

vl_status vl_ctx_set_wait_limit(vl_ctx* c, long long cycles) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (cycles < 0) return fail(c, VL_ERR_INVALID_ARG, "wait limit must be >= 0 cycles");
  set_wait_limit_kernel<<<1, 1, 0, VL_STREAM(c)>>>(c->dstatus, cycles);
  VL_CUDA(c, cudaGetLastError());
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status vl_ctx_wait_probe(vl_ctx* c) {
  if (!c) return VL_ERR_INVALID_ARG;
  Scratch S(c);
  int* flag = S.get<int>(1);
  if (!flag) return fail(c, VL_ERR_OOM, "workspace exhausted (wait probe)");
  VL_CUDA(c, cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  VL_CUDA(c, status_clear(c));
  wait_probe_kernel<<<1, 32, 0, VL_STREAM(c)>>>(flag, c->dstatus);
  VL_CUDA(c, cudaGetLastError());
  return check_dev_status(c, "wait probe");
}

vl_status vl_ctx_set_autotune(vl_ctx* c, int enable) {
  if (!c) return VL_ERR_INVALID_ARG;
  c->autotune = enable != 0;
  return VL_OK;
}

size_t vl_tune_report(char* buf, size_t len) {
  std::string out = "[";
  {
    std::lock_guard<std::mutex> lk(tuner().mu);
    bool first = true;
    for (auto& kv : tuner().best) {
      const TuneKey& k = kv.first;
      char head[160];
      snprintf(head, sizeof head, "%s{\"device\": %d, \"class\": %d, \"value_bytes\": %d, \"ld\": %d, \"log2_n\": %d, "
               "\"choice\": %d, \"ms\": [", first ? "" : ", ", k.device, k.cls, k.vbytes, k.ld, k.nbucket, kv.second);
      out += head;
      const std::vector<float>& ms = tuner().times[k];
      for (size_t i = 0; i < ms.size(); ++i) {
        char v[32];
        snprintf(v, sizeof v, "%s%.4f", i ? ", " : "", ms[i]);
        out += v;
      }
      out += "]}";
      first = false;
    }
  }
  out += "]";
  if (buf && len > 0) {
    const size_t k = std::min(len - 1, out.size());
    std::memcpy(buf, out.data(), k);
    buf[k] = 0;
  }
  return out.size() + 1;
}

void vl_tune_reset(void) {
  std::lock_guard<std::mutex> lk(tuner().mu);
  tuner().best.clear();
  tuner().times.clear();
}

vl_status vl_ctx_set_solve_form(vl_ctx* c, int form) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (form < VL_SOLVE_AUTO || form > VL_SOLVE_TILE) return fail(c, VL_ERR_INVALID_ARG, "unknown solve form");
  c->solve_form = form;
  return VL_OK;
}

vl_status vl_ctx_mem(const vl_ctx* c, size_t* in_use, size_t* peak) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (in_use) *in_use = c->arena.in_use();
  if (peak) *peak = c->arena.peak();
  return VL_OK;
}

// --------------------------------------------------------------------------- neighbours
vl_status vl_knn_prev(vl_ctx* c, const double* locs, int64_t n, int m, int32_t* N_out) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (n < 0 || n > INT32_MAX / 2 || m < 0 || m > 64 || (!locs && n > 0) || (!N_out && n > 0 && m > 0))
    return fail(c, VL_ERR_INVALID_ARG, "vl_knn_prev: invalid argument");
  if (n == 0 || m == 0) return VL_OK;
  Scratch S(c);
  const double* dl;
  VL_TRY(stage_in(c, S, locs, (size_t)n * 2, &dl));
  int32_t* N = S.get<int32_t>((size_t)n * m);
  if (!N) return fail(c, VL_ERR_OOM, "workspace exhausted (kNN)");
  VL_TRY(knn_prev_dev(c, dl, n, m, N));
  return stage_out(c, N, N_out, (size_t)n * m);
}

vl_status vl_knn_cross(vl_ctx* c, const double* train, int64_t n, const double* test, int64_t np, int m,
                       int32_t* N_out) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (n < 0 || np < 0 || m < 0 || m > 64 || (!train && n > 0) || (!test && np > 0) || (!N_out && np > 0 && m > 0))
    return fail(c, VL_ERR_INVALID_ARG, "vl_knn_cross: invalid argument");
  if (np == 0 || m == 0) return VL_OK;
  Scratch S(c);
  const double *dt, *dq;
  VL_TRY(stage_in(c, S, train, (size_t)n * 2, &dt));
  VL_TRY(stage_in(c, S, test, (size_t)np * 2, &dq));
  int32_t* N = S.get<int32_t>((size_t)np * m);
  if (!N) return fail(c, VL_ERR_OOM, "workspace exhausted (kNN)");
  VL_TRY(knn_cross_dev(c, dt, n, dq, np, m, N));
  return stage_out(c, N, N_out, (size_t)np * m);
}

// --------------------------------------------------------------------------- factor
static double nugget_of(const vl_opts* o, double sigma2) {
  return (o && o->nugget >= 0.0) ? o->nugget : 1e-10 * sigma2;
}

vl_status vl_factor_refit(vl_factor* f, double sigma2, double range, const vl_opts* opts) {
  if (!f) return VL_ERR_INVALID_ARG;
  Ctx* c = f->ctx;
  if (!(sigma2 > 0) || !(range > 0)) return fail(c, VL_ERR_INVALID_ARG, "sigma2 and range must be > 0");
  f->sigma2 = sigma2;
  f->rho = range;
  f->nugget = nugget_of(opts, sigma2);
  lrac_drop(f);   // L_k belongs to the old covariance parameters
  VL_CUDA(c, status_clear(c));
  VL_TRY(factor_rows(c, f->n, f->m, f->locs_s, f->locs_s, f->nbr, f->cov, f->sigma2, f->rho, f->nugget, f->A64, f->D64,
                     f->s2v));
  VL_TRY(refresh_transpose_values(f));
  return check_dev_status(c, "Vecchia factor");
}

vl_status vl_build_factor(vl_ctx* c, const double* locs, int64_t n, const int32_t* order, int cov, double sigma2,
                          double range, int m, const vl_opts* opts, vl_factor** out) {
  if (!c) return VL_ERR_INVALID_ARG;
  if (!out || !locs || n < 1 || n > (1LL << 30) || m < 0 || m > 64 || (cov != VL_COV_EXPONENTIAL && cov != VL_COV_MATERN15))
    return fail(c, VL_ERR_INVALID_ARG, "vl_build_factor: invalid argument");
  if (!(sigma2 > 0) || !(range > 0)) return fail(c, VL_ERR_INVALID_ARG, "sigma2 and range must be > 0");
  *out = nullptr;
  vl_factor* f = new vl_factor();
  f->ctx = c;
  f->mem.ctx = c;
  f->n = n;
  f->m = m;
  f->cov = cov;
  auto bail = [&](vl_status s) {
    f->mem.free_all();
    delete f;
    return s;
  };
  Scratch S(c);
  const double* dl;
  const int32_t* dord = nullptr;
  vl_status st = stage_in(c, S, locs, (size_t)n * 2, &dl);
  if (st == VL_OK && order) st = stage_in(c, S, order, (size_t)n, &dord);
  if (st != VL_OK) return bail(st);
  const int64_t nm = n * (int64_t)m;
  f->locs_v = f->mem.get<double>((size_t)n * 2);
  f->locs_s = f->mem.get<double>((size_t)n * 2);
  f->s2v = f->mem.get<int32_t>(n);
  f->v2s = f->mem.get<int32_t>(n);
  f->s2u = f->mem.get<int32_t>(n);
  f->u2s = f->mem.get<int32_t>(n);
  f->nbr = f->mem.get<int32_t>(std::max<int64_t>(nm, 1));
  f->A64 = f->mem.get<double>(std::max<int64_t>(nm, 1));
  f->A32 = f->mem.get<float>(std::max<int64_t>(nm, 1));
  f->D64 = f->mem.get<double>(n);
  f->lev_fwd = f->mem.get<int32_t>(n);
  f->lev_bwd = f->mem.get<int32_t>(n);
  f->task_fwd = f->mem.get<int32_t>(n);
  f->task_bwd = f->mem.get<int32_t>(n);
  if (!f->locs_v || !f->locs_s || !f->s2v || !f->v2s || !f->s2u || !f->u2s || !f->nbr || !f->A64 || !f->A32 ||
      !f->D64 || !f->lev_fwd || !f->lev_bwd || !f->task_fwd || !f->task_bwd)
    return bail(fail(c, VL_ERR_OOM, "workspace exhausted (factor)"));
  gather2_kernel<<<(int)((n + 255) / 256), 256, 0, VL_STREAM(c)>>>((int)n, dl, dord, f->locs_v);
  int32_t* Nv = S.get<int32_t>(std::max<int64_t>(nm, 1));
  if (!Nv) return bail(fail(c, VL_ERR_OOM, "workspace exhausted (neighbours)"));
  if (m > 0) {
    st = knn_prev_dev(c, f->locs_v, n, m, Nv);
    if (st != VL_OK) return bail(st);
  }
  st = build_graph_impl(f, Nv, f->locs_v, dord);
  if (st != VL_OK) return bail(st);
  st = vl_factor_refit(f, sigma2, range, opts);
  if (st != VL_OK) return bail(st);
  ++c->refs;
  *out = f;
  return VL_OK;
}

vl_status vl_factor_export(const vl_factor* fc, int32_t* N, double* A, double* D, int32_t* lev_fwd, int32_t* lev_bwd) {
  if (!fc) return VL_ERR_INVALID_ARG;
  vl_factor* f = const_cast<vl_factor*>(fc);
  Ctx* c = f->ctx;
  const int64_t n = f->n, nm = n * f->m;
  Scratch S(c);
  int32_t* dN = N ? S.get<int32_t>(std::max<int64_t>(nm, 1)) : nullptr;
  double* dA = A ? S.get<double>(std::max<int64_t>(nm, 1)) : nullptr;
  double* dD = D ? S.get<double>(n) : nullptr;
  int32_t* dlf = lev_fwd ? S.get<int32_t>(n) : nullptr;
  int32_t* dlb = lev_bwd ? S.get<int32_t>(n) : nullptr;
  if ((N && !dN) || (A && !dA) || (D && !dD) || (lev_fwd && !dlf) || (lev_bwd && !dlb))
    return fail(c, VL_ERR_OOM, "workspace exhausted (export)");
  export_kernel<<<(int)((n + 255) / 256), 256, 0, VL_STREAM(c)>>>((int)n, f->m, f->s2v, f->nbr, f->A64, f->D64,
                                                               f->lev_fwd, f->lev_bwd, dN, dA, dD, dlf, dlb);
  VL_CUDA(c, cudaGetLastError());
  VL_TRY(stage_out(c, dN, N, nm));
  VL_TRY(stage_out(c, dA, A, nm));
  VL_TRY(stage_out(c, dD, D, n));
  VL_TRY(stage_out(c, dlf, lev_fwd, n));
  VL_TRY(stage_out(c, dlb, lev_bwd, n));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

vl_status vl_factor_info(const vl_factor* f, int64_t* n, int* m, int* nf, int* nb) {
  if (!f) return VL_ERR_INVALID_ARG;
  if (n) *n = f->n;
  if (m) *m = f->m;
  if (nf) *nf = f->nlev_fwd;
  if (nb) *nb = f->nlev_bwd;
  return VL_OK;
}

void vl_factor_destroy(vl_factor* f) {
  if (!f) return;
  Ctx* c = f->ctx;
  cudaStreamSynchronize(c->stream);
  lrac_drop(f);
  f->mem.free_all();
  delete f;
  ctx_release(c);
}

// --------------------------------------------------------------------------- mode
vl_status vl_find_mode(vl_factor* f, int lik, const double* y, const double* F, const vl_opts* opts,
                       double* mode_out, vl_state** out) {
  if (!f) return VL_ERR_INVALID_ARG;
  Ctx* c = f->ctx;
  if (!out || !y || (lik != VL_LIK_BERNOULLI_LOGIT && lik != VL_LIK_POISSON_LOG && lik != VL_LIK_GAMMA_LOG))
    return fail(c, VL_ERR_INVALID_ARG, "vl_find_mode: invalid argument");
  VL_TRY(check_opts(c, opts));
  if (lik == VL_LIK_GAMMA_LOG && !(opts->lik_shape > 0.0 && std::isfinite(opts->lik_shape)))
    return fail(c, VL_ERR_INVALID_ARG, "vl_find_mode: the gamma shape must be > 0");
  *out = nullptr;
  const int n = (int)f->n;
  cudaEventRecord(c->ev0, c->stream);
  vl_state* st = new vl_state();
  st->f = f;
  st->ctx = c;
  st->mem.ctx = c;
  st->lik = lik;
  st->shape = lik == VL_LIK_GAMMA_LOG ? opts->lik_shape : 1.0;
  auto bail = [&](vl_status s) {
    st->mem.free_all();
    delete st;
    return s;
  };
  st->y = st->mem.get<double>(n);
  st->F = st->mem.get<double>(n);
  st->b = st->mem.get<double>(n);
  st->W = st->mem.get<double>(n);
  if (!st->y || !st->F || !st->b || !st->W) return bail(fail(c, VL_ERR_OOM, "workspace exhausted (state)"));
  vl_status s;
  {
    Scratch S(c);
    const double *dy, *dF = nullptr;
    s = stage_in(c, S, y, n, &dy);
    if (s == VL_OK && F) s = stage_in(c, S, F, n, &dF);
    if (s != VL_OK) return bail(s);
    to_storage_kernel<double><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 1, 1, f->s2u, dy, st->y);
    if (dF)
      to_storage_kernel<double><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 1, 1, f->s2u, dF, st->F);
    else
      cudaMemsetAsync(st->F, 0, sizeof(double) * n, c->stream);
    cudaMemsetAsync(st->b, 0, sizeof(double) * n, c->stream);
    if (cudaGetLastError() != cudaSuccess) return bail(fail(c, VL_ERR_CUDA, "staging y/F"));
    // responses in the likelihood's support, finite offsets
    int* bad = S.get<int>(2);
    if (!bad) return bail(fail(c, VL_ERR_OOM, "workspace exhausted (input check)"));
    cudaMemsetAsync(bad, 0x7f, sizeof(int), c->stream);
    check_inputs_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, lik_spec(st), st->y, st->F, bad);
    int hb[2] = {0, 0};
    double hv[2] = {0.0, 0.0};
    if (cudaMemcpyAsync(hb, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
      return bail(fail(c, VL_ERR_CUDA, "input check"));
    if (hb[0] >= 0 && hb[0] < n) {
      cudaMemcpyAsync(&hb[1], f->s2u + hb[0], sizeof(int), cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(&hv[0], st->y + hb[0], sizeof(double), cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(&hv[1], st->F + hb[0], sizeof(double), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
      char buf[256];
      snprintf(buf, sizeof buf,
               "vl_find_mode: y[%d] = %g (offset %g) is not a finite value in the support of the likelihood", hb[1],
               hv[0], hv[1]);
      return bail(fail(c, VL_ERR_INVALID_ARG, buf));
    }
  }
  // Newton iterations (Eq. newton)
  std::vector<vl_stats> ss;
  std::vector<char> conv;
  s = newton_run(st, opts, ss, conv);
  if (s != VL_OK) return bail(s);
  if (mode_out) {
    Scratch S(c);
    double* mu = S.get<double>(n);
    if (!mu) return bail(fail(c, VL_ERR_OOM, "workspace exhausted (mode out)"));
    from_storage_kernel<double><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 1, 1, f->s2u, st->b, mu);
    s = stage_out(c, mu, mode_out, n);
    if (s != VL_OK) return bail(s);
  }
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(fail(c, VL_ERR_CUDA, "sync"));
  st->mode_stats = ss[0];
  ++c->refs;
  *out = st;
  if (!conv[0]) return fail(c, VL_ERR_NOT_CONVERGED, "Newton reached newton_max_iter");
  return VL_OK;
}

vl_status vl_state_stats(const vl_state* s, vl_stats* out) {
  if (!s || !out) return VL_ERR_INVALID_ARG;
  *out = s->mode_stats;
  return VL_OK;
}

void vl_state_destroy(vl_state* s) {
  if (!s) return;
  Ctx* c = s->ctx;
  cudaStreamSynchronize(c->stream);
  s->mem.free_all();
  delete s;
  ctx_release(c);
}

// --------------------------------------------------------------------------- L^VLA
vl_status vl_log_marglik(vl_state* st, const vl_opts* o, double* lml, double* logdet, vl_stats* stats) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  VL_TRY(check_opts(c, o));
  if (!lml) return fail(c, VL_ERR_INVALID_ARG, "lml is NULL");
  const int t = o->t;
  VL_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  SlqOut q;
  if (o->precision == VL_FP64)
    VL_TRY(slq_run<double>(st, o, q));
  else
    VL_TRY(slq_run<float>(st, o, q));
  LmlOut L;
  VL_TRY(lml_assemble(st, o, q, L));
  *lml = L.lml[0];
  if (logdet) *logdet = L.logdet[0];
  st->h_gammas.assign(q.gam.begin(), q.gam.begin() + t);
  st->last_t = t;
  VL_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  VL_CUDA(c, cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (stats) {
    *stats = vl_stats{};
    stats->cg_calls = 1;
    stats->cg_iters_max = *std::max_element(q.iters.begin(), q.iters.end());
    stats->cg_iters_total = (int)(std::accumulate(q.iters.begin(), q.iters.end(), (int64_t)0) + q.extra_iters);
    stats->cg_relres_max = *std::max_element(q.relres.begin(), q.relres.end());
    stats->true_relres_max = q.true_rel[0];
    stats->probe_relres_max = q.true_rel[0];
    stats->probe_refine_steps = q.passes[0];
    stats->slq_mean = L.mean[0];
    stats->slq_stderr = L.se[0];
    stats->logdet = L.logdet[0];
    stats->ms_total = ms;
  }
  return VL_OK;
}

vl_status vl_slq_gammas(const vl_state* st, double* gammas, int t) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  if (!gammas || t != st->last_t || (int)st->h_gammas.size() != t)
    return fail(c, VL_ERR_STATE, "vl_slq_gammas: no SLQ result of that size");
  if (is_device_ptr(gammas)) {
    VL_CUDA(c, cudaMemcpyAsync(gammas, st->h_gammas.data(), sizeof(double) * t, cudaMemcpyHostToDevice, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
  } else {
    std::memcpy(gammas, st->h_gammas.data(), sizeof(double) * t);
  }
  return VL_OK;
}

// --------------------------------------------------------------------------- prediction
vl_status vl_pred_var(vl_state* st, const double* test_locs, int64_t np, const double* Fp, const vl_opts* o,
                      double* mean, double* var, vl_stats* stats) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  VL_TRY(check_opts(c, o));
  if (np < 0 || (np > 0 && !test_locs) || np > (1LL << 30)) return fail(c, VL_ERR_INVALID_ARG, "vl_pred_var: invalid argument");
  if (np == 0) return VL_OK;
  Factor* f = st->f;
  const int m = f->m, n = (int)f->n;
  VL_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  vl_stats loc{};
  Scratch S(c);
  const double *dq, *dF = nullptr;
  VL_TRY(stage_in(c, S, test_locs, (size_t)np * 2, &dq));
  if (Fp) VL_TRY(stage_in(c, S, Fp, (size_t)np, &dF));
  const int64_t npm = np * (int64_t)std::max(m, 1);
  int32_t* Np = S.get<int32_t>(npm);
  double* Ap = S.get<double>(npm);
  double* Dp = S.get<double>(np);
  double* dmean = S.get<double>(np);
  double* dvar = S.get<double>(np);
  if (!Np || !Ap || !Dp || !dmean || !dvar) return fail(c, VL_ERR_OOM, "workspace exhausted (prediction)");
  if (m > 0) {
    VL_TRY(knn_cross_dev(c, f->locs_v, n, dq, np, m, Np));   // Vecchia indices, Section 4.1
    translate_kernel<<<grid_for(c, npm), 256, 0, VL_STREAM(c)>>>(npm, f->v2s, Np);
    VL_CUDA(c, cudaGetLastError());
  }
  VL_CUDA(c, status_clear(c));
  VL_TRY(factor_rows(c, np, m, dq, f->locs_s, Np, f->cov, f->sigma2, f->rho, f->nugget, Ap, Dp, nullptr));
  VL_TRY(check_dev_status(c, "prediction rows"));
  VL_TRY(pred_from_rows(st, o, np, m, Np, Ap, Dp, dF, dmean, var ? dvar : nullptr, &loc));
  VL_TRY(stage_out(c, dmean, mean, np));
  VL_TRY(stage_out(c, dvar, var, np));
  VL_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  VL_CUDA(c, cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  loc.ms_total = ms;
  if (stats) *stats = loc;
  return VL_OK;
}

vl_status vl_pred_var_lanczos(vl_state* st, const double* test_locs, int64_t np, const double* Fp, int k, int precond_l,
                              double* mean, double* var, vl_stats* stats) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int m = f->m, n = (int)f->n;
  if (np < 0 || (np > 0 && !test_locs) || np > (1LL << 30) || k < 1)
    return fail(c, VL_ERR_INVALID_ARG, "vl_pred_var_lanczos: invalid argument");
  if (precond_l != 1)
    return fail(c, VL_ERR_INVALID_ARG, "vl_pred_var_lanczos: only the Lanczos preconditioner P_L1 is available");
  if (f->nseg != 1) return fail(c, VL_ERR_INVALID_ARG, "vl_pred_var_lanczos: single problems only");
  if (np == 0) return VL_OK;
  k = std::min(k, n);
  VL_CUDA(c, cudaEventRecord(c->ev0, c->stream));
  Scratch S(c);
  const double *dq, *dF = nullptr;
  VL_TRY(stage_in(c, S, test_locs, (size_t)np * 2, &dq));
  if (Fp) VL_TRY(stage_in(c, S, Fp, (size_t)np, &dF));
  const int64_t npm = np * (int64_t)std::max(m, 1);
  int32_t* Np = S.get<int32_t>(npm);
  double* Ap = S.get<double>(npm);
  double* Dp = S.get<double>(np);
  double* dmean = S.get<double>(np);
  double* dvar = S.get<double>(np);
  if (!Np || !Ap || !Dp || !dmean || !dvar) return fail(c, VL_ERR_OOM, "workspace exhausted (prediction)");
  if (m > 0) {
    VL_TRY(knn_cross_dev(c, f->locs_v, n, dq, np, m, Np));   // Vecchia indices, Section 4.1
    translate_kernel<<<grid_for(c, npm), 256, 0, VL_STREAM(c)>>>(npm, f->v2s, Np);
    VL_CUDA(c, cudaGetLastError());
  }
  VL_CUDA(c, status_clear(c));
  VL_TRY(factor_rows(c, np, m, dq, f->locs_s, Np, f->cov, f->sigma2, f->rho, f->nugget, Ap, Dp, nullptr));
  VL_TRY(check_dev_status(c, "prediction rows"));
  const int pg = (int)((np * 32 + 255) / 256);
  pred_kernel<double><<<pg, 256, 0, VL_STREAM(c)>>>((int)np, m, Np, Ap, Dp, dF, st->b, nullptr, 0, 1, dmean, nullptr);
  VL_CUDA(c, cudaGetLastError());
  int kk = 0;
  if (var) {
    // CSR of the test neighbours by training row (entries in increasing (p, slot) order)
    std::vector<int32_t> hN;
    VL_TRY(to_host(c, hN, (const int32_t*)Np, (size_t)(m > 0 ? npm : 0)));
    std::vector<int32_t> rp(n + 1, 0), ent;
    for (int64_t e = 0; e < (int64_t)hN.size(); ++e)
      if (hN[e] >= 0) ++rp[hN[e] + 1];
    for (int j = 0; j < n; ++j) rp[j + 1] += rp[j];
    ent.resize(rp[n]);
    std::vector<int32_t> fill(rp.begin(), rp.end() - 1);
    for (int64_t e = 0; e < (int64_t)hN.size(); ++e)
      if (hN[e] >= 0) ent[fill[hN[e]]++] = (int32_t)e;
    int32_t* drp = S.get<int32_t>(n + 1);
    int32_t* dent = S.get<int32_t>(std::max<size_t>(ent.size(), 1));
    Engine<double> E(c);
    VL_TRY(E.init(f, 1, VL_PREC_VADU, st->W, 0));
    const int rows = 4096, nch = (n + rows - 1) / rows;
    double* Q = S.get<double>((size_t)n * k);
    double* sv = S.get<double>(n);
    double* v = S.get<double>(n);
    double* t1 = S.get<double>(n);
    double* t2 = S.get<double>(n);
    double* w = S.get<double>(n);
    double* h = S.get<double>(k);
    double* part = S.get<double>((size_t)nch * k);
    if (!drp || !dent || !Q || !sv || !v || !t1 || !t2 || !w || !h || !part)
      return fail(c, VL_ERR_OOM, "workspace exhausted (Lanczos)");
    VL_TRY(to_device(c, drp, rp));
    VL_TRY(to_device(c, dent, ent));
    // s = S^{1/2} = (W + D^{-1})^{-1/2}
    diag_fn_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 0, st->W, f->D64, t1);
    VL_CUDA(c, cudaGetLastError());
    {   // sv = 1 / sqrt(W + 1/D)
      std::vector<double> hs;
      VL_TRY(to_host(c, hs, (const double*)t1, (size_t)n));
      for (double& x : hs) x = 1.0 / x;
      VL_TRY(to_device(c, sv, hs));
    }
    // q_0 = P^{-1/2} v / ||P^{-1/2} v||, v = the mean of the columns of B_po^T
    lanczos_start_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, drp, dent, Ap, 1.0 / (double)np, v);
    VL_TRY(E.solveBt(v, nullptr, t1));
    lanczos_scale_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, sv, t1, 1.0, w);
    auto norm = [&](const double* x, double* out) -> vl_status {
      VL_TRY(E.coldot(x, x, nullptr, E.red));
      std::vector<double> hr;
      VL_TRY(to_host(c, hr, (const double*)E.red, 1));
      *out = std::sqrt(hr[0]);
      return VL_OK;
    };
    // h[0 .. ncol) = Q[:, c0 .. c0 + ncol)^T x
    auto qtw = [&](int c0, int ncol, const double* x) -> vl_status {
      lanczos_qtw_kernel<<<dim3(nch, ncol), 256, 0, VL_STREAM(c)>>>(n, ncol, rows, Q + (size_t)c0 * n, x, part);
      lanczos_sum_kernel<<<(ncol + 255) / 256, 256, 0, VL_STREAM(c)>>>(nch, ncol, part, h);
      VL_CUDA(c, cudaGetLastError());
      return VL_OK;
    };
    double nrm = 0.0;
    VL_TRY(norm(w, &nrm));
    if (!(nrm > 0.0)) return fail(c, VL_ERR_INVALID_ARG, "vl_pred_var_lanczos: the start vector is zero");
    lanczos_scale_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, nullptr, w, nrm, Q);
    std::vector<double> alpha, beta;
    for (int j = 0; j < k; ++j) {
      double* qj = Q + (size_t)j * n;
      // w = M q_j = S^{1/2} B^{-T} A B^{-1} S^{1/2} q_j
      VL_TRY(E.solveB(qj, sv, t1));
      VL_TRY(E.opA(t1, t2));
      VL_TRY(E.solveBt(t2, nullptr, t1));
      lanczos_scale_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, sv, t1, 1.0, w);
      VL_TRY(qtw(j, 1, w));
      std::vector<double> ha;
      VL_TRY(to_host(c, ha, (const double*)h, 1));
      alpha.push_back(ha[0]);
      for (int pass = 0; pass < 2; ++pass) {   // full reorthogonalisation, twice
        VL_TRY(qtw(0, j + 1, w));
        lanczos_axpy_kernel<<<grid_for(c, n), 256, sizeof(double) * (j + 1), VL_STREAM(c)>>>(n, j + 1, Q, h, w);
        VL_CUDA(c, cudaGetLastError());
      }
      double bj = 0.0;
      VL_TRY(norm(w, &bj));
      kk = j + 1;
      if (j + 1 == k || !(bj > 1e-13 * std::max(std::fabs(alpha[0]), 1e-300))) break;
      beta.push_back(bj);
      lanczos_scale_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, nullptr, w, bj, Q + (size_t)(j + 1) * n);
    }
    // T = L diag(d) L^T
    std::vector<double> d(kk), l(std::max(kk - 1, 1), 0.0);
    d[0] = alpha[0];
    for (int i = 0; i + 1 < kk; ++i) {
      l[i] = beta[i] / d[i];
      d[i + 1] = alpha[i + 1] - l[i] * beta[i];
    }
    for (double x : d)
      if (!(x > 0.0)) return fail(c, VL_ERR_NOT_SPD, "vl_pred_var_lanczos: the Lanczos tridiagonal is not positive definite");
    double* dd = S.get<double>(kk);
    double* dl = S.get<double>(std::max(kk - 1, 1));
    double* Z = S.get<double>((size_t)np * kk);
    if (!dd || !dl || !Z) return fail(c, VL_ERR_OOM, "workspace exhausted (Lanczos)");
    VL_TRY(to_device(c, dd, d));
    VL_TRY(to_device(c, dl, l));
    // U = B^{-1} S^{1/2} Q in blocks of at most 128 columns, then z_p = U^T B_po^T e_p
    for (int c0 = 0; c0 < kk; c0 += 128) {
      const int kc = std::min(128, kk - c0);
      Engine<double> Ek(c);
      VL_TRY(Ek.init(f, kc, VL_PREC_VADU, st->W, 0, /*ops_only=*/true));
      double* X = S.get<double>((size_t)n * Ek.ld);
      double* U = S.get<double>((size_t)n * Ek.ld);
      if (!X || !U) return fail(c, VL_ERR_OOM, "workspace exhausted (Lanczos blocks)");
      lanczos_rows_kernel<<<grid_for(c, (int64_t)n * Ek.ld), 256, 0, VL_STREAM(c)>>>(n, kc, Ek.ld, c0, sv, Q, X);
      VL_TRY(Ek.solveB(X, nullptr, U));
      lanczos_gather_kernel<<<(unsigned)np, 128, 0, VL_STREAM(c)>>>((int)np, m, kc, Ek.ld, c0, kk, Np, Ap, U, Z);
      VL_CUDA(c, cudaGetLastError());
      VL_CUDA(c, cudaStreamSynchronize(c->stream));
      c->arena.release(U);
      c->arena.release(X);
      S.blocks.erase(std::remove_if(S.blocks.begin(), S.blocks.end(), [&](void* p) { return p == U || p == X; }),
                     S.blocks.end());
    }
    lanczos_quad_kernel<<<grid_for(c, np), 256, 0, VL_STREAM(c)>>>((int)np, kk, Z, dl, dd, Dp, dvar);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(check_dev_status(c, "Lanczos predictive variances"));
  }
  VL_TRY(stage_out(c, dmean, mean, np));
  VL_TRY(stage_out(c, dvar, var, np));
  VL_CUDA(c, cudaEventRecord(c->ev1, c->stream));
  VL_CUDA(c, cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  if (stats) {
    *stats = vl_stats{};
    stats->cg_iters_max = kk;
    stats->ms_total = ms;
  }
  return VL_OK;
}

// --------------------------------------------------------------------------- building blocks
vl_status vl_apply(vl_state* st, int op, const double* X, int t, const vl_opts* o, double* Y) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  VL_TRY(check_opts(c, o));
  if (!X || !Y || t < 1 || t > 256) return fail(c, VL_ERR_INVALID_ARG, "vl_apply: invalid argument");
  const int64_t nt = st->f->n * (int64_t)t;
  Scratch S(c);
  const double* dX;
  VL_TRY(stage_in(c, S, X, nt, &dX));
  double* dY = S.get<double>(nt);
  if (!dY) return fail(c, VL_ERR_OOM, "workspace exhausted (vl_apply)");
  if (o->precision == VL_FP64)
    VL_TRY(apply_op<double>(st, op, dX, t, o, dY));
  else
    VL_TRY(apply_op<float>(st, op, dX, t, o, dY));
  return stage_out(c, dY, Y, nt);
}

vl_status vl_pcg_solve(vl_state* st, const double* RHS, int t, const vl_opts* o, double* U, int lmax, double* T_diag,
                       double* T_off, int* iters, double* relres) {
  if (!st) return VL_ERR_INVALID_ARG;
  Ctx* c = st->ctx;
  VL_TRY(check_opts(c, o));
  if (!RHS || !U || t < 1 || t > 256 || lmax < 0) return fail(c, VL_ERR_INVALID_ARG, "vl_pcg_solve: invalid argument");
  const int64_t nt = st->f->n * (int64_t)t;
  Scratch S(c);
  const double* dR;
  VL_TRY(stage_in(c, S, RHS, nt, &dR));
  double* dU = S.get<double>(nt);
  if (!dU) return fail(c, VL_ERR_OOM, "workspace exhausted (vl_pcg_solve)");
  if (o->precision == VL_FP64)
    VL_TRY(pcg_op<double>(st, dR, t, o, dU, lmax, T_diag, T_off, iters, relres));
  else
    VL_TRY(pcg_op<float>(st, dR, t, o, dU, lmax, T_diag, T_off, iters, relres));
  return stage_out(c, dU, U, nt);
}

vl_status vl_lrac_export(vl_factor* f, int k, int32_t* piv, double* L) {
  if (!f) return VL_ERR_INVALID_ARG;
  Ctx* c = f->ctx;
  VL_TRY(lrac_build(f, k));
  const int n = (int)f->n;
  Scratch S(c);
  if (L) {
    double* dL = S.get<double>((size_t)n * k);
    if (!dL) return fail(c, VL_ERR_OOM, "workspace exhausted (LRAC export)");
    lrac_export_kernel<<<grid_for(c, (int64_t)n * k), 256, 0, VL_STREAM(c)>>>(n, k, f->s2u, f->L64, dL);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(stage_out(c, dL, L, (size_t)n * k));
  }
  if (piv) VL_TRY(stage_out(c, f->piv_v, piv, (size_t)k));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

}  // extern "C"
