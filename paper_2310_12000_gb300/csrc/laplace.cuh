// Newton's mode (Eq. newton), the SLQ log-determinant (Eq. def_SLQ) and the pieces of L^VLA
// (Eqs. VLA_loss, logdetsplit) for one problem or for a batch of independent problems merged
// into one block-diagonal system. A batch's problems are segments of the storage rows: every
// kernel runs once over all of them, reductions are per segment (segment-aligned blocks) and
// the Newton and PCG scalars are per segment and column, so each problem follows its own
// iteration while sharing the launches. A single problem is the case of one segment.
#pragma once

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "engine.cuh"

namespace vl {

// ----------------------------------------------------------------------------- kernels
// The likelihood of each row: one (lik, shape) for a single problem, per segment for a batch.
struct LikSpec {
  int lik;
  double shape;
  const int32_t* row_seg;   // storage row -> segment (null: one segment)
  const int* seg_lik;
  const double* seg_shape;
  __device__ __forceinline__ void at(int s, int& l, double& a) const {
    if (row_seg) {
      const int k = row_seg[s];
      l = seg_lik[k];
      a = seg_shape[k];
    } else {
      l = lik;
      a = shape;
    }
  }
};

// mu = F + b; g = d log p / d mu; W = -d^2 log p / d mu^2; logp; rhs = W b + g.
static __global__ void lik_seg_kernel(int n, LikSpec L, const double* __restrict__ y, const double* __restrict__ F,
                                      const double* __restrict__ b, double* __restrict__ W, double* __restrict__ g,
                                      double* __restrict__ rhs, double* __restrict__ logp) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int lik;
    double shape, lp, gg, ww;
    L.at(s, lik, shape);
    lik_terms(lik, shape, y[s], F[s] + b[s], lp, gg, ww);
    if (W) W[s] = ww;
    if (g) g[s] = gg;
    if (rhs) rhs[s] = ww * b[s] + gg;
    if (logp) logp[s] = lp;
  }
}

// Smallest storage row whose response lies outside its likelihood's support (Bernoulli:
// {0, 1}; Poisson: non-negative integers; gamma: y > 0) or whose y or offset is not finite.
static __global__ void check_inputs_kernel(int n, LikSpec L, const double* __restrict__ y,
                                           const double* __restrict__ F, int* __restrict__ first_bad) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    int lik;
    double shape;
    L.at(s, lik, shape);
    const double v = y[s];
    bool ok = isfinite(v) && isfinite(F[s]);
    if (lik == VL_LIK_BERNOULLI_LOGIT)
      ok = ok && (v == 0.0 || v == 1.0);
    else if (lik == VL_LIK_POISSON_LOG)
      ok = ok && v >= 0.0 && v == floor(v);
    else
      ok = ok && v > 0.0;
    if (!ok) atomicMin(first_bad, s);
  }
}

// Per segment sums of mode-selected terms over the reduction blocks of a t = 1 engine:
// mode 0: a; 1: log a; 2: log(b + 1 / a) (a = D, b = W: log det of the VADU preconditioner).
static __global__ void segsum_kernel(BlockRows br, int mode, const double* __restrict__ a,
                                     const double* __restrict__ b, double* __restrict__ partial, ReduceTail rt) {
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  double acc = 0.0;
  for (int s = r0 + threadIdx.y; s < r1; s += blockDim.y) {
    double v;
    if (mode == 0)
      v = a[s];
    else if (mode == 1)
      v = log(a[s]);
    else
      v = log(b[s] + 1.0 / a[s]);
    acc += v;
  }
  extern __shared__ double sh[];
  const double sum = block_col_sum(acc, sh);
  if (threadIdx.y == 0) {
    partial[blockIdx.x] = sum;
    __threadfence();
  }
  reduce_tail(br, 1, partial, rt);
}

// Per block: max |a - b| and max |a| (b may be null).
static __global__ void blockmax_kernel(BlockRows br, const double* __restrict__ a, const double* __restrict__ b,
                                       double* __restrict__ out) {
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  double m1 = 0.0, m2 = 0.0;
  for (int s = r0 + threadIdx.y; s < r1; s += blockDim.y) {
    m1 = fmax(m1, fabs(a[s] - (b ? b[s] : 0.0)));
    m2 = fmax(m2, fabs(a[s]));
  }
  __shared__ double s1[1024], s2[1024];
  s1[threadIdx.y] = m1;
  s2[threadIdx.y] = m2;
  __syncthreads();
  for (int h = blockDim.y >> 1; h > 0; h >>= 1) {
    if (threadIdx.y < h) {
      s1[threadIdx.y] = fmax(s1[threadIdx.y], s1[threadIdx.y + h]);
      s2[threadIdx.y] = fmax(s2[threadIdx.y], s2[threadIdx.y + h]);
    }
    __syncthreads();
  }
  if (threadIdx.y == 0) {
    out[2 * blockIdx.x] = s1[0];
    out[2 * blockIdx.x + 1] = s2[0];
  }
}

// Rows of segments whose flag is 0 set to zero (every column).
template <typename T>
__global__ void mask_rows_kernel(int n, int ld, const int32_t* __restrict__ row_seg, const int* __restrict__ keep,
                                 T* __restrict__ X) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld);
    if (!keep[row_seg ? row_seg[s] : 0]) X[e] = T(0);
  }
}

// Columns (segment k, column c) whose flag keep[k * t + c] is 0 set to zero.
template <typename T>
__global__ void mask_columns_kernel(int n, int t, int ld, const int32_t* __restrict__ row_seg,
                                    const int* __restrict__ keep, T* __restrict__ X) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    if (c < t && !keep[(row_seg ? row_seg[s] : 0) * t + c]) X[e] = T(0);
  }
}

// b_new <- b + 0.5 (b_new - b) on the rows of flagged segments
static __global__ void halve_seg_kernel(int n, const int32_t* __restrict__ row_seg, const int* __restrict__ flag,
                                        const double* __restrict__ b, double* __restrict__ bn) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    if (flag[row_seg ? row_seg[s] : 0]) bn[s] = b[s] + 0.5 * (bn[s] - b[s]);
}

// elementwise diagonal scalings used by probes / simulation
static __global__ void diag_fn_kernel(int n, int mode, const double* __restrict__ W, const double* __restrict__ D,
                                      double* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double v;
    if (mode == 0) v = sqrt(W[s] + 1.0 / D[s]);   // VADU P^{1/2} diagonal
    else if (mode == 1) v = 1.0 / sqrt(D[s]);     // D^{-1/2}
    else if (mode == 2) v = sqrt(W[s]);           // W^{1/2}
    else v = 1.0 / sqrt(W[s]);                    // W^{-1/2} (LRAC probes)
    out[s] = v;
  }
}

// ----------------------------------------------------------------------------- host helpers
template <typename V>
inline vl_status to_device(Ctx* c, V* dst, const std::vector<V>& src) {
  if (src.empty()) return VL_OK;
  VL_CUDA(c, cudaMemcpyAsync(dst, src.data(), sizeof(V) * src.size(), cudaMemcpyHostToDevice, c->stream));
  return VL_OK;
}
template <typename V>
inline vl_status to_host(Ctx* c, std::vector<V>& dst, const V* src, size_t count) {
  dst.resize(count);
  if (count == 0) return VL_OK;
  VL_CUDA(c, cudaMemcpyAsync(dst.data(), src, sizeof(V) * count, cudaMemcpyDeviceToHost, c->stream));
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

// Per segment sums (see segsum_kernel) through a t = 1 engine's reduction blocks.
inline vl_status seg_sums(Engine<double>& E, int mode, const double* a, const double* b, std::vector<double>& out) {
  Ctx* c = E.c;
  segsum_kernel<<<E.nblk, E.cb, E.csh, VL_STREAM(c)>>>(E.br, mode, a, b, E.partial, E.tail(EPI_NONE, E.red));
  VL_CUDA(c, cudaGetLastError());
  return to_host(c, out, (const double*)E.red, (size_t)E.nseg);
}

// Per segment max |a - b| and max |a|.
inline vl_status seg_absmax(Engine<double>& E, const double* a, const double* b, std::vector<double>& diff,
                            std::vector<double>& amax) {
  Ctx* c = E.c;
  blockmax_kernel<<<E.nblk, E.cb, 0, VL_STREAM(c)>>>(E.br, a, b, E.partial);
  VL_CUDA(c, cudaGetLastError());
  std::vector<double> h;
  VL_TRY(to_host(c, h, (const double*)E.partial, (size_t)2 * E.nblk));
  diff.assign(E.nseg, 0.0);
  amax.assign(E.nseg, 0.0);
  for (int q = 0; q < E.nblk; ++q) {
    const int k = E.h_blk_seg.empty() ? 0 : E.h_blk_seg[q];
    diff[k] = std::max(diff[k], h[2 * q]);
    amax[k] = std::max(amax[k], h[2 * q + 1]);
  }
  return VL_OK;
}

inline LikSpec lik_spec(const State* st) {
  return LikSpec{st->lik, st->shape, st->f->row_seg, st->d_seg_lik, st->d_seg_shape};
}

// psi_k(b) = sum_k log p(y | F + b) - b^T Sigma_tilde^{-1} b / 2 per segment, and its two parts.
inline vl_status psi_seg(State* st, Engine<double>& E1, double* lp, const double* b, std::vector<double>& psi,
                         std::vector<double>* logp_out = nullptr, std::vector<double>* quad_out = nullptr) {
  Ctx* c = st->ctx;
  const int n = (int)st->f->n;
  lik_seg_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, lik_spec(st), st->y, st->F, b, nullptr, nullptr, nullptr,
                                                           lp);
  VL_CUDA(c, cudaGetLastError());
  std::vector<double> logp, quad;
  VL_TRY(seg_sums(E1, 0, lp, nullptr, logp));
  VL_TRY(E1.opB(b, nullptr, E1.y));
  VL_TRY(E1.coldot(E1.y, E1.y, E1.Dinv, E1.red));
  VL_TRY(to_host(c, quad, (const double*)E1.red, (size_t)E1.nseg));
  psi.resize(E1.nseg);
  for (int k = 0; k < E1.nseg; ++k) psi[k] = logp[k] - 0.5 * quad[k];
  if (logp_out) *logp_out = logp;
  if (quad_out) *quad_out = quad;
  return VL_OK;
}

// Inexact Newton forcing terms (Eisenstat & Walker, SIAM J. Sci. Comput. 17, 1996, choice 2):
// eta_k = 0.9 (||g_k|| / ||g_{k-1}||)^2, kept at least 0.9 eta_{k-1}^2 while that exceeds 0.1,
// at most eta_max; eta_max while no history exists; 0 once a full solve is asked for.
struct Forcing {
  double eta_max = 0.0;    // 0: every solve to the full tolerance
  double g_prev = -1.0;    // ||grad psi|| at the previous Newton iterate (< 0: none yet)
  double eta_prev = -1.0;
  bool force_full = false;
  double next(double g) {
    double eta = eta_max;
    if (force_full || eta_max <= 0.0) {
      eta = 0.0;
    } else if (g_prev > 0.0) {
      eta = 0.9 * (g / g_prev) * (g / g_prev);
      if (eta_prev > 0.0 && 0.9 * eta_prev * eta_prev > 0.1) eta = std::max(eta, 0.9 * eta_prev * eta_prev);
      eta = std::min(eta, eta_max);
    }
    g_prev = g;
    eta_prev = eta;
    return eta;
  }
};

// Device scratch of the Newton iteration: per segment flags and tolerances.
struct SegScratch {
  int* flag = nullptr;
  double* tol2 = nullptr;
};

// Newton systems (W + Sigma_tilde^{-1}) x_k = rhs_k of every segment not frozen (Eq. newton),
// float64 in and out; x enters holding the current iterates b_k, whose residuals rhs - A b
// are grad psi(b_k). The corrections are solved by PCG from zero (the appendix algorithm)
// until ||rhs_k - A x_k|| <= target_k = max(cg_tol ||rhs_k||, eta_k ||rhs_k - A b_k||), eta_k
// from the segment's forcing term (0: the full tolerance). FP64: float64 PCG. Mixed: float32
// PCG on corrections of the float64 residual, each column to the relative accuracy it still
// lacks (at least 1e-6), until every float64 residual meets its target (iterative
// refinement). Segments that are frozen or done get a zero right-hand side (an inactive PCG
// column) and keep their x. full[k]: the solve met cg_tol ||rhs_k||.
inline vl_status solve_seg(State* st, const vl_opts* o, Engine<double>& E64, Engine<float>* E32, const double* rhs,
                           double* x, std::vector<Forcing>& fc, const std::vector<char>& frozen,
                           std::vector<vl_stats>& ss, std::vector<char>& full, SegScratch& dev) {
  Ctx* c = st->ctx;
  const int n = (int)st->f->n, nseg = E64.nseg;
  const bool fp64 = o->precision == VL_FP64;
  const int32_t* row_seg = st->f->row_seg;
  Scratch S(c);
  double* res = S.get<double>(n);
  double* d64 = fp64 ? S.get<double>(n) : nullptr;
  float* r32 = fp64 ? nullptr : S.get<float>(n);
  float* d32 = fp64 ? nullptr : S.get<float>(n);
  if (!res || (fp64 ? !d64 : (!r32 || !d32))) return fail(c, VL_ERR_OOM, "workspace exhausted (Newton solve)");
  std::vector<double> bn, rn, target(nseg, 0.0), tol2(nseg, 1.0);
  std::vector<int> keep(nseg, 0);
  VL_TRY(E64.coldot(rhs, rhs, nullptr, E64.red));
  VL_TRY(to_host(c, bn, (const double*)E64.red, (size_t)nseg));
  for (double& v : bn) v = std::sqrt(v);
  for (int pass = 0; pass < 12; ++pass) {
    VL_TRY(E64.opA(x, res));
    residual_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, rhs, res);
    VL_TRY(E64.coldot(res, res, nullptr, E64.red));
    VL_TRY(to_host(c, rn, (const double*)E64.red, (size_t)nseg));
    for (double& v : rn) v = std::sqrt(v);
    bool any = false;
    for (int k = 0; k < nseg; ++k) {
      if (pass == 0) target[k] = frozen[k] ? INFINITY : std::max(o->cg_tol * bn[k], fc[k].next(rn[k]) * rn[k]);
      keep[k] = !frozen[k] && rn[k] > target[k];
      any = any || keep[k];
      const double inner = std::min(0.1, std::max(fp64 ? 1e-15 : 1e-6, 0.5 * target[k] / std::max(rn[k], 1e-300)));
      tol2[k] = keep[k] ? inner * inner : 1.0;
    }
    if (!any) break;
    VL_TRY(to_device(c, dev.flag, keep));
    VL_TRY(to_device(c, dev.tol2, tol2));
    mask_rows_kernel<double><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, 1, row_seg, dev.flag, res);
    int used = 0;
    if (fp64) {
      VL_TRY(E64.solve_A1(res, d64, 1.0, o->cg_max_iter, &used, dev.tol2));
      accumulate_kernel<double, double><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, x, d64);
    } else {
      convert_kernel<double, float><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, res, r32);
      VL_CUDA(c, cudaGetLastError());
      VL_TRY(E32->solve_A1(r32, d32, 1.0, o->cg_max_iter, &used, dev.tol2));
      accumulate_kernel<double, float><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, x, d32);
    }
    VL_CUDA(c, cudaGetLastError());
    std::vector<int> its;
    std::vector<double> rel;
    if (fp64)
      VL_TRY(E64.column_stats(its, rel));
    else
      VL_TRY(E32->column_stats(its, rel));
    for (int k = 0; k < nseg; ++k) {
      if (!keep[k]) continue;
      ss[k].cg_calls++;
      ss[k].cg_iters_total += its[k];
      ss[k].cg_iters_max = its[k];
      if (!fp64) ss[k].refine_steps++;
      // a float64 PCG that stopped at cg_max_iter above its tolerance cannot be refined
      if (fp64 && its[k] >= o->cg_max_iter && rel[k] * rel[k] > tol2[k])
        return fail(c, VL_ERR_NOT_CONVERGED, "Newton solve: PCG reached cg_max_iter above cg_tol");
    }
  }
  bool missed = false;
  for (int k = 0; k < nseg; ++k) {
    const double r = bn[k] > 0 ? rn[k] / bn[k] : 0.0;
    full[k] = !frozen[k] && r <= o->cg_tol;
    if (full[k]) ss[k].true_relres_max = std::max(ss[k].true_relres_max, r);
    missed = missed || (!frozen[k] && rn[k] > target[k]);
  }
  if (missed)
    return fail(c, VL_ERR_NOT_CONVERGED, fp64 ? "Newton solve did not reach its tolerance"
                                              : "mixed-precision refinement did not reach cg_tol");
  return VL_OK;
}

// Newton's iteration (Eq. newton) for every segment of st->f: b^0 = 0; each step solves the
// Newton system in the correction form (solve_seg), halves the step (at most 30 times) while
// it lowers psi_k by more than 1e-12 (1 + |psi_k|), and a segment stops once max |b_new - b|
// <= newton_tol (1 + max |b_new|) after a solve to the full tolerance. Segments step together
// and a stopped segment is frozen. On return W holds W(b*) and conv[k] tells which segments
// stopped; ss[k] holds their statistics.
inline vl_status newton_run(State* st, const vl_opts* o, std::vector<vl_stats>& ss, std::vector<char>& conv) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n, nseg = std::max(1, f->nseg);
  const bool mixed = o->precision == VL_FP32_REFINE;
  Scratch S(c);
  double* g = S.get<double>(n);
  double* rhs = S.get<double>(n);
  double* bn = S.get<double>(n);
  double* lp = S.get<double>(n);
  SegScratch dev;
  dev.flag = S.get<int>(nseg);
  dev.tol2 = S.get<double>(nseg);
  if (!g || !rhs || !bn || !lp || !dev.flag || !dev.tol2) return fail(c, VL_ERR_OOM, "workspace exhausted (Newton)");
  Engine<double> E64(c);
  Engine<float> E32(c);
  if (o->precond == VL_PREC_LRAC) VL_TRY(lrac_build(f, o->k));
  VL_TRY(E64.init(f, 1, o->precond, st->W, mixed ? 0 : o->cg_max_iter + 1));
  std::vector<double> psi, psi_new, step, bmax;
  VL_TRY(psi_seg(st, E64, lp, st->b, psi));
  ss.assign(nseg, vl_stats{});
  conv.assign(nseg, 0);
  std::vector<Forcing> fc(nseg);
  for (Forcing& x : fc) x.eta_max = o->newton_eta_max > 0.0 ? std::min(o->newton_eta_max, 0.9) : 0.0;
  std::vector<char> full(nseg, 0);
  std::vector<int> hflag(nseg, 0);
  const LikSpec L = lik_spec(st);
  for (int it = 1; it <= o->newton_max_iter; ++it) {
    lik_seg_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, L, st->y, st->F, st->b, st->W, g, rhs, nullptr);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(E64.set_W(st->W));
    if (mixed) VL_TRY(E32.W ? E32.set_W(st->W) : E32.init(f, 1, o->precond, st->W, o->cg_max_iter + 1));
    VL_CUDA(c, cudaMemcpyAsync(bn, st->b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    VL_TRY(solve_seg(st, o, E64, mixed ? &E32 : nullptr, rhs, bn, fc, conv, ss, full, dev));
    VL_TRY(psi_seg(st, E64, lp, bn, psi_new));
    for (int hlv = 0; hlv < 30; ++hlv) {
      bool any = false;
      for (int k = 0; k < nseg; ++k) {
        hflag[k] = !conv[k] && psi_new[k] < psi[k] - 1e-12 * (1.0 + std::fabs(psi[k]));
        any = any || hflag[k];
      }
      if (!any) break;
      VL_TRY(to_device(c, dev.flag, hflag));
      halve_seg_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, f->row_seg, dev.flag, st->b, bn);
      VL_TRY(psi_seg(st, E64, lp, bn, psi_new));
    }
    VL_TRY(seg_absmax(E64, bn, st->b, step, bmax));
    VL_CUDA(c, cudaMemcpyAsync(st->b, bn, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    bool all = true;
    for (int k = 0; k < nseg; ++k) {
      if (conv[k]) continue;
      ss[k].newton_iters = it;
      psi[k] = psi_new[k];
      if (!std::isfinite(psi[k])) return fail(c, VL_ERR_NOT_CONVERGED, "Newton: non-finite objective");
      if (step[k] <= o->newton_tol * (1.0 + bmax[k])) {
        if (full[k])
          conv[k] = 1;
        else
          fc[k].force_full = true;   // a small step from an inexact solve: confirm with a full one
      }
      all = all && conv[k];
    }
    if (all) break;
  }
  // W at the mode
  lik_seg_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, L, st->y, st->F, st->b, st->W, nullptr, nullptr, nullptr);
  VL_CUDA(c, cudaGetLastError());
  VL_CUDA(c, cudaStreamSynchronize(c->stream));
  return VL_OK;
}

// Float64 relative residuals ||z_q - S u_q|| / ||z_q|| of the SLQ probe solves (S the system
// operator of the preconditioner's form, z = P^{1/2} r built again in float64 from the same
// probes), per (segment, column) q. Float32 solves are refined by float32 correction solves
// of the float64 residual until every column meets cg_tol; this leaves T (already turned into
// gamma_q) alone. relres: per segment, the largest over its columns.
template <typename T>
inline vl_status probe_residuals(State* st, const vl_opts* o, Engine<T>& E, T* Rm, T* Zm, T* Um, const double* r1,
                                 std::vector<double>& relres, std::vector<int>& passes, int64_t* extra_iters) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n, t = o->t, ld = E.ld, nseg = E.nseg, ncol = E.ncol;
  const int64_t vec = (int64_t)n * ld;
  std::vector<double> bn, rn;
  auto worst = [&]() {
    relres.assign(nseg, 0.0);
    for (int q = 0; q < ncol; ++q)
      relres[q / t] = std::max(relres[q / t], bn[q] > 0 ? std::sqrt(rn[q] / bn[q]) : 0.0);
  };
  passes.assign(nseg, 0);
  if (extra_iters) *extra_iters = 0;
  if constexpr (std::is_same<T, double>::value) {
    VL_TRY(E.opSys(Um, E.v));
    residual_kernel<<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, Zm, E.v);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(E.coldot(Zm, Zm, nullptr, E.red));
    VL_TRY(to_host(c, bn, (const double*)E.red, (size_t)ncol));
    VL_TRY(E.coldot(E.v, E.v, nullptr, E.red));
    VL_TRY(to_host(c, rn, (const double*)E.red, (size_t)ncol));
    worst();
    return VL_OK;
  } else {
    Scratch S(c);
    Engine<double> E64(c);
    VL_TRY(E64.init(f, t, o->precond, st->W, 0, /*ops_only=*/true));
    double* Zd = S.get<double>(vec);
    double* Ud = S.get<double>(vec);
    double* Res = S.get<double>(vec);
    double* sc64 = S.get<double>(n);
    int* keep = S.get<int>(ncol);
    if (!Zd || !Ud || !Res || !sc64 || !keep) return fail(c, VL_ERR_OOM, "workspace exhausted (probe residuals)");
    // the probes again, in float64
    rademacher_kernel<double><<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, t, ld, f->s2u_probe(), o->seed, 0, 0, Res);
    const int dmode = o->precond == VL_PREC_VADU ? 0 : (o->precond == VL_PREC_LVA ? 1 : 3);
    diag_fn_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, dmode, st->W, f->D64, sc64);
    VL_CUDA(c, cudaGetLastError());
    if (o->precond == VL_PREC_LRAC)
      VL_TRY(E64.lrac_lowrank_plus(r1, Res, sc64, Zd));
    else
      VL_TRY(E64.opBt(Res, sc64, nullptr, nullptr, Zd));
    VL_TRY(E64.coldot(Zd, Zd, nullptr, E64.red));
    VL_TRY(to_host(c, bn, (const double*)E64.red, (size_t)ncol));
    std::vector<int> hkeep(ncol, 0);
    // the solution is carried in float64 from here on: a float32 copy of it could not hold
    // a residual below about cond * 2^-24
    convert_kernel<float, double><<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, Um, Ud);
    int pass = 0;
    for (;; ++pass) {
      VL_TRY(E64.opSys(Ud, Res));
      residual_kernel<<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, Zd, Res);
      VL_CUDA(c, cudaGetLastError());
      VL_TRY(E64.coldot(Res, Res, nullptr, E64.red));
      VL_TRY(to_host(c, rn, (const double*)E64.red, (size_t)ncol));
      worst();
      double rel = 0.0;
      for (double v : relres) rel = std::max(rel, v);
      if (rel <= o->cg_tol || pass == 12) break;
      // correction solves for the columns still above cg_tol, each to the accuracy it lacks
      double inner = 0.5;
      for (int q = 0; q < ncol; ++q) {
        const double rq = bn[q] > 0 ? std::sqrt(rn[q] / bn[q]) : 0.0;
        hkeep[q] = rq > o->cg_tol ? 1 : 0;
        if (hkeep[q]) inner = std::min(inner, 0.5 * o->cg_tol / rq);
        if (hkeep[q]) passes[q / t] = pass + 1;
      }
      inner = std::max(inner, 1e-6);
      VL_TRY(to_device(c, keep, hkeep));
      convert_kernel<double, float><<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, Res, Zm);
      mask_columns_kernel<float><<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(n, t, ld, f->row_seg, keep, Zm);
      VL_CUDA(c, cudaGetLastError());
      int used = 0;
      VL_TRY(E.pcg(Zm, Rm, inner, o->cg_max_iter, &used));
      accumulate_kernel<double, float><<<grid_for(c, vec), 256, 0, VL_STREAM(c)>>>(vec, Ud, Rm);
      VL_CUDA(c, cudaGetLastError());
      if (extra_iters) *extra_iters += used;
    }
    double rel = 0.0;
    for (double v : relres) rel = std::max(rel, v);
    if (rel > o->cg_tol) return fail(c, VL_ERR_NOT_CONVERGED, "SLQ probe solves: refinement did not reach cg_tol");
    return VL_OK;
  }
}

// SLQ (Eq. def_SLQ) for every segment: probes z = P^{1/2} r (VADU: z = B^T (W + D^{-1})^{1/2} r;
// LVA: z = B^T D^{-1/2} r; Section 3.1.1), PCG on the preconditioner's system with T
// extraction, gamma_q = (r_0^T z_0)_q e1^T log(T_q) e1 per (segment, column) q = k * t + c.
// r is Rademacher by the problem's own caller index, so each problem of a batch draws the
// probes it would draw alone. For LRAC (single problems), log det(I + L^T W L) in *logdetC.
struct SlqOut {
  std::vector<double> gam;       // ncol
  std::vector<int> iters;        // ncol
  std::vector<double> relres;    // ncol (PCG recursive residual)
  std::vector<double> true_rel;  // nseg (float64 residual after refinement)
  std::vector<int> passes;       // nseg refinement passes
  int64_t extra_iters = 0;
  double logdetC = 0.0;
};

template <typename T>
inline vl_status slq_run(State* st, const vl_opts* o, SlqOut& out) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n, t = o->t;
  Scratch S(c);
  Engine<T> E(c);
  if (o->precond == VL_PREC_LRAC) VL_TRY(lrac_build(f, o->k));
  VL_TRY(E.init(f, t, o->precond, st->W, o->cg_max_iter + 1));
  const int ncol = E.ncol;
  T* Rm = S.get<T>((size_t)n * E.ld);
  T* Zm = S.get<T>((size_t)n * E.ld);
  T* Um = S.get<T>((size_t)n * E.ld);
  double* sc64 = S.get<double>(n);
  T* sc = S.get<T>(n);
  double* gdev = S.get<double>(ncol);
  double* work = S.get<double>((size_t)ncol * kQuadMaxNodes);
  double* qu0 = S.get<double>(ncol);
  int* qnodes = S.get<int>(ncol);
  int* bad = S.get<int>(1);
  if (!Rm || !Zm || !Um || !sc64 || !sc || !gdev || !work || !qu0 || !qnodes || !bad)
    return fail(c, VL_ERR_OOM, "workspace exhausted (SLQ)");
  rademacher_kernel<T><<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, t, E.ld, f->s2u_probe(), o->seed, 0, 0, Rm);
  const int dmode = o->precond == VL_PREC_VADU ? 0 : (o->precond == VL_PREC_LVA ? 1 : 3);
  diag_fn_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, dmode, st->W, f->D64, sc64);
  convert_kernel<double, T><<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, sc64, sc);
  VL_CUDA(c, cudaGetLastError());
  double* r1 = nullptr;
  if (o->precond == VL_PREC_LRAC) {
    // z = L r1 + W^{-1/2} r2, r1 in {+-1}^k drawn by rank index on stream 3 (Section 3.1.2)
    r1 = S.get<double>((size_t)E.kr * t);
    if (!r1) return fail(c, VL_ERR_OOM, "workspace exhausted (SLQ probes)");
    rademacher_kernel<double><<<(E.kr + 127) / 128, 128, 0, VL_STREAM(c)>>>(E.kr, t, t, nullptr, o->seed, 3, 0, r1);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(E.lrac_lowrank_plus(r1, Rm, sc, Zm));
  } else {
    VL_TRY(E.opBt(Rm, sc, nullptr, nullptr, Zm));
  }
  int used = 0;
  VL_TRY(E.pcg(Zm, Um, o->cg_tol, o->cg_max_iter, &used));
  VL_CUDA(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
  {
    // the node range of every column, then every (column, node) in its own thread, then the
    // per-column sums in node order
    ProfScope ps(c, "slq_quad", t);
    const size_t qsm = sizeof(double) * 2 * (size_t)E.lmax;
    const int staged = qsm <= kSmemSolveBytes ? 1 : 0;
    if (staged) VL_TRY(smem_limit_once(c, (const void*)slq_node_kernel, kSmemSolveBytes));
    slq_range_kernel<<<ncol, 32, 0, VL_STREAM(c)>>>(ncol, E.lmax, E.S.Tdiag, E.S.Toff, E.S.iters, qu0, qnodes, bad);
    slq_node_kernel<<<dim3(kQuadMaxNodes / 64, ncol), 64, staged ? qsm : 0, VL_STREAM(c)>>>(
        ncol, E.lmax, E.S.Tdiag, E.S.Toff, E.S.iters, qu0, qnodes, work, staged);
    slq_sum_kernel<<<(ncol + 127) / 128, 128, 0, VL_STREAM(c)>>>(ncol, qnodes, E.S.rz0, work, gdev);
  }
  VL_CUDA(c, cudaGetLastError());
  VL_TRY(E.column_stats(out.iters, out.relres));
  std::vector<int> hbad;
  VL_TRY(to_host(c, hbad, (const int*)bad, 1));
  VL_TRY(to_host(c, out.gam, (const double*)gdev, (size_t)ncol));
  if (hbad[0]) return fail(c, VL_ERR_NOT_CONVERGED, "SLQ: a Lanczos tridiagonal is not positive definite (non-positive Ritz value)");
  for (int q = 0; q < ncol; ++q)
    if (out.relres[q] > o->cg_tol && out.iters[q] >= o->cg_max_iter)
      return fail(c, VL_ERR_NOT_CONVERGED, "SLQ probe solves reached cg_max_iter");
  out.logdetC = (o->precond == VL_PREC_LRAC) ? E.logdetC : 0.0;
  return probe_residuals<T>(st, o, E, Rm, Zm, Um, r1, out.true_rel, out.passes, &out.extra_iters);
}

// L^VLA of every segment (Eq. VLA_loss) from the SLQ terms: -log p(y | mu*) + b*^T Sigma^{-1} b* / 2
// + log det(Sigma_tilde W + I) / 2 with the log-determinant split by the preconditioner
// (Eq. logdetsplit: sum log D + log det P + SLQ; LRAC, Eq. logdetsplit2: log det C + SLQ).
struct LmlOut {
  std::vector<double> lml, logdet, mean, se;
};

inline vl_status lml_assemble(State* st, const vl_opts* o, const SlqOut& q, LmlOut& out) {
  Ctx* c = st->ctx;
  Factor* f = st->f;
  const int n = (int)f->n, t = o->t, nseg = std::max(1, f->nseg);
  Scratch S(c);
  double* lp = S.get<double>(n);
  if (!lp) return fail(c, VL_ERR_OOM, "workspace exhausted (L^VLA)");
  Engine<double> E1(c);
  VL_TRY(E1.init(f, 1, VL_PREC_VADU, st->W, 0));   // B products and per-segment sums only
  std::vector<double> psi, logp, quad, sld, slp;
  VL_TRY(psi_seg(st, E1, lp, st->b, psi, &logp, &quad));
  if (o->precond != VL_PREC_LRAC) {
    VL_TRY(seg_sums(E1, 1, f->D64, nullptr, sld));
    if (o->precond == VL_PREC_VADU) VL_TRY(seg_sums(E1, 2, f->D64, st->W, slp));
  }
  out.lml.assign(nseg, 0.0);
  out.logdet.assign(nseg, 0.0);
  out.mean.assign(nseg, 0.0);
  out.se.assign(nseg, 0.0);
  for (int k = 0; k < nseg; ++k) {
    double mean = 0.0;
    for (int j = 0; j < t; ++j) mean += q.gam[k * t + j];
    mean /= t;
    double var = 0.0;
    for (int j = 0; j < t; ++j) var += (q.gam[k * t + j] - mean) * (q.gam[k * t + j] - mean);
    out.mean[k] = mean;
    out.se[k] = t > 1 ? std::sqrt(var / (t - 1) / t) : 0.0;
    double ld;
    if (o->precond == VL_PREC_LRAC)
      ld = q.logdetC + mean;                                     // log det P = log det C - log det W
    else if (o->precond == VL_PREC_VADU)
      ld = sld[k] + slp[k] + mean;                               // log det P = log det(W + D^{-1})
    else
      ld = sld[k] - sld[k] + mean;                               // log det P = log det D^{-1}
    out.logdet[k] = ld;
    out.lml[k] = -logp[k] + 0.5 * quad[k] + 0.5 * ld;
  }
  return VL_OK;
}

}  // namespace vl
