// Gradient of L^VLA with respect to theta = (sigma2, rho) by stochastic trace
// estimation on the SLQ probes with the control variate of Section 3 (VADU
// preconditioner, float64), following the appendix "Gradients of Vecchia-Laplace
// approximations":
//   dL/dtheta = 1/2 b*^T dSinv b* + 1/2 dlogdet(Sigma_tilde W + I)/dtheta - (A^{-1} g)^T dSinv b*
//   dlogdet/dtheta ~ sum dD_i/D_i - c sum dD_i / (D_i^2 (W_i + 1/D_i)) + mean_k [h(z_k) - c r(z_k)]
//   h(z) = (A^{-1} z)^T dSinv P^{-1} z,  r(z) = (P^{-1} z)^T (dSinv + dB^T W B + B^T W dB) P^{-1} z
//   g_j = 1/2 [c_j W'_j / (W_j + 1/D_j) + mean_k (h_j - c_j r_j)],
//   h_j = (A^{-1} z)_j W'_j (P^{-1} z)_j,  r_j = (B P^{-1} z)_j^2 W'_j
//   dL/dF = -grad log p(y | mu*) + g - W o (A^{-1} g)        (db*/dF_i = -A^{-1} W e_i)
// with A = W + Sigma_tilde^{-1}, W' = dW/dmu, c = Cov(h, r) / Var(r) (0 when r does not
// vary over the probes: then any c gives the same estimate, and the ratio would only
// amplify rounding). The factor derivatives (appendix "Derivatives of the
// Vecchia-approximated precision"):
//   dA_i = (dSigma_{i,N} - A_i dSigma_N) Sigma_N^{-1},  dD_i = dSigma_ii - dA_i Sigma_{N,i} - A_i dSigma_{N,i}
//   dSinv = dB^T D^{-1} B + B^T D^{-1} dB - B^T D^{-1} dD D^{-1} B,  dB_{i,N(i)} = -dA_i
// The nugget follows sigma2 (tau = nugget / sigma2 * sigma2), so dSigma/dsigma2 = Sigma / sigma2.
#include <cmath>
#include <vector>

#include "engine.cuh"

struct vl_state : vl::State {};   // the same definition as in api.cu

namespace vl {
namespace {

constexpr int kDerivWarps = 2;

__device__ __forceinline__ double dcov_eval(double h, int cov, double sigma2, double rho, int param) {
  if (param == 0) return cov_eval(h, cov, 1.0, rho);   // d / d sigma2
  if (cov == VL_COV_EXPONENTIAL) return sigma2 * exp(-h / rho) * h / (rho * rho);
  const double a = kSqrt3 * h / rho;
  return sigma2 * a * a * exp(-a) / rho;
}

__device__ __forceinline__ double pdist(double ax, double ay, double bx, double by) {
  const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
  return sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// One warp per row: dA_i and dD_i (storage rows, aligned with nbr / A).
__global__ void factor_deriv_kernel(int rows, int m, const double* __restrict__ locs, const int32_t* __restrict__ nbr,
                                    const double* __restrict__ A, int cov, double sigma2, double rho, double nugget,
                                    int param, double* __restrict__ dA, double* __restrict__ dD,
                                    DevStatus* st) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int ld = m + 1;
  double* S = smem + (size_t)wib * (m * ld + 4 * m);
  double* v = S + m * ld;    // Sigma_{N,i}
  double* q = v + m;         // rhs, then dA_i
  double* P = q + m;         // 2m neighbour coordinates
  const int r = blockIdx.x * kDerivWarps + wib;
  if (r >= rows) return;
  const double ratio = nugget / sigma2;
  const double dsii = param == 0 ? 1.0 + ratio : 0.0;
  const double qx = locs[2 * (int64_t)r], qy = locs[2 * (int64_t)r + 1];
  int cnt = 0;
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int c = c0 + lane;
    const int j = c < m ? nbr[(int64_t)r * m + c] : -1;
    cnt += __popc(__ballot_sync(0xffffffffu, j >= 0));
    if (j >= 0) {
      P[2 * c] = locs[2 * (int64_t)j];
      P[2 * c + 1] = locs[2 * (int64_t)j + 1];
    }
  }
  __syncwarp();
  if (cnt == 0) {
    for (int c = lane; c < m; c += 32) dA[(int64_t)r * m + c] = 0.0;
    if (lane == 0) dD[r] = dsii;
    return;
  }
  const double* Ai = A + (int64_t)r * m;
  // Sigma_N (lower triangle), Sigma_{N,i}, and q_b = dSigma_{b,i} - (A_i dSigma_N)_b
  for (int a = lane; a < cnt; a += 32) {
    for (int b = 0; b <= a; ++b) {
      const double cv = cov_eval(pdist(P[2 * a], P[2 * a + 1], P[2 * b], P[2 * b + 1]), cov, sigma2, rho);
      S[a * ld + b] = (a == b) ? cv + nugget : cv;
    }
    const double h = pdist(P[2 * a], P[2 * a + 1], qx, qy);
    v[a] = cov_eval(h, cov, sigma2, rho);
    double acc = 0.0;
    for (int b = 0; b < cnt; ++b) {
      double d = dcov_eval(pdist(P[2 * a], P[2 * a + 1], P[2 * b], P[2 * b + 1]), cov, sigma2, rho, param);
      if (a == b && param == 0) d += ratio;
      acc += Ai[b] * d;
    }
    q[a] = dcov_eval(h, cov, sigma2, rho, param) - acc;
  }
  __syncwarp();
  // Cholesky of Sigma_N (as in the factor kernel), then q <- Sigma_N^{-1} q
  bool bad = false;
  for (int j = 0; j < cnt; ++j) {
    const double piv = S[j * ld + j];
    if (!(piv > 0.0)) {
      bad = true;
      break;
    }
    const double ljj = sqrt(piv);
    __syncwarp();
    for (int a = j + 1 + lane; a < cnt; a += 32) S[a * ld + j] /= ljj;
    if (lane == 0) S[j * ld + j] = ljj;
    __syncwarp();
    for (int a = j + 1 + lane; a < cnt; a += 32) {
      const double laj = S[a * ld + j];
      for (int b = j + 1; b <= a; ++b) S[a * ld + b] -= laj * S[b * ld + j];
    }
    __syncwarp();
  }
  if (!bad) {
    for (int j = 0; j < cnt; ++j) {
      const double wj = q[j] / S[j * ld + j];
      __syncwarp();
      if (lane == 0) q[j] = wj;
      for (int a = j + 1 + lane; a < cnt; a += 32) q[a] -= S[a * ld + j] * wj;
      __syncwarp();
    }
    for (int j = cnt - 1; j >= 0; --j) {
      const double aj = q[j] / S[j * ld + j];
      __syncwarp();
      if (lane == 0) q[j] = aj;
      for (int b = lane; b < j; b += 32) q[b] -= S[j * ld + b] * aj;
      __syncwarp();
    }
  }
  // dD_i = dSigma_ii - dA_i Sigma_{N,i} - A_i dSigma_{N,i}
  double part = 0.0;
  for (int a = lane; a < cnt; a += 32) {
    const double dv = dcov_eval(pdist(P[2 * a], P[2 * a + 1], qx, qy), cov, sigma2, rho, param);
    part += q[a] * v[a] + Ai[a] * dv;
  }
  const double s = warp_sum(part);
  if (bad && lane == 0) raise_error(st, VL_ERR_NOT_SPD, r);
  for (int c = lane; c < m; c += 32) dA[(int64_t)r * m + c] = (c < cnt && !bad) ? q[c] : 0.0;
  if (lane == 0) dD[r] = bad ? NAN : dsii - s;
}

__global__ void gather_kernel(int64_t n, const int32_t* __restrict__ perm, const double* __restrict__ in,
                              double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    out[e] = in[perm[e]];
}

// Y[s, c] = alpha sum_k vals[s, k] X[nbr[s, k], c]        (ELL rows of B without the diagonal)
__global__ void ell_apply_kernel(int n, int m, int t, int ld, const int32_t* __restrict__ nbr,
                                 const double* __restrict__ vals, const double* __restrict__ X, double alpha,
                                 double* __restrict__ Y) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    double acc = 0.0;
    if (c < t)
      for (int k = 0; k < m; ++k) {
        const int j = nbr[(int64_t)s * m + k];
        if (j >= 0) acc += vals[(int64_t)s * m + k] * X[(int64_t)j * ld + c];
      }
    Y[e] = alpha * acc;
  }
}

// Y[s, c] = alpha sum_{e in row s of the transpose} valsT[e] X[colT[e], c]
__global__ void csrT_apply_kernel(int n, int t, int ld, const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ col, const double* __restrict__ valsT,
                                  const double* __restrict__ X, double alpha, double* __restrict__ Y) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    double acc = 0.0;
    if (c < t)
      for (int k = rowptr[s]; k < rowptr[s + 1]; ++k) acc += valsT[k] * X[(int64_t)col[k] * ld + c];
    Y[e] = alpha * acc;
  }
}

// For u = B X, du = dB X (n x ld blocks): the two right-hand vectors of
//   dSinv X = -dA^T (D^{-1} u) + B^T [D^{-1} (du - dD D^{-1} u)]
//   M X     = -dA^T (D^{-1} u + W u) + B^T [D^{-1} (du - dD D^{-1} u) + W du]
__global__ void dsinv_parts_kernel(int n, int t, int ld, const double* __restrict__ D, const double* __restrict__ dD,
                                   const double* __restrict__ W, const double* __restrict__ u,
                                   const double* __restrict__ du, int with_w, double* __restrict__ y1,
                                   double* __restrict__ y2) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    if (c >= t) {
      y1[e] = 0.0;
      y2[e] = 0.0;
      continue;
    }
    const double di = 1.0 / D[s], us = u[e], dus = du[e];
    y1[e] = di * us + (with_w ? W[s] * us : 0.0);
    y2[e] = di * (dus - dD[s] * di * us) + (with_w ? W[s] * dus : 0.0);
  }
}

// Z = X + Y (n x ld)
__global__ void add_kernel(int64_t total, const double* __restrict__ X, const double* __restrict__ Y,
                           double* __restrict__ Z) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Z[e] = X[e] + Y[e];
}

__device__ __forceinline__ double w_prime(int lik, double mu) {
  if (lik == VL_LIK_BERNOULLI_LOGIT) {
    const double p = 1.0 / (1.0 + exp(-mu));
    return p * (1.0 - p) * (1.0 - 2.0 * p);
  }
  return exp(mu);
}

// Per row j over the t probes: h_j = AZ W'_j PZ, r_j = BPZ^2 W'_j, their control-variate
// weight and g_j = 1/2 dlogdet / dmu_j.
__global__ void implicit_g_kernel(int n, int t, int ld, int lik, const double* __restrict__ F,
                                  const double* __restrict__ b, const double* __restrict__ W,
                                  const double* __restrict__ D, const double* __restrict__ AZ,
                                  const double* __restrict__ PZ, const double* __restrict__ BPZ, int use_cv,
                                  double* __restrict__ g) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double wp = w_prime(lik, (F ? F[j] : 0.0) + b[j]);
  double mh = 0.0, mr = 0.0;
  for (int k = 0; k < t; ++k) {
    const int64_t e = (int64_t)j * ld + k;
    mh += AZ[e] * wp * PZ[e];
    mr += BPZ[e] * BPZ[e] * wp;
  }
  mh /= t;
  mr /= t;
  double c = 0.0;
  if (use_cv && t > 1) {
    double vr = 0.0, chr = 0.0;
    for (int k = 0; k < t; ++k) {
      const int64_t e = (int64_t)j * ld + k;
      const double hk = AZ[e] * wp * PZ[e], rk = BPZ[e] * BPZ[e] * wp;
      vr += (rk - mr) * (rk - mr);
      chr += (hk - mh) * (rk - mr);
    }
    vr /= (t - 1);
    chr /= (t - 1);
    if (vr > 1e-20 * mr * mr) c = chr / vr;
  }
  const double s = 1.0 / (W[j] + 1.0 / D[j]);
  g[j] = 0.5 * (c * wp * s + mh - c * mr);
}

// out[0] = sum dD_i / D_i, out[1] = -sum dD_i / (D_i^2 (W_i + 1/D_i))  (one block, fixed order)
__global__ void dlog_sums_kernel(int n, const double* __restrict__ D, const double* __restrict__ dD,
                                 const double* __restrict__ W, double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double a0 = 0.0, a1 = 0.0;
  for (int s = threadIdx.x; s < n; s += blockDim.x) {
    a0 += dD[s] / D[s];
    a1 -= dD[s] / (D[s] * D[s] * (W[s] + 1.0 / D[s]));
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      x += s0[i];
      y += s1[i];
    }
    out[0] = x;
    out[1] = y;
  }
}

// dF[s2u[s]] = -d log p / d mu_s + g_s - W_s (A^{-1} g)_s     (caller order)
__global__ void offset_grad_kernel(int n, int lik, const int32_t* __restrict__ s2u, const double* __restrict__ y,
                                   const double* __restrict__ F, const double* __restrict__ b,
                                   const double* __restrict__ W, const double* __restrict__ g,
                                   const double* __restrict__ Ag, double* __restrict__ dF) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double mu = (F ? F[s] : 0.0) + b[s];
    const double gl = lik == VL_LIK_BERNOULLI_LOGIT ? y[s] - 1.0 / (1.0 + exp(-mu)) : y[s] - exp(mu);
    dF[s2u[s]] = -gl + g[s] - W[s] * Ag[s];
  }
}

__global__ void probe_scale_kernel(int n, const double* __restrict__ W, const double* __restrict__ D,
                                   double* __restrict__ sc) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
    sc[s] = sqrt(W[s] + 1.0 / D[s]);
}

// dSinv X (and, when M is non-null, M X as well) for an n x ld block X on engine E.
vl_status apply_dsinv(Engine<double>& E, Factor* f, const double* dA, const double* dAT, const double* dD,
                      const double* W, const double* X, double* dSX, double* MX, double* u, double* du, double* y1,
                      double* y2, double* tmp) {
  Ctx* c = E.c;
  const int n = E.n, t = E.t, ld = E.ld, m = f->m;
  const int64_t tot = (int64_t)n * ld;
  VL_TRY(E.opB(X, nullptr, u));                                                   // u = B X
  ell_apply_kernel<<<grid_for(c, tot), 256, 0, VL_STREAM(c)>>>(n, m, t, ld, f->nbr, dA, X, -1.0, du);   // dB X
  for (int pass = 0; pass < (MX ? 2 : 1); ++pass) {
    double* out = pass == 0 ? dSX : MX;
    dsinv_parts_kernel<<<grid_for(c, tot), 256, 0, VL_STREAM(c)>>>(n, t, ld, f->D64, dD, W, u, du, pass, y1, y2);
    csrT_apply_kernel<<<grid_for(c, tot), 256, 0, VL_STREAM(c)>>>(n, t, ld, f->rowptrT, f->colT, dAT, y1, -1.0, tmp);
    VL_TRY(E.opBt(y2, nullptr, nullptr, nullptr, out));                          // B^T y2
    add_kernel<<<grid_for(c, tot), 256, 0, VL_STREAM(c)>>>(tot, out, tmp, out);
  }
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

}  // namespace
}  // namespace vl

extern "C" vl_status vl_lml_grad(vl_state* st, const vl_opts* o, double* grad, double* dF, vl_stats* stats) {
  using namespace vl;
  if (!st) return VL_ERR_INVALID_ARG;
  State* S = static_cast<State*>(st);
  Ctx* c = S->ctx;
  Factor* f = S->f;
  if (!o || !grad) return fail(c, VL_ERR_INVALID_ARG, "vl_lml_grad: opts and grad must be non-null");
  if (o->precision != VL_FP64 || o->precond != VL_PREC_VADU)
    return fail(c, VL_ERR_INVALID_ARG, "vl_lml_grad: supported for float64 with the VADU preconditioner only");
  if (S->lik != VL_LIK_BERNOULLI_LOGIT && S->lik != VL_LIK_POISSON_LOG)
    return fail(c, VL_ERR_INVALID_ARG, "vl_lml_grad: supported for the Bernoulli and Poisson likelihoods only");
  if (o->t < 1 || o->t > 256 || !(o->cg_tol > 0) || o->cg_max_iter < 1)
    return fail(c, VL_ERR_INVALID_ARG, "vl_lml_grad: invalid option value");
  const int n = (int)f->n, m = f->m, t = o->t;
  Engine<double> E(c), E1(c);
  VL_TRY(E.init(f, t, VL_PREC_VADU, S->W, o->cg_max_iter + 1));
  VL_TRY(E1.init(f, 1, VL_PREC_VADU, S->W, o->cg_max_iter + 1));
  const int ld = E.ld;
  const int64_t blk = (int64_t)n * ld;
  Scratch M(c);
  double* R = M.get<double>(blk);
  double* Z = M.get<double>(blk);
  double* AZ = M.get<double>(blk);
  double* PZ = M.get<double>(blk);
  double* BPZ = M.get<double>(blk);
  double* dSX = M.get<double>(blk);
  double* MX = M.get<double>(blk);
  double* u = M.get<double>(blk);
  double* du = M.get<double>(blk);
  double* y1 = M.get<double>(blk);
  double* y2 = M.get<double>(blk);
  double* tmp = M.get<double>(blk);
  double* sc = M.get<double>(n);
  double* g = M.get<double>(n);
  double* Ag = M.get<double>(n);
  double* dSb = M.get<double>(n);
  double* dA = M.get<double>((size_t)n * std::max(m, 1));
  double* dAT = M.get<double>((size_t)std::max<int64_t>(f->nnz, 1));
  double* dD = M.get<double>(n);
  double* sums = M.get<double>(2);
  double* hd = M.get<double>(t);
  double* rd = M.get<double>(t);
  double* sd = M.get<double>(2);
  if (!R || !Z || !AZ || !PZ || !BPZ || !dSX || !MX || !u || !du || !y1 || !y2 || !tmp || !sc || !g || !Ag ||
      !dSb || !dA || !dAT || !dD || !sums || !hd || !rd || !sd)
    return fail(c, VL_ERR_OOM, "workspace exhausted (vl_lml_grad)");
  // probes z = P^{1/2} r = B^T (W + D^{-1})^{1/2} r, the same as vl_log_marglik's
  rademacher_kernel<double><<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, t, ld, f->s2u, o->seed, 0, 0, R);
  probe_scale_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, S->W, f->D64, sc);
  VL_CUDA(c, cudaGetLastError());
  VL_TRY(E.opBt(R, sc, nullptr, nullptr, Z));
  int used = 0;
  VL_TRY(E.pcg(Z, AZ, o->cg_tol, o->cg_max_iter, &used));      // A^{-1} z
  VL_TRY(E.opPinv(Z, PZ));                                      // P^{-1} z
  VL_TRY(E.opB(PZ, nullptr, BPZ));                              // B P^{-1} z
  implicit_g_kernel<<<(n + 127) / 128, 128, 0, VL_STREAM(c)>>>(n, t, ld, S->lik, S->F, S->b, S->W, f->D64, AZ, PZ,
                                                             BPZ, 1, g);
  VL_CUDA(c, cudaGetLastError());
  int used1 = 0;
  VL_TRY(E1.pcg(g, Ag, o->cg_tol, o->cg_max_iter, &used1));     // A^{-1} g
  const int threads = 32 * kDerivWarps;
  const size_t smem = sizeof(double) * (size_t)kDerivWarps * (m * (m + 1) + 4 * m);
  const size_t smem_max = sizeof(double) * (size_t)kDerivWarps * (64 * 65 + 4 * 64);
  VL_CUDA(c, cudaFuncSetAttribute(factor_deriv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
  for (int par = 0; par < 2; ++par) {
    VL_CUDA(c, status_clear(c));
    factor_deriv_kernel<<<(n + kDerivWarps - 1) / kDerivWarps, threads, smem, VL_STREAM(c)>>>(
        n, m, f->locs_s, f->nbr, f->A64, f->cov, f->sigma2, f->rho, f->nugget, par, dA, dD, c->dstatus);
    if (f->nnz > 0) gather_kernel<<<grid_for(c, f->nnz), 256, 0, VL_STREAM(c)>>>(f->nnz, f->permT, dA, dAT);
    VL_CUDA(c, cudaGetLastError());
    VL_TRY(check_dev_status(c, "factor derivatives"));
    // h and r over the probes
    VL_TRY(apply_dsinv(E, f, dA, dAT, dD, S->W, PZ, dSX, MX, u, du, y1, y2, tmp));
    VL_TRY(E.coldot(AZ, dSX, nullptr, hd));
    VL_TRY(E.coldot(PZ, MX, nullptr, rd));
    // dSinv b*, then 1/2 b*^T dSinv b* and (A^{-1} g)^T dSinv b*
    VL_TRY(apply_dsinv(E1, f, dA, dAT, dD, S->W, S->b, dSb, nullptr, u, du, y1, y2, tmp));
    VL_TRY(E1.coldot(S->b, dSb, nullptr, sd));
    VL_TRY(E1.coldot(Ag, dSb, nullptr, sd + 1));
    dlog_sums_kernel<<<1, 256, 0, VL_STREAM(c)>>>(n, f->D64, dD, S->W, sums);
    VL_CUDA(c, cudaGetLastError());
    std::vector<double> h(t), r(t), s2(2), sm(2);
    VL_CUDA(c, cudaMemcpyAsync(h.data(), hd, sizeof(double) * t, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(r.data(), rd, sizeof(double) * t, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(s2.data(), sd, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaMemcpyAsync(sm.data(), sums, sizeof(double) * 2, cudaMemcpyDeviceToHost, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
    double mh = 0.0, mr = 0.0;
    for (int k = 0; k < t; ++k) {
      mh += h[k];
      mr += r[k];
    }
    mh /= t;
    mr /= t;
    double cw = 0.0;
    if (t > 1) {
      double vr = 0.0, chr = 0.0;
      for (int k = 0; k < t; ++k) {
        vr += (r[k] - mr) * (r[k] - mr);
        chr += (h[k] - mh) * (r[k] - mr);
      }
      vr /= (t - 1);
      chr /= (t - 1);
      if (vr > 1e-20 * mr * mr) cw = chr / vr;
    }
    const double dlogdet = sm[0] + cw * sm[1] + (mh - cw * mr);
    grad[par] = 0.5 * s2[0] + 0.5 * dlogdet - s2[1];
  }
  if (dF) {
    double* dFd = M.get<double>(n);
    if (!dFd) return fail(c, VL_ERR_OOM, "workspace exhausted (vl_lml_grad)");
    offset_grad_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, S->lik, f->s2u, S->y, S->F, S->b, S->W, g, Ag,
                                                               dFd);
    VL_CUDA(c, cudaGetLastError());
    VL_CUDA(c, cudaMemcpyAsync(dF, dFd, sizeof(double) * n, cudaMemcpyDefault, c->stream));
    VL_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  if (stats) {
    *stats = vl_stats{};
    stats->cg_calls = 2;
    stats->cg_iters_max = used;
    stats->cg_iters_total = used + used1;
  }
  return VL_OK;
}
