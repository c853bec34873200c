// Predictive variances by a preconditioned partial Lanczos factorisation (Section 4,
// "Predictive (co-)variances using preconditioned Lanczos algorithms", preconditioner P_L1).
//
// k steps of Lanczos with full reorthogonalisation (two classical Gram-Schmidt passes per
// step) on M = P^{-1/2} A P^{-T/2}, A = W + Sigma_tilde^{-1}, P_L1 = B^T (W + D^{-1}) B so
// that P^{-1/2} = S^{1/2} B^{-T}, S = (W + D^{-1})^{-1}, started from P^{-1/2} times the
// mean of the columns of B_po^T (B_p = I: test points condition on training points only).
// With M ~ Q T Q^T, A^{-1} B_po^T ~ P^{-T/2} Q T^{-1} Q^T P^{-1/2} B_po^T, so with
// U = P^{-T/2} Q = B^{-1} S^{1/2} Q (n x k, one block triangular solve) and
// z_p = U^T B_po^T e_p (a gather of the m neighbour rows of U):
//   diag(Omega_p)_p ~ D_p + z_p^T T^{-1} z_p,
// the quadratic form taken through T = L diag(d) L^T (unit lower bidiagonal L). Float64.
#pragma once

#include "laplace.cuh"

namespace vl {

// h[c] = sum_i Q[i, c] w[i] for c < ncol: block (chunk, c) sums rows of its chunk into
// part[chunk * ncol + c]; lanczos_sum_kernel adds the chunks in order (deterministic).
static __global__ void lanczos_qtw_kernel(int n, int ncol, int rows, const double* __restrict__ Q,
                                          const double* __restrict__ w, double* __restrict__ part) {
  const int c = blockIdx.y, ch = blockIdx.x;
  const int r0 = ch * rows, r1 = min(n, r0 + rows);
  double acc = 0.0;
  const double* q = Q + (int64_t)c * n;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) acc += q[i] * w[i];
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
    if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(int64_t)ch * ncol + c] = sh[0];
}

static __global__ void lanczos_sum_kernel(int nch, int ncol, const double* __restrict__ part, double* __restrict__ h) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int ch = 0; ch < nch; ++ch) s += part[(int64_t)ch * ncol + c];
    h[c] = s;
  }
}

// w[i] -= sum_{c < ncol} Q[i, c] h[c]   (Q column-major, n rows)
static __global__ void lanczos_axpy_kernel(int n, int ncol, const double* __restrict__ Q, const double* __restrict__ h,
                                           double* __restrict__ w) {
  extern __shared__ double hs[];
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) hs[c] = h[c];
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int c = 0; c < ncol; ++c) acc += Q[(int64_t)c * n + i] * hs[c];
    w[i] -= acc;
  }
}

// y = a o x (elementwise), or y = x / nrm when a is null
static __global__ void lanczos_scale_kernel(int n, const double* __restrict__ a, const double* __restrict__ x,
                                            double nrm, double* __restrict__ y) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    y[i] = a ? a[i] * x[i] : x[i] / nrm;
}

// v[j] = -(1 / np) sum over test points p and slots c with nbr[p, c] = j of Ap[p, c]: the mean of
// the columns of B_po^T, one thread per training row over a CSR of the test neighbours sorted
// by training row (entries in a fixed order).
static __global__ void lanczos_start_kernel(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ent,
                                            const double* __restrict__ Ap, double inv_np, double* __restrict__ v) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rp[j]; e < rp[j + 1]; ++e) s -= Ap[ent[e]];
    v[j] = s * inv_np;
  }
}

// Row-major block X[i, c] = s[i] Q[i, c0 + c] (columns c < kc, zero padding up to ld).
static __global__ void lanczos_rows_kernel(int n, int kc, int ld, int c0, const double* __restrict__ s,
                                           const double* __restrict__ Q, double* __restrict__ X) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), c = (int)(e % ld);
    X[e] = c < kc ? s[i] * Q[(int64_t)(c0 + c) * n + i] : 0.0;
  }
}

// Z[p, c0 + c] = -sum_slot Ap[p, slot] U[nbr[p, slot], c] for c < kc (U row-major n x ld).
static __global__ void lanczos_gather_kernel(int np, int m, int kc, int ld, int c0, int k,
                                             const int32_t* __restrict__ nbr, const double* __restrict__ Ap,
                                             const double* __restrict__ U, double* __restrict__ Z) {
  const int p = blockIdx.x;
  for (int c = threadIdx.x; c < kc; c += blockDim.x) {
    double z = 0.0;
    for (int sl = 0; sl < m; ++sl) {
      const int j = nbr[(int64_t)p * m + sl];
      if (j >= 0) z -= Ap[(int64_t)p * m + sl] * U[(int64_t)j * ld + c];
    }
    Z[(int64_t)p * k + c0 + c] = z;
  }
}

// var[p] = Dp[p] + z_p^T T^{-1} z_p with T = L diag(d) L^T (l: the k - 1 subdiagonal entries of L):
// forward substitution w = L^{-1} z, then sum w_i^2 / d_i.
static __global__ void lanczos_quad_kernel(int np, int k, const double* __restrict__ Z, const double* __restrict__ l,
                                           const double* __restrict__ d, const double* __restrict__ Dp,
                                           double* __restrict__ var) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    const double* z = Z + (int64_t)p * k;
    double w = 0.0, sum = 0.0;
    for (int i = 0; i < k; ++i) {
      w = z[i] - (i > 0 ? l[i - 1] * w : 0.0);
      sum += w * w / d[i];
    }
    var[p] = Dp[p] + sum;
  }
}

}  // namespace vl
