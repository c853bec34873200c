// LRAC preconditioner (Section 3.1.2, Eq. P_LRAC; Eqs. pcls2 and logdetsplit2):
//   P = L_k L_k^T + W^{-1},  L_k the rank-k pivoted Cholesky factor of the covariance
//   Sigma of the Vecchia-ordered points (nugget on its diagonal), not of Sigma_tilde.
//   P^{-1} R = W R - W L C^{-1} L^T W R,  C = I_k + L^T W L         (Woodbury identity)
//   log det P = log det C - sum_i log W_i                            (determinant lemma)
// so log det(Sigma_tilde W + I) = log det C + log det(P^{-1/2}(Sigma_tilde + W^{-1})P^{-T/2}).
//
// L_k depends only on the covariance parameters and is built once per factor; C, its
// Cholesky factor and C^{-1} depend on W and are rebuilt whenever W changes.
//
// Layout: L is column-major over the storage rows (n x k, column j contiguous), so
// the pivoted Cholesky writes one coalesced column per step and the rank-k products
// read coalesced 32-row segments of each column. k x k matrices are row-major float64.
//
// Products with L (all deterministic: fixed chunking and fixed-order sums):
//   G = L^T (w o X)   split over row chunks, per-chunk partials summed in float64
//   Z = a o Y + beta (b o (L V))
// In float32 the per-thread accumulators of G are flushed into float64 every 32 rows.
#pragma once

#include <climits>

#include "kernels.cuh"

namespace vl {

// ----------------------------------------------------------------------------- pivoted Cholesky
// Harbrecht, Peters & Schneider (2012): residual diagonal d (initially diag Sigma),
// pivot p = argmax d (ties to the lowest Vecchia index), column
//   L[:, j] = (Sigma[:, p] - L[:, :j] L[p, :j]^T) / sqrt(d_p),   d -= L[:, j]^2,  d_p = 0,
// exactly k steps, float64 throughout.
struct PivotBest {
  double d;
  int v;   // Vecchia index (tie break)
  int s;   // storage row
};

__device__ __forceinline__ bool pivot_better(double d1, int v1, double d2, int v2) {
  return d1 > d2 || (d1 == d2 && v1 < v2);
}

// Block-wide reduction of (d, v, s) candidates; thread 0 writes the block's best.
__device__ __forceinline__ void pivot_block_reduce(double bd, int bv, int bs, PivotBest* out) {
  __shared__ double sd[32];
  __shared__ int sv[32], ss[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    const double od = __shfl_down_sync(0xffffffffu, bd, o);
    const int ov = __shfl_down_sync(0xffffffffu, bv, o);
    const int os = __shfl_down_sync(0xffffffffu, bs, o);
    if (pivot_better(od, ov, bd, bv)) {
      bd = od;
      bv = ov;
      bs = os;
    }
  }
  if (lane == 0) {
    sd[wid] = bd;
    sv[wid] = bv;
    ss[wid] = bs;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    bd = lane < nw ? sd[lane] : -INFINITY;
    bv = lane < nw ? sv[lane] : INT_MAX;
    bs = lane < nw ? ss[lane] : -1;
    for (int o = 16; o > 0; o >>= 1) {
      const double od = __shfl_down_sync(0xffffffffu, bd, o);
      const int ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int os = __shfl_down_sync(0xffffffffu, bs, o);
      if (pivot_better(od, ov, bd, bv)) {
        bd = od;
        bv = ov;
        bs = os;
      }
    }
    if (lane == 0) *out = PivotBest{bd, bv, bs};
  }
}

// d = sigma2 + nugget; per-block best for the first pivot.
static __global__ void pchol_init_kernel(int n, double d0, const int32_t* __restrict__ s2v, double* __restrict__ d,
                                         PivotBest* __restrict__ part) {
  double bd = -INFINITY;
  int bv = INT_MAX, bs = -1;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    d[s] = d0;
    const int v = s2v[s];
    if (pivot_better(d0, v, bd, bv)) {
      bd = d0;
      bv = v;
      bs = s;
    }
  }
  pivot_block_reduce(bd, bv, bs, &part[blockIdx.x]);
}

// One thread: reduce the block bests into pivot j (storage row, Vecchia index, d_p).
// A pivot with d_p <= 0 (Sigma numerically of rank < k) sets bad = j + 1.
static __global__ void pchol_pick_kernel(int nb, const PivotBest* __restrict__ part, int j, int32_t* __restrict__ piv_s,
                                         int32_t* __restrict__ piv_v, double* __restrict__ dpiv, int* __restrict__ bad) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  PivotBest b{-INFINITY, INT_MAX, -1};
  for (int i = 0; i < nb; ++i)
    if (pivot_better(part[i].d, part[i].v, b.d, b.v)) b = part[i];
  if (!(b.d > 0.0) || b.s < 0) {
    if (*bad == 0) *bad = j + 1;
    b.d = 1.0;   // keep the remaining steps finite; the host reports the breakdown
    if (b.s < 0) b.s = 0;
  }
  piv_s[j] = b.s;
  piv_v[j] = b.v;
  dpiv[j] = b.d;
}

// Column j of L, the diagonal update, and per-block bests for pivot j + 1.
static __global__ void pchol_column_kernel(int n, int j, const double* __restrict__ locs, const int32_t* __restrict__ s2v,
                                           int cov, double sigma2, double rho, double nugget,
                                           const int32_t* __restrict__ piv_s, const double* __restrict__ dpiv,
                                           double* __restrict__ L, double* __restrict__ d, PivotBest* __restrict__ part) {
  extern __shared__ double Lp[];   // row p of L, columns 0 .. j-1
  const int p = piv_s[j];
  for (int q = threadIdx.x; q < j; q += blockDim.x) Lp[q] = L[(int64_t)q * n + p];
  __syncthreads();
  const double inv = 1.0 / sqrt(dpiv[j]);
  const double px = locs[2 * (int64_t)p], py = locs[2 * (int64_t)p + 1];
  double bd = -INFINITY;
  int bv = INT_MAX, bs = -1;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const double dx = __dsub_rn(locs[2 * (int64_t)s], px), dy = __dsub_rn(locs[2 * (int64_t)s + 1], py);
    double col = cov_eval(sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))), cov, sigma2, rho);
    if (s == p) col += nugget;
    double acc = 0.0;
    for (int q = 0; q < j; ++q) acc = fma(L[(int64_t)q * n + s], Lp[q], acc);
    const double l = (col - acc) * inv;
    L[(int64_t)j * n + s] = l;
    const double dn = (s == p) ? 0.0 : d[s] - l * l;
    d[s] = dn;
    const int v = s2v[s];
    if (pivot_better(dn, v, bd, bv)) {
      bd = dn;
      bv = v;
      bs = s;
    }
  }
  pivot_block_reduce(bd, bv, bs, &part[blockIdx.x]);
}

// ----------------------------------------------------------------------------- G = L^T (w o X)
// part[chunk][q][c] over the rows of one chunk. L column-major (n x k); X element
// (s, c) at X[s * xs + c * xc]: row-major blocks (xs = ld, xc = 1) or another
// column-major matrix (xs = 1, xc = n, the Gram L^T W L). w may be null (ones).
// Block tile 64 (q) x 64 (c), 32 rows per step, 256 threads with 4 x 4 outputs each.
// sym (the Gram): tiles with q0 < c0 are skipped; lrac_sum_chunks_kernel mirrors them.
template <typename T>
__global__ void __launch_bounds__(256) lrac_tn_kernel(int n, int k, int tc, int rows_per_chunk, const T* __restrict__ L,
                                                      const T* __restrict__ X, int64_t xs, int64_t xc,
                                                      const T* __restrict__ w, int sym, double* __restrict__ part) {
  __shared__ T sA[32][64 + 1];
  __shared__ T sX[32][64 + 1];
  if (sym && blockIdx.x < blockIdx.y) return;
  const int q0 = blockIdx.x * 64, c0 = blockIdx.y * 64, chunk = blockIdx.z;
  const int r0 = chunk * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // c = c0 + tx + 16 v, q = q0 + ty + 16 u
  double acc[4][4];
  T tmp[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
  const bool xcol = (xc != 1);   // X column-major
  for (int s0 = r0; s0 < r1; s0 += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int r = e & 31, cc = e >> 5, s = s0 + r;   // row-fastest: coalesced column segments
      const int q = q0 + cc;
      sA[r][cc] = (s < r1 && q < k) ? L[(int64_t)q * n + s] : T(0);
      if (xcol) {
        const int c = c0 + cc;
        sX[r][cc] = (s < r1 && c < tc) ? X[(int64_t)c * xc + s] * (w ? w[s] : T(1)) : T(0);
      }
    }
    if (!xcol) {
      for (int e = threadIdx.x; e < 32 * 64; e += 256) {
        const int cc = e & 63, r = e >> 6, s = s0 + r, c = c0 + cc;   // column-fastest: contiguous rows
        sX[r][cc] = (s < r1 && c < tc) ? X[(int64_t)s * xs + c] * (w ? w[s] : T(1)) : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) tmp[u][v] = T(0);
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      T a[4], x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = sA[r][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 4; ++v) x[v] = sX[r][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) tmp[u][v] = fma(a[u], x[v], tmp[u][v]);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += (double)tmp[u][v];
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int q = q0 + ty + 16 * u;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + tx + 16 * v;
      if (q < k && c < tc) part[((int64_t)chunk * k + q) * tc + c] = acc[u][v];
    }
  }
}

// Single right-hand side: part[chunk][q] = sum over the chunk of L[s, q] w_s x_s.
// One warp per column q; lanes stride the rows.
template <typename T>
__global__ void __launch_bounds__(256) lrac_tn1_kernel(int n, int k, int rows_per_chunk, const T* __restrict__ L,
                                                       const T* __restrict__ x, const T* __restrict__ w,
                                                       double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int q = blockIdx.x * 8 + (threadIdx.x >> 5), chunk = blockIdx.y;
  if (q >= k) return;
  const int r0 = chunk * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const T* Lq = L + (int64_t)q * n;
  double acc = 0.0;
  for (int b = r0; b < r1; b += 32 * 16) {
    T tmp = T(0);
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      const int s = b + i * 32 + lane;
      if (s < r1) tmp = fma(Lq[s], x[s] * (w ? w[s] : T(1)), tmp);
    }
    acc += (double)tmp;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) part[(int64_t)chunk * k + q] = acc;
}

// out[e] = sum over chunks of part[chunk][e] (fixed order). gram_k > 0: the output is
// the k x k matrix I + L^T W L, built from its lower triangle (the tiles above the
// diagonal were skipped) so that it is exactly symmetric.
static __global__ void lrac_sum_chunks_kernel(int nchunk, int64_t kt, const double* __restrict__ part,
                                              double* __restrict__ out, int gram_k) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kt; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t src = e;
    if (gram_k > 0) {
      const int64_t q = e / gram_k, c = e % gram_k;
      if (q < c) src = c * gram_k + q;   // exact symmetry
    }
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ++ch) s += part[(int64_t)ch * kt + src];
    if (gram_k > 0 && e / gram_k == e % gram_k) s += 1.0;
    out[e] = s;
  }
}

// ----------------------------------------------------------------------------- Z = a o Y + beta b o (L V)
// V: k x t float64 row-major. Z, Y: n x ld (row-major, padding columns written 0).
// a, b may be null (a = 0: no Y term; b = 1). Block tile 64 rows x 64 columns over
// ranks in steps of 32; 256 threads with 4 x 4 outputs each.
template <typename T>
__global__ void __launch_bounds__(256) lrac_nn_kernel(int n, int k, int t, int ld, const T* __restrict__ L,
                                                      const double* __restrict__ V, const T* __restrict__ Y,
                                                      const T* __restrict__ a, const T* __restrict__ b, T beta,
                                                      T* __restrict__ Z) {
  __shared__ T sL[32][64 + 1];
  __shared__ T sV[32][64 + 1];
  const int s0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // c = c0 + tx + 16 v, s = s0 + ty + 16 u
  T acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
  for (int q0 = 0; q0 < k; q0 += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int r = e & 63, qq = e >> 6, s = s0 + r, q = q0 + qq;   // row-fastest
      sL[qq][r] = (s < n && q < k) ? L[(int64_t)q * n + s] : T(0);
      const int c = c0 + r;
      sV[qq][r] = (q < k && c < t) ? (T)V[(int64_t)q * t + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int qq = 0; qq < 32; ++qq) {
      T l[4], v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) l[u] = sL[qq][ty + 16 * u];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = sV[qq][tx + 16 * j];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[u][j] = fma(l[u], v[j], acc[u][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int s = s0 + ty + 16 * u;
    if (s >= n) continue;
    const T as = a ? a[s] : T(0), bs = (b ? b[s] : T(1)) * beta;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx + 16 * j;
      if (c < t) {
        const T y = (a && Y) ? Y[(int64_t)s * ld + c] : T(0);
        Z[(int64_t)s * ld + c] = as * y + bs * acc[u][j];
      } else if (c < ld) {
        Z[(int64_t)s * ld + c] = T(0);
      }
    }
  }
}

// Single column: z_s = a_s y_s + beta b_s sum_q L[s, q] v_q; v staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) lrac_nn1_kernel(int n, int k, const T* __restrict__ L, const double* __restrict__ v,
                                                       const T* __restrict__ y, const T* __restrict__ a,
                                                       const T* __restrict__ b, T beta, T* __restrict__ z) {
  extern __shared__ unsigned char sm_raw[];
  T* sv = reinterpret_cast<T*>(sm_raw);
  for (int q = threadIdx.x; q < k; q += blockDim.x) sv[q] = (T)v[q];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  T acc0 = T(0), acc1 = T(0);
  int q = 0;
  for (; q + 1 < k; q += 2) {
    acc0 = fma(L[(int64_t)q * n + s], sv[q], acc0);
    acc1 = fma(L[(int64_t)(q + 1) * n + s], sv[q + 1], acc1);
  }
  if (q < k) acc0 = fma(L[(int64_t)q * n + s], sv[q], acc0);
  const T as = a ? a[s] : T(0), bs = (b ? b[s] : T(1)) * beta;
  z[s] = ((a && y) ? as * y[s] : T(0)) + bs * (acc0 + acc1);
}

// ----------------------------------------------------------------------------- k x k, float64
// Blocked lower Cholesky C = R R^T in place (row-major, float64), panels of 32
// columns: lrac_chol_panel_kernel factors the diagonal block (in shared memory, in
// every block) and solves the rows below it, R[i, J:J+b] = C[i, J:J+b] R_JJ^{-T};
// lrac_chol_update_kernel subtracts the panel's outer product from the trailing lower
// triangle. *logdet accumulates 2 sum log R_jj (block 0 of each panel, in order);
// a non-positive pivot sets *bad.
constexpr int kCholNB = 32;

static __global__ void __launch_bounds__(128) lrac_chol_panel_kernel(int k, int J, double* __restrict__ C,
                                                                     double* __restrict__ logdet, int* __restrict__ bad) {
  __shared__ double Dg[kCholNB][kCholNB + 1];
  const int b = min(kCholNB, k - J);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Dg[e / b][e % b] = C[(int64_t)(J + e / b) * k + J + e % b];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int j = 0; j < b; ++j) {
      if (lane == 0) {
        const double v = Dg[j][j];
        if (!(v > 0.0)) *bad = 1;
        Dg[j][j] = v > 0.0 ? sqrt(v) : 1.0;
      }
      __syncwarp();
      const double ip = 1.0 / Dg[j][j];
      for (int i = j + 1 + lane; i < b; i += 32) Dg[i][j] *= ip;
      __syncwarp();
      for (int i = j + 1 + lane; i < b; i += 32)
        for (int c = j + 1; c <= i; ++c) Dg[i][c] -= Dg[i][j] * Dg[c][j];
      __syncwarp();
    }
  }
  __syncthreads();
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
      const int i = e / b, c = e % b;
      if (c <= i) C[(int64_t)(J + i) * k + J + c] = Dg[i][c];
    }
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int j = 0; j < b; ++j) s += log(Dg[j][j]);
      *logdet += 2.0 * s;
    }
  }
  const int i = J + b + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double x[kCholNB];
#pragma unroll
  for (int j = 0; j < kCholNB; ++j) x[j] = j < b ? C[(int64_t)i * k + J + j] : 0.0;
#pragma unroll
  for (int j = 0; j < kCholNB; ++j) {
    if (j < b) {
      double a = x[j];
#pragma unroll
      for (int l = 0; l < j; ++l) a -= x[l] * Dg[j][l];
      x[j] = a / Dg[j][j];
    }
  }
#pragma unroll
  for (int j = 0; j < kCholNB; ++j)
    if (j < b) C[(int64_t)i * k + J + j] = x[j];
}

// C[i][c] -= sum_{l in panel} C[i][l] C[c][l] for J + b <= c <= i < k; 32 x 32 tiles.
static __global__ void __launch_bounds__(256) lrac_chol_update_kernel(int k, int J, double* __restrict__ C) {
  const int b = min(kCholNB, k - J), T0 = J + b;
  const int ti = blockIdx.y, tcx = blockIdx.x;
  if (tcx > ti) return;
  const int i0 = T0 + ti * 32, c0 = T0 + tcx * 32;
  __shared__ double Pi[32][kCholNB + 1], Pc[32][kCholNB + 1];
  for (int e = threadIdx.x; e < 32 * kCholNB; e += blockDim.x) {
    const int r = e / kCholNB, l = e % kCholNB;
    Pi[r][l] = (i0 + r < k && l < b) ? C[(int64_t)(i0 + r) * k + J + l] : 0.0;
    Pc[r][l] = (c0 + r < k && l < b) ? C[(int64_t)(c0 + r) * k + J + l] : 0.0;
  }
  __syncthreads();
  const int cc = threadIdx.x & 31;
  for (int ri = threadIdx.x >> 5; ri < 32; ri += 8) {
    const int i = i0 + ri, c = c0 + cc;
    if (i >= k || c > i) continue;
    double a = 0.0;
#pragma unroll 8
    for (int l = 0; l < kCholNB; ++l) a = fma(Pi[ri][l], Pc[cc][l], a);
    C[(int64_t)i * k + c] -= a;
  }
}

// Rinv = R^{-1} (lower, upper part written 0). A block owns 16 columns j0 .. j0+15 and
// keeps them in shared memory (k x 16); rows are produced in order, each as a dot
// product over l split across 16 slices of threads and summed in a fixed order.
constexpr int kMaxRank = 1024;

static __global__ void __launch_bounds__(256) lrac_trinv_kernel(int k, const double* __restrict__ R,
                                                                double* __restrict__ Rinv) {
  extern __shared__ double X[];   // k x 16, then 16 x 16 partials
  double* part = X + (size_t)k * 16;
  const int j0 = blockIdx.x * 16, jj = threadIdx.x & 15, slice = threadIdx.x >> 4;
  const int j = j0 + jj;
  for (int i = j0; i < k; ++i) {
    // a = sum_{l in [j0, i)} R[i][l] X[l][jj]   (X[l][jj] = 0 for l < j)
    double a = 0.0;
    for (int l = j0 + slice; l < i; l += 16) a = fma(R[(int64_t)i * k + l], X[(size_t)(l - j0) * 16 + jj], a);
    part[slice * 16 + jj] = a;
    __syncthreads();
    if (slice == 0) {
      double s = 0.0;
      for (int q = 0; q < 16; ++q) s += part[q * 16 + jj];
      const double rii = R[(int64_t)i * k + i];
      X[(size_t)(i - j0) * 16 + jj] = (j >= k || i < j) ? 0.0 : (i == j ? 1.0 / rii : -s / rii);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < k * 16; e += blockDim.x) {
    const int i = e / 16, c = e % 16;
    if (j0 + c < k) Rinv[(int64_t)i * k + j0 + c] = i < j0 ? 0.0 : X[(size_t)(i - j0) * 16 + c];
  }
}

// Cinv = Rinv^T Rinv: Cinv[i][c] = sum_{l >= max(i, c)} Rinv[l][i] Rinv[l][c]
// (computed for i <= c and mirrored, so Cinv is exactly symmetric).
// The sum starts at max(i, first column of the block) so that a warp reads rows of
// Rinv together; the terms with l < c are exact zeros.
static __global__ void lrac_cinv_kernel(int k, const double* __restrict__ Rinv, double* __restrict__ Cinv) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (c >= k || c < i) return;
  double a0 = 0.0, a1 = 0.0;
  int l = max(i, (int)(blockIdx.x * blockDim.x));
  for (; l + 1 < k; l += 2) {
    a0 = fma(Rinv[(int64_t)l * k + i], Rinv[(int64_t)l * k + c], a0);
    a1 = fma(Rinv[(int64_t)(l + 1) * k + i], Rinv[(int64_t)(l + 1) * k + c], a1);
  }
  if (l < k) a0 = fma(Rinv[(int64_t)l * k + i], Rinv[(int64_t)l * k + c], a0);
  Cinv[(int64_t)i * k + c] = a0 + a1;
  Cinv[(int64_t)c * k + i] = a0 + a1;
}

// V = Cinv G (k x k times k x t, float64): one thread per (row i, column c).
static __global__ void lrac_cinv_apply_kernel(int k, int t, const double* __restrict__ Cinv, const double* __restrict__ G,
                                              double* __restrict__ V) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (c >= t) return;
  const double* Ci = Cinv + (int64_t)i * k;
  double a0 = 0.0, a1 = 0.0;
  int j = 0;
  for (; j + 1 < k; j += 2) {
    a0 = fma(Ci[j], G[(int64_t)j * t + c], a0);
    a1 = fma(Ci[j + 1], G[(int64_t)(j + 1) * t + c], a1);
  }
  if (j < k) a0 = fma(Ci[j], G[(int64_t)j * t + c], a0);
  V[(int64_t)i * t + c] = a0 + a1;
}

// Single column: one warp per row i, lanes split the k terms.
static __global__ void lrac_cinv_apply1_kernel(int k, const double* __restrict__ Cinv, const double* __restrict__ g,
                                               double* __restrict__ v) {
  const int lane = threadIdx.x & 31, i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= k) return;
  const double* Ci = Cinv + (int64_t)i * k;
  double a = 0.0;
  for (int j = lane; j < k; j += 32) a = fma(Ci[j], g[j], a);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) v[i] = a;
}

// X[s, c] *= w_s for c < t
template <typename T>
__global__ void scale_rows_kernel(int n, int t, int ld, const T* __restrict__ w, T* __restrict__ X) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    if (c < t) X[e] *= w[s];
  }
}

}  // namespace vl
