// Vecchia factor rows (Section 2.1), one warp per row, float64:
//   Sigma_N = [c(|s_a - s_b|)]_{a,b in N(i)} + nugget I,  v = [c(|s_a - s_i|)]_{a in N(i)}
//   Sigma_N = L L^T (Cholesky),  w = L^{-1} v,  A_i = L^{-T} w,  D_i = c(0) + nugget - w^T w
// which is A_i = Sigma_{i,N} Sigma_N^{-1} and D_i = Sigma_ii - Sigma_{N,i}^T Sigma_N^{-1} Sigma_{N,i}.
// The same kernel builds the prediction rows B_po, D_p (Section 4.1: each test
// point conditioned on training neighbours only) with self/reference locations
// taken from different arrays.
//
// A pivot <= 0 (or D_i <= 0) is reported as VL_ERR_NOT_SPD with the row.
#include "vl_device.cuh"

namespace vl {

constexpr int kFactorWarps = 4;

__device__ __forceinline__ void tri_index(int e, int& a, int& b) {
  int r = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  while (r * (r + 1) / 2 > e) --r;
  a = r;
  b = e - r * (r + 1) / 2;
}

__global__ void factor_kernel(int rows, int m, const double* __restrict__ self_locs,
                              const double* __restrict__ ref_locs, const int32_t* __restrict__ nbr, int cov,
                              double sigma2, double rho, double nugget, double* __restrict__ A,
                              double* __restrict__ D, const int32_t* __restrict__ row_ids, DevStatus* st) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int ld = m + 1;
  double* S = smem + (size_t)wib * (m * ld + 3 * m);
  double* v = S + m * ld;
  double* P = v + m;   // 2m: neighbour coordinates
  const int r = blockIdx.x * kFactorWarps + wib;
  if (r >= rows) return;
  const double sii = sigma2 + nugget;
  const double qx = self_locs[2 * (int64_t)r], qy = self_locs[2 * (int64_t)r + 1];
  // neighbours: a valid prefix followed by -1 padding
  int cnt = 0;
  for (int c0 = 0; c0 < m; c0 += 32) {
    const int c = c0 + lane;
    int j = c < m ? nbr[(int64_t)r * m + c] : -1;
    unsigned ok = __ballot_sync(0xffffffffu, j >= 0);
    cnt += __popc(ok);
    if (j >= 0) {
      P[2 * c] = ref_locs[2 * (int64_t)j];
      P[2 * c + 1] = ref_locs[2 * (int64_t)j + 1];
    }
  }
  __syncwarp();
  const int ne = cnt * (cnt + 1) / 2;
  for (int e = lane; e < ne; e += 32) {
    int a, b;
    tri_index(e, a, b);
    double dx = __dsub_rn(P[2 * a], P[2 * b]), dy = __dsub_rn(P[2 * a + 1], P[2 * b + 1]);
    double h = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    double cv = cov_eval(h, cov, sigma2, rho);
    S[a * ld + b] = (a == b) ? cv + nugget : cv;
  }
  for (int a = lane; a < cnt; a += 32) {
    double dx = __dsub_rn(P[2 * a], qx), dy = __dsub_rn(P[2 * a + 1], qy);
    v[a] = cov_eval(sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy))), cov, sigma2, rho);
  }
  __syncwarp();
  bool bad = false;
  // right-looking Cholesky, lanes over rows of the trailing block
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
  double Di = sii;
  if (!bad) {
    // w = L^{-1} v (in place)
    for (int j = 0; j < cnt; ++j) {
      const double wj = v[j] / S[j * ld + j];
      __syncwarp();
      if (lane == 0) v[j] = wj;
      for (int a = j + 1 + lane; a < cnt; a += 32) v[a] -= S[a * ld + j] * wj;
      __syncwarp();
    }
    double part = 0.0;
    for (int a = lane; a < cnt; a += 32) part += v[a] * v[a];
    Di = sii - warp_sum(part);
    // A_i = L^{-T} w (in place)
    for (int j = cnt - 1; j >= 0; --j) {
      const double aj = v[j] / S[j * ld + j];
      __syncwarp();
      if (lane == 0) v[j] = aj;
      for (int b = lane; b < j; b += 32) v[b] -= S[j * ld + b] * aj;
      __syncwarp();
    }
    if (!(Di > 0.0)) bad = true;
  }
  if (bad && lane == 0) raise_error(st, VL_ERR_NOT_SPD, row_ids ? row_ids[r] : r);
  for (int c = lane; c < m; c += 32) A[(int64_t)r * m + c] = (c < cnt && !bad) ? v[c] : 0.0;
  if (lane == 0) D[r] = bad ? NAN : Di;
}

vl_status factor_rows(Ctx* c, int64_t rows, int m, const double* self_locs, const double* ref_locs,
                      const int32_t* nbr, int cov, double sigma2, double rho, double nugget, double* A,
                      double* D, const int32_t* row_ids) {
  if (rows <= 0) return VL_OK;
  const size_t smem = sizeof(double) * (size_t)kFactorWarps * (m * (m + 1) + 3 * m + 1);
  // the attribute is per kernel and process-wide: always the bound for the largest m
  // (64), so that calls on other threads with another m never lower it under a launch
  const size_t smem_max = sizeof(double) * (size_t)kFactorWarps * (64 * 65 + 3 * 64 + 1);
  VL_CUDA(c, cudaFuncSetAttribute(factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max));
  const int grid = (int)((rows + kFactorWarps - 1) / kFactorWarps);
  ProfScope ps(c, "factor", m);
  factor_kernel<<<grid, 32 * kFactorWarps, smem, VL_STREAM(c)>>>((int)rows, m, self_locs, ref_locs, nbr, cov, sigma2, rho,
                                                              nugget, A, D, row_ids, c->dstatus);
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

}  // namespace vl
