// Rank-k pivoted Cholesky factor of Sigma for the LRAC preconditioner (Section 3.1.2):
// k steps of three launches (pick the pivot, write its column and update the
// residual diagonal, which also yields the per-block candidates for the next pivot).
#include <algorithm>
#include <string>

#include "engine.cuh"

namespace vl {

void lrac_drop(Factor* f) {
  if (f->lrac_mem.ctx) f->lrac_mem.free_all();
  f->lrac_k = 0;
  f->L64 = nullptr;
  f->L32 = nullptr;
  f->piv_s = nullptr;
  f->piv_v = nullptr;
}

vl_status lrac_build(Factor* f, int k) {
  Ctx* c = f->ctx;
  if (f->lrac_k == k && f->L64) return VL_OK;
  if (k < 1 || k > kMaxRank || k > f->n)
    return fail(c, VL_ERR_INVALID_ARG, "LRAC rank k must satisfy 1 <= k <= min(n, " + std::to_string(kMaxRank) + ")");
  lrac_drop(f);
  f->lrac_mem.ctx = c;
  const int n = (int)f->n;
  f->L64 = f->lrac_mem.get<double>((size_t)n * k);
  f->piv_s = f->lrac_mem.get<int32_t>(k);
  f->piv_v = f->lrac_mem.get<int32_t>(k);
  if (!f->L64 || !f->piv_s || !f->piv_v) {
    lrac_drop(f);
    return fail(c, VL_ERR_OOM, "workspace exhausted (LRAC factor)");
  }
  const int grid = std::max(1, std::min((n + 255) / 256, c->num_sms * 8));
  Owned tmp;
  tmp.ctx = c;
  double* d = tmp.get<double>(n);
  double* dpiv = tmp.get<double>(k);
  PivotBest* part = tmp.get<PivotBest>(grid);
  int* bad = tmp.get<int>(1);
  auto done = [&](vl_status s) {
    cudaStreamSynchronize(c->stream);
    tmp.free_all();
    if (s != VL_OK) lrac_drop(f);
    return s;
  };
  if (!d || !dpiv || !part || !bad) return done(fail(c, VL_ERR_OOM, "workspace exhausted (pivoted Cholesky)"));
  {
    ProfScope ps(c, "pivoted_cholesky", k);
    cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
    pchol_init_kernel<<<grid, 256, 0, VL_STREAM(c)>>>(n, f->sigma2 + f->nugget, f->s2v, d, part);
    for (int j = 0; j < k; ++j) {
      pchol_pick_kernel<<<1, 32, 0, VL_STREAM(c)>>>(grid, part, j, f->piv_s, f->piv_v, dpiv, bad);
      pchol_column_kernel<<<grid, 256, sizeof(double) * j, VL_STREAM(c)>>>(
          n, j, f->locs_s, f->s2v, f->cov, f->sigma2, f->rho, f->nugget, f->piv_s, dpiv, f->L64, d, part);
    }
  }
  if (cudaGetLastError() != cudaSuccess) return done(fail(c, VL_ERR_CUDA, "pivoted Cholesky launch"));
  int hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return done(fail(c, VL_ERR_CUDA, "pivoted Cholesky"));
  if (hbad)
    return done(fail(c, VL_ERR_NOT_SPD,
                     "LRAC pivoted Cholesky: residual diagonal not positive at step " + std::to_string(hbad - 1) +
                         " (k exceeds the numerical rank of Sigma)"));
  f->lrac_k = k;
  return done(VL_OK);
}

vl_status lrac_float(Factor* f) {
  Ctx* c = f->ctx;
  if (f->L32) return VL_OK;
  if (!f->L64) return fail(c, VL_ERR_STATE, "LRAC factor not built");
  const int64_t total = f->n * (int64_t)f->lrac_k;
  f->L32 = f->lrac_mem.get<float>(total);
  if (!f->L32) return fail(c, VL_ERR_OOM, "workspace exhausted (LRAC float factor)");
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)c->num_sms * 16));
  convert_kernel<double, float><<<grid, 256, 0, VL_STREAM(c)>>>(total, f->L64, f->L32);
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}

}  // namespace vl
