// vl_apply_A_noalloc: the product (W + B^T D^{-1} B) X without any device
// allocation, for callers that may not allocate at call time.
//
// Some callers cannot reserve device memory when they call in: a process that has
// handed all free device memory to its own pool before this library was loaded,
// or host code on a latency-critical path that must not enter the CUDA allocator.
// vl_apply already avoids cudaMalloc, but it carves its intermediate blocks out
// of the context workspace, so it fails when that workspace is full. This variant
// keeps its intermediates in a fixed array compiled into the library instead.
//
// The array below lives in every device that loads the library, for the life of
// the process. Its device address is looked up once per device (with that device
// current) by the first call made on a context of that device; that first call
// should therefore be made before any stream capture begins. All calls share the
// array and each call overwrites it completely before reading it, so nothing
// carries over between calls; two calls whose work overlaps on the GPU (for
// example on different streams) race on it and must be serialised by the caller.
#include <cstdio>
#include <map>
#include <mutex>

#include "engine.cuh"

struct vl_state : vl::State {};   // the same definition as in api.cu

namespace vl {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;   // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_addr;   // device -> device address of g_noalloc_scratch

// Xs[s, c] = X[s2u[s], c] for c < t, zero in the padding columns.
__global__ void na_to_storage_kernel(int n, int t, int ld, const int32_t* __restrict__ s2u,
                                     const double* __restrict__ X, double* __restrict__ Xs) {
  const int64_t total = (int64_t)n * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / ld), c = (int)(e % ld);
    Xs[e] = c < t ? X[(int64_t)s2u[s] * t + c] : 0.0;
  }
}

__global__ void na_from_storage_kernel(int n, int t, int ld, const int32_t* __restrict__ s2u,
                                       const double* __restrict__ Zs, double* __restrict__ Y) {
  const int64_t total = (int64_t)n * t;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / t), c = (int)(e % t);
    Y[(int64_t)s2u[s] * t + c] = Zs[(int64_t)s * ld + c];
  }
}

__global__ void na_dinv_kernel(int n, const double* __restrict__ D, double* __restrict__ Dinv) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) Dinv[s] = 1.0 / D[s];
}

vl_status noalloc_scratch(Ctx* c, char** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_addr.find(c->device);
  if (it != g_noalloc_addr.end()) {
    *out = static_cast<char*>(it->second);
    return VL_OK;
  }
  int prev = 0;
  VL_CUDA(c, cudaGetDevice(&prev));
  VL_CUDA(c, cudaSetDevice(c->device));
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  const cudaError_t e2 = cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(no-allocation scratch)");
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaSetDevice");
  g_noalloc_addr[c->device] = p;
  *out = static_cast<char*>(p);
  return VL_OK;
}

// Device (or managed) memory of the given device: the kernels of this call run on the
// context's device and must not touch another GPU's memory.
bool on_device(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return device_memory_usable(a.type, a.device, device);
}

}  // namespace
}  // namespace vl

extern "C" vl_status vl_apply_A_noalloc(vl_state* st, const double* X, int t, double* Y) {
  using namespace vl;
  if (!st) return VL_ERR_INVALID_ARG;
  State* S = static_cast<State*>(st);
  Ctx* c = S->ctx;
  Factor* f = S->f;
  if (!X || !Y || t < 1 || t > 256)
    return fail(c, VL_ERR_INVALID_ARG, "vl_apply_A_noalloc: X and Y must be non-null and 1 <= t <= 256");
  if (!on_device(X, c->device) || !on_device(Y, c->device))
    return fail(c, VL_ERR_INVALID_ARG, "vl_apply_A_noalloc: X and Y must be device pointers on the context's device");
  const int n = (int)f->n, m = f->m;
  const int ld = Engine<double>::lead(t);
  const size_t vec = (size_t)n * ld * sizeof(double);
  const size_t vec_al = (vec + 255) / 256 * 256;
  const size_t need = 3 * vec_al + (size_t)n * sizeof(double);
  if (need > kNoAllocScratchBytes) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "vl_apply_A_noalloc: n = %d, t = %d needs %zu bytes of scratch, above the fixed limit of %zu bytes "
             "(64 MiB); use vl_apply",
             n, t, need, kNoAllocScratchBytes);
    return fail(c, VL_ERR_INVALID_ARG, buf);
  }
  char* base = nullptr;
  VL_TRY(noalloc_scratch(c, &base));
  double* Xs = reinterpret_cast<double*>(base);
  double* Ys = reinterpret_cast<double*>(base + vec_al);
  double* Zs = reinterpret_cast<double*>(base + 2 * vec_al);
  double* Dinv = reinterpret_cast<double*>(base + 3 * vec_al);
  const int64_t tot = (int64_t)n * ld;
  na_to_storage_kernel<<<grid_for(c, tot), 256, 0, VL_STREAM(c)>>>(n, t, ld, f->s2u, X, Xs);
  na_dinv_kernel<<<grid_for(c, n), 256, 0, VL_STREAM(c)>>>(n, f->D64, Dinv);
  const int g = std::max(1, std::min((n + 7) / 8, c->num_sms * 8));
  if (t == 1) {
    spmv_B_t1_kernel<double, 8><<<g, 256, 0, VL_STREAM(c)>>>(n, m, f->nbr, f->A64, Xs, Dinv, Ys);
    spmv_Bt_t1_kernel<double, 8><<<g, 256, 0, VL_STREAM(c)>>>(n, f->rowptrT, f->colT, f->valT64, Ys, nullptr, Xs,
                                                              S->W, Zs);
  } else {
    with_shape<double>(ld, [&](auto L, auto N, auto U) {
      constexpr int LPV = decltype(L)::value, NV = decltype(N)::value, UNR = decltype(U)::value;
      spmv_B_kernel<double, LPV, NV, UNR><<<g, 256, 0, VL_STREAM(c)>>>(n, m, f->nbr, f->A64, Xs, ld, Dinv, Ys);
      spmv_Bt_kernel<double, LPV, NV, UNR><<<g, 256, 0, VL_STREAM(c)>>>(n, f->rowptrT, f->colT, f->valT64, Ys, nullptr,
                                                                        Xs, S->W, ld, Zs);
      return VL_OK;
    });
  }
  na_from_storage_kernel<<<grid_for(c, (int64_t)n * t), 256, 0, VL_STREAM(c)>>>(n, t, ld, f->s2u, Zs, Y);
  VL_CUDA(c, cudaGetLastError());
  return VL_OK;
}
