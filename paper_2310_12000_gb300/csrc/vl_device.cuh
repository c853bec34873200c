// Device helpers shared by the libvl kernels.
#pragma once

#include <cstdint>

#include "vl_internal.h"

namespace vl {

constexpr double kSqrt3 = 1.7320508075688772;   // sqrt(3) rounded to float64

// Upper bound on one bounded wait, in SM clock cycles (about 2 s at 2 GHz).
constexpr long long kSpinLimitCycles = 4000000000LL;

// ----------------------------------------------------------------------------- memory order
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }

// Records the first device-side error and asks every bounded wait to stop.
__device__ __forceinline__ void raise_error(DevStatus* st, int code, int row) {
  if (atomicCAS(&st->code, 0, code) == 0) st->row = row;
  atomicExch(&st->abort, 1);
}

// Bounded wait until pred() holds. Returns false (after recording VL_ERR_TIMEOUT)
// when the wait runs past the status block's limit (kSpinLimitCycles unless a
// positive limit was set on the context), or at once when another wait aborted.
template <typename Pred>
__device__ __forceinline__ bool bounded_wait(Pred pred, DevStatus* st, int row) {
  if (pred()) return true;
  long long t0 = clock64();
  const long long set = *(volatile const long long*)&st->limit;
  const long long limit = set > 0 ? set : kSpinLimitCycles;
  for (int it = 1;; ++it) {
    if (pred()) return true;
    if ((it & 31) == 0) {
      if (ld_volatile(&st->abort)) return false;
      if (clock64() - t0 > limit) {
        raise_error(st, VL_ERR_TIMEOUT, row);
        return false;
      }
    }
    __nanosleep(it < 4 ? 32 : (it < 16 ? 64 : 256));
  }
}

// ----------------------------------------------------------------------------- geometry
// Squared distance with every operation rounded separately (no contraction), the
// key that makes neighbour sets bit-exact.
__device__ __forceinline__ double dist2_exact(double ax, double ay, double bx, double by) {
  double dx = __dsub_rn(ax, bx);
  double dy = __dsub_rn(ay, by);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// c(h) for the supported covariance families (float64). Host-callable for checks on the CPU
// (there the product sqrt(3) h is an ordinary, separately rounded multiply).
__host__ __device__ __forceinline__ double cov_eval(double h, int cov, double sigma2, double rho) {
  if (cov == VL_COV_EXPONENTIAL) return sigma2 * exp(-h / rho);
#ifdef __CUDA_ARCH__
  double a = __dmul_rn(kSqrt3, h) / rho;
#else
  double a = (kSqrt3 * h) / rho;
#endif
  return sigma2 * (1.0 + a) * exp(-a);
}

// ----------------------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror & Shaw (SC'11): 10 rounds of two 64x64 -> 128-bit products
// with the key bumped by the Weyl constants between rounds.
struct Philox4 {
  uint64_t v[4];
};
// High word of the 64 x 64 -> 128-bit product. The host form (for checks on the CPU) sums the
// four 32 x 32-bit partial products, so it needs no 128-bit integer type.
__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  const uint64_t al = a & 0xFFFFFFFFull, ah = a >> 32, bl = b & 0xFFFFFFFFull, bh = b >> 32;
  const uint64_t ll = al * bl, lh = al * bh, hl = ah * bl, hh = ah * bh;
  const uint64_t mid = (ll >> 32) + (lh & 0xFFFFFFFFull) + (hl & 0xFFFFFFFFull);
  return hh + (lh >> 32) + (hl >> 32) + (mid >> 32);
#endif
}
__host__ __device__ __forceinline__ Philox4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                          uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t lo0 = M0 * c0, hi0 = mulhi64(M0, c0);
    uint64_t lo1 = M1 * c2, hi1 = mulhi64(M1, c2);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  Philox4 o;
  o.v[0] = c0;
  o.v[1] = c1;
  o.v[2] = c2;
  o.v[3] = c3;
  return o;
}

// ----------------------------------------------------------------------------- warp
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

}  // namespace vl
