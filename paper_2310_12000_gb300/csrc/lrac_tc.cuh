// Tensor-core (tcgen05, kind::tf32) forms of the two rank-k products of the LRAC
// Woodbury apply for float32 blocks of t <= 64 columns and rank k <= 512:
//   G = L^T (w o R)     (k x t, summed over the rows: per-chunk partials)
//   Z = a o Y + beta b o (L V)
// Each float32 operand is split into a tf32 head and its remainder, and every
// product is taken as hi*hi + hi*lo + lo*hi accumulated in float32 in tensor
// memory, which keeps about 21 bits of each operand: the preconditioner stays a
// fixed linear operator to float32 accuracy, as PCG requires.
//
// Operands are staged by the threads into shared memory in the canonical
// no-swizzle K-major layout (see tc.cuh), double buffered: while the tensor core
// works on one K chunk the threads load and split the next. One elected thread
// issues the MMAs and commits them to a per-stage mbarrier; the epilogue reads the
// accumulators back with tcgen05.ld. Every wait is bounded; on a timeout the kernel
// records VL_ERR_TIMEOUT, waits once more (bounded) and still frees its tensor memory.
#pragma once

#include "lrac.cuh"
#include "tc.cuh"

namespace vl {

constexpr int kTcN = 64;         // accumulator columns (t <= 64)
constexpr int kTcMaxRank = 512;  // four 128-row M tiles for G

// ----------------------------------------------------------------------------- V image
// Vt: for each chunk of 32 ranks, two 8 KB tiles (tf32 head, remainder) holding the
// 64 x 32 (columns x ranks) block of V in canonical K-major core-matrix order.
static __global__ void lrac_vprep_kernel(int k, int t, int nkc, const double* __restrict__ V, float* __restrict__ Vt) {
  const int total = nkc * 32 * kTcN;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int kc = e / (32 * kTcN), rem = e % (32 * kTcN), c = rem / 32, qq = rem % 32, q = kc * 32 + qq;
    const float v = (q < k && c < t) ? (float)V[(int64_t)q * t + c] : 0.f;
    float hi, lo;
    tc::split_tf32(v, hi, lo);
    const int off = (((c >> 3) * 8 + (qq >> 2)) * 32) + (c & 7) * 4 + (qq & 3);
    Vt[(int64_t)kc * 4096 + off] = hi;
    Vt[(int64_t)kc * 4096 + 2048 + off] = lo;
  }
}

// ----------------------------------------------------------------------------- Z = a o Y + beta b o (L V)
// 128 threads, one 128-row tile at a time (thread i owns row i of the tile), K
// chunks of 32 ranks; per stage: A head / remainder (16 KB each), B head / remainder
// (8 KB each). Tensor memory: 64 columns (the 128 x 64 float32 accumulator).
constexpr int kNnStage = 48 * 1024;
constexpr int kNnSmem = 2 * kNnStage + 64;

static __global__ void __launch_bounds__(128, 2)
    lrac_nn_tc_kernel(int n, int k, int t, int ld, const float* __restrict__ L, const float* __restrict__ Vt,
                      const float* __restrict__ Y, const float* __restrict__ a, const float* __restrict__ b, float beta,
                      float* __restrict__ Z, DevStatus* st) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * kNnStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * kNnStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int nkc = (k + 31) / 32, ntiles = (n + 127) / 128;
  if (warp == 0) tc::tmem_alloc(tslot, 64);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(128, kTcN);
  bool ok = true;
  uint32_t g = 0;   // chunks issued by this block

  float av[32];
  float4 bv[8];
  auto load = [&](int tile, int kc) {
    const int r = tile * 128 + tid;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int q = kc * 32 + j;
      av[j] = (r < n && q < k) ? __ldcs(&L[(int64_t)q * n + r]) : 0.f;   // streamed once per apply
    }
    const float4* src = reinterpret_cast<const float4*>(Vt + (int64_t)kc * 4096);
#pragma unroll
    for (int i = 0; i < 8; ++i) bv[i] = src[tid + 128 * i];
  };
  int tile = blockIdx.x, kc = 0;
  if (tile < ntiles) load(tile, 0);
  while (tile < ntiles) {
    const int stage = g & 1;
    const uint32_t use = g >> 1;
    unsigned char* S = sm + stage * kNnStage;
    float* Ahi = reinterpret_cast<float*>(S);
    float* Alo = reinterpret_cast<float*>(S + 16384);
    float4* B4 = reinterpret_cast<float4*>(S + 32768);
    if (use >= 1) ok &= tc::mbar_wait(&mbar[stage], (use - 1) & 1);
    // A: row rr = tid, core matrix (rr / 8, kg), row rr % 8 -> 16 bytes
#pragma unroll
    for (int kg = 0; kg < 8; ++kg) {
      float4 h, l;
      tc::split_tf32(av[4 * kg + 0], h.x, l.x);
      tc::split_tf32(av[4 * kg + 1], h.y, l.y);
      tc::split_tf32(av[4 * kg + 2], h.z, l.z);
      tc::split_tf32(av[4 * kg + 3], h.w, l.w);
      const int off = (((tid >> 3) * 8 + kg) * 32) + (tid & 7) * 4;
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) B4[tid + 128 * i] = bv[i];
    // next chunk (or the next tile's first) into registers while this one runs
    const int cur_kc = kc, cur_tile = tile;
    if (++kc == nkc) {
      kc = 0;
      tile += gridDim.x;
    }
    if (tile < ntiles) load(tile, kc);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_hi = tc::smem_u32(Ahi), a_lo = tc::smem_u32(Alo), b_hi = tc::smem_u32(B4),
                     b_lo = b_hi + 8192;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint64_t dah = tc::smem_desc(a_hi + 256 * j, 128, 1024), dal = tc::smem_desc(a_lo + 256 * j, 128, 1024);
        const uint64_t dbh = tc::smem_desc(b_hi + 256 * j, 128, 1024), dbl = tc::smem_desc(b_lo + 256 * j, 128, 1024);
        tc::mma_tf32(tbase, dah, dbh, idesc, (cur_kc > 0 || j > 0) ? 1u : 0u);
        tc::mma_tf32(tbase, dah, dbl, idesc, 1u);
        tc::mma_tf32(tbase, dal, dbh, idesc, 1u);
      }
      tc::commit(&mbar[stage]);
    }
    ++g;
    if (cur_kc == nkc - 1) {
      // epilogue of cur_tile: all of its MMAs are done once this stage's commit lands
      ok &= tc::mbar_wait(&mbar[stage], use & 1);
      tc::fence_after_sync();
      const int r = cur_tile * 128 + tid;
      float acc[kTcN];
#pragma unroll
      for (int i = 0; i < kTcN / 16; ++i) tc::tmem_ld16(tbase + ((uint32_t)(32 * warp) << 16) + 16 * i, acc + 16 * i);
      if (r < n) {
        const float as = a ? a[r] : 0.f, bs = (b ? b[r] : 1.f) * beta;
#pragma unroll
        for (int c = 0; c < kTcN; ++c) {
          if (c < t) {
            const float y = (a && Y) ? Y[(int64_t)r * ld + c] : 0.f;
            Z[(int64_t)r * ld + c] = as * y + bs * acc[c];
          } else if (c < ld) {
            Z[(int64_t)r * ld + c] = 0.f;
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();
    }
  }
  if (g > 0) ok &= tc::mbar_wait(&mbar[(g - 1) & 1], ((g - 1) >> 1) & 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 64);
  if (!ok && tid == 0) raise_error(st, VL_ERR_TIMEOUT, -1);
}

// ----------------------------------------------------------------------------- G = L^T (w o R)
// 256 threads, one chunk of rows per block, K chunks of 16 rows. M = four 128-rank
// tiles (ranks >= k are zero), N = 64 columns. Per stage: A head / remainder (4 x 8
// KB each), B head / remainder (4 KB each). Tensor memory: 256 columns (the four
// 128 x 64 accumulators side by side). part[chunk][q][c] receives the block's sums.
constexpr int kTnStage = 72 * 1024;
constexpr int kTnSmem = 2 * kTnStage + 64;

static __global__ void __launch_bounds__(256, 1)
    lrac_tn_tc_kernel(int n, int k, int t, int ld, int rows_per_chunk, const float* __restrict__ L,
                      const float* __restrict__ R, const float* __restrict__ w, double* __restrict__ part,
                      DevStatus* st) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 2 * kTnStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * kTnStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int chunk = blockIdx.x;
  const int r0 = chunk * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
  const int nks = r1 > r0 ? (r1 - r0 + 15) / 16 : 0;
  if (warp == 0) tc::tmem_alloc(tslot, 256);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  constexpr uint32_t idesc = tc::idesc_tf32(128, kTcN);
  bool ok = true;

  // A: 512 ranks x 16 rows = 8 quads per thread: quad i -> rank qb + (lane & 7),
  // row quad (lane >> 3) of the chunk, with qb = 8 (warp + 8 i).
  // B: 64 columns x 16 rows = one quad per thread: column tid & 63, row quad tid >> 6.
  const bool vec4 = (n & 3) == 0 && (rows_per_chunk & 15) == 0 && (reinterpret_cast<uintptr_t>(L) & 15) == 0;
  float4 aq[8];
  float4 bq;
  auto load = [&](int ks) {
    const int rb = r0 + ks * 16;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = 8 * (warp + 8 * i) + (lane & 7), r = rb + 4 * (lane >> 3);
      const float* col = L + (int64_t)q * n;
      float4 v;
      if (vec4 && q < k && r + 3 < r1) {   // column start and r are multiples of 4: 16-byte aligned
        v = __ldcs(reinterpret_cast<const float4*>(col + r));
      } else {
        v.x = (q < k && r + 0 < r1) ? __ldcs(col + r + 0) : 0.f;
        v.y = (q < k && r + 1 < r1) ? __ldcs(col + r + 1) : 0.f;
        v.z = (q < k && r + 2 < r1) ? __ldcs(col + r + 2) : 0.f;
        v.w = (q < k && r + 3 < r1) ? __ldcs(col + r + 3) : 0.f;
      }
      aq[i] = v;
    }
    const int c = tid & 63, r = rb + 4 * (tid >> 6);
    const bool cv = c < t;
    bq.x = (cv && r + 0 < r1) ? R[(int64_t)(r + 0) * ld + c] * w[r + 0] : 0.f;
    bq.y = (cv && r + 1 < r1) ? R[(int64_t)(r + 1) * ld + c] * w[r + 1] : 0.f;
    bq.z = (cv && r + 2 < r1) ? R[(int64_t)(r + 2) * ld + c] * w[r + 2] : 0.f;
    bq.w = (cv && r + 3 < r1) ? R[(int64_t)(r + 3) * ld + c] * w[r + 3] : 0.f;
  };
  auto split4 = [](const float4& v, float4& h, float4& l) {
    tc::split_tf32(v.x, h.x, l.x);
    tc::split_tf32(v.y, h.y, l.y);
    tc::split_tf32(v.z, h.z, l.z);
    tc::split_tf32(v.w, h.w, l.w);
  };
  if (nks > 0) load(0);
  for (int ks = 0; ks < nks; ++ks) {
    const int stage = ks & 1;
    const uint32_t use = (uint32_t)ks >> 1;
    unsigned char* S = sm + stage * kTnStage;
    float* Ahi = reinterpret_cast<float*>(S);               // 4 tiles x 8 KB
    float* Alo = reinterpret_cast<float*>(S + 32768);
    float* Bhi = reinterpret_cast<float*>(S + 65536);       // 4 KB
    float* Blo = reinterpret_cast<float*>(S + 65536 + 4096);
    if (use >= 1) ok &= tc::mbar_wait(&mbar[stage], (use - 1) & 1);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int q = 8 * (warp + 8 * i) + (lane & 7), kg = lane >> 3;
      const int mt = q >> 7, qq = q & 127;
      // tile mt: core matrix (qq / 8, kg) of a 16-row chunk (4 K groups), row qq % 8
      const int off = mt * 2048 + ((qq >> 3) * 4 + kg) * 32 + (qq & 7) * 4;
      float4 h, l;
      split4(aq[i], h, l);
      *reinterpret_cast<float4*>(Ahi + off) = h;
      *reinterpret_cast<float4*>(Alo + off) = l;
    }
    {
      const int c = tid & 63, kg = tid >> 6;
      const int off = ((c >> 3) * 4 + kg) * 32 + (c & 7) * 4;
      float4 h, l;
      split4(bq, h, l);
      *reinterpret_cast<float4*>(Bhi + off) = h;
      *reinterpret_cast<float4*>(Blo + off) = l;
    }
    if (ks + 1 < nks) load(ks + 1);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t a_hi = tc::smem_u32(Ahi), a_lo = tc::smem_u32(Alo), b_hi = tc::smem_u32(Bhi),
                     b_lo = tc::smem_u32(Blo);
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const uint64_t dah = tc::smem_desc(a_hi + 8192 * mt + 256 * j, 128, 512);
          const uint64_t dal = tc::smem_desc(a_lo + 8192 * mt + 256 * j, 128, 512);
          const uint64_t dbh = tc::smem_desc(b_hi + 256 * j, 128, 512);
          const uint64_t dbl = tc::smem_desc(b_lo + 256 * j, 128, 512);
          const uint32_t d = tbase + (uint32_t)(mt * kTcN);
          tc::mma_tf32(d, dah, dbh, idesc, (ks > 0 || j > 0) ? 1u : 0u);
          tc::mma_tf32(d, dah, dbl, idesc, 1u);
          tc::mma_tf32(d, dal, dbh, idesc, 1u);
        }
      }
      tc::commit(&mbar[stage]);
    }
  }
  if (nks > 0) ok &= tc::mbar_wait(&mbar[(nks - 1) & 1], ((uint32_t)(nks - 1) >> 1) & 1);
  tc::fence_after_sync();
  // epilogue: warp w reads lanes 32 (w % 4) of tiles 2 (w / 4) and 2 (w / 4) + 1
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int mt = 2 * (warp >> 2) + u;
    const int q = mt * 128 + 32 * (warp & 3) + lane;
    float acc[kTcN];
    if (nks > 0) {
#pragma unroll
      for (int i = 0; i < kTcN / 16; ++i)
        tc::tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mt * kTcN + 16 * i), acc + 16 * i);
    } else {
#pragma unroll
      for (int i = 0; i < kTcN; ++i) acc[i] = 0.f;
    }
    if (q < k)
      for (int c = 0; c < t; ++c) part[((int64_t)chunk * k + q) * t + c] = (double)acc[c];
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
  if (!ok && tid == 0) raise_error(st, VL_ERR_TIMEOUT, -1);
}

}  // namespace vl
