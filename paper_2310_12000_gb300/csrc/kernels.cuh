// Kernels of the Krylov hot path (Section 3): products with B, B^T and the
// diagonals, sync-free level-ordered triangular solves with B and B^T, the
// per-column PCG scalar recurrences with Lanczos T extraction (Appendix, PCG
// algorithm), the SLQ quadrature e1^T log(T) e1, likelihood terms and probes.
//
// Right-hand-side blocks are n x ld row-major (ld >= t, the columns of one point
// contiguous) in storage order. One warp owns one row; for t = 1 its lanes split
// the row's m neighbours, otherwise they split the columns.
#pragma once

#include <cooperative_groups.h>

#include "vl_device.cuh"

namespace vl {


// ----------------------------------------------------------------------------- row teams
// A team of LPV lanes (LPV in {8, 16, 32}) owns one row; a warp runs 32 / LPV
// teams on different rows at once. Teams synchronise only within their own lane
// segment (masked shuffles), so teams of one warp never wait on each other.
// Row blocks (ld columns, ld a multiple of 8) are read as float4 / double2 words,
// NV words per lane; dependency rows are broadcast inside the team UNR at a time,
// so each lane has UNR row loads outstanding before it accumulates. Padding
// columns are computed too and stay zero. For t = 1 the team's lanes split the
// row's dependencies instead and reduce at the end.
template <typename T>
struct VecT;
template <>
struct VecT<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct VecT<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <int LPV>
__device__ __forceinline__ unsigned team_mask() {
  const int lane = threadIdx.x & 31;
  return LPV == 32 ? 0xffffffffu : (((1u << LPV) - 1u) << (lane / LPV * LPV));
}

__device__ __forceinline__ float4 ldg_vec(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ double2 ldg_vec(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

// L2 (not L1) vector loads for values written earlier in the same launch.
__device__ __forceinline__ float4 ldcg_vec(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ double2 ldcg_vec(const double* p) { return __ldcg(reinterpret_cast<const double2*>(p)); }

__device__ __forceinline__ void fma_vec(float* a, float s, float4 v) {
  a[0] += s * v.x;
  a[1] += s * v.y;
  a[2] += s * v.z;
  a[3] += s * v.w;
}
__device__ __forceinline__ void fma_vec(double* a, double s, double2 v) {
  a[0] += s * v.x;
  a[1] += s * v.y;
}
__device__ __forceinline__ void store_vec(float* p, const float* a) {
  *reinterpret_cast<float4*>(p) = make_float4(a[0], a[1], a[2], a[3]);
}
__device__ __forceinline__ void store_vec(double* p, const double* a) {
  *reinterpret_cast<double2*>(p) = make_double2(a[0], a[1]);
}
// acc (this lane's NV words of the row) += sum_e coef_e * X[idx_e, :] over e in [beg, end),
// coef_e = sgn * val[e] * (dscale ? dscale[idx_e] : 1); negative indices are skipped.
// PRODUCED: X rows were written earlier in the same launch (read through L2).
template <typename T, int LPV, int NV, int UNR, bool PRODUCED>
__device__ __forceinline__ void team_gather(T* acc, const int32_t* __restrict__ idx, const T* __restrict__ val,
                                            const T* __restrict__ dscale, T sgn, int beg, int end, const T* X,
                                            int ld, DevStatus* st, int row) {
  constexpr int VEC = VecT<T>::n;
  using V = typename VecT<T>::type;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  for (int e0 = beg; e0 < end; e0 += LPV) {
    const int cnt = min(LPV, end - e0);
    int jl = -1;
    T al = T(0);
    if (sl < cnt) {
      jl = idx[e0 + sl];
      if (jl >= 0) al = sgn * val[e0 + sl] * (dscale ? dscale[jl] : T(1));
    }
    for (int q0 = 0; q0 < cnt; q0 += UNR) {
      int j[UNR];
      T a[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int q = q0 + u;
        const int src = q < LPV ? q : LPV - 1;
        const int jj = __shfl_sync(mask, jl, src, LPV);
        const T aa = __shfl_sync(mask, al, src, LPV);
        j[u] = (q < cnt) ? jj : -1;
        a[u] = aa;
      }
      V xv[UNR][NV];
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int col = (sl + LPV * v) * VEC;
          if (j[u] >= 0 && col < ld) {
            const T* p = X + (int64_t)j[u] * ld + col;
            xv[u][v] = PRODUCED ? ldcg_vec(p) : ldg_vec(p);
          } else {
            xv[u][v] = V{};
          }
        }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int v = 0; v < NV; ++v) fma_vec(acc + v * VEC, j[u] >= 0 ? a[u] : T(0), xv[u][v]);
    }
  }
}

// acc = s1 * A1[row] + s2 * A2[row] (either array may be null) for the lane's words.
template <typename T, int LPV, int NV>
__device__ __forceinline__ void team_init(T* acc, int64_t row, int ld, T s1, const T* __restrict__ A1, T s2,
                                          const T* __restrict__ A2) {
  constexpr int VEC = VecT<T>::n;
  const int sl = (threadIdx.x & 31) % LPV;
#pragma unroll
  for (int i = 0; i < NV * VEC; ++i) acc[i] = T(0);
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = (sl + LPV * v) * VEC;
    if (col < ld) {
      if (A1) fma_vec(acc + v * VEC, s1, ldg_vec(A1 + row * ld + col));
      if (A2) fma_vec(acc + v * VEC, s2, ldg_vec(A2 + row * ld + col));
    }
  }
}

template <typename T, int LPV, int NV>
__device__ __forceinline__ void team_store(T* Y, int64_t row, int ld, T scale, T* acc) {
  constexpr int VEC = VecT<T>::n;
  const int sl = (threadIdx.x & 31) % LPV;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = (sl + LPV * v) * VEC;
    if (col < ld) {
#pragma unroll
      for (int i = 0; i < VEC; ++i) acc[v * VEC + i] *= scale;
      store_vec(Y + row * ld + col, acc + v * VEC);
    }
  }
}

// Scalar rows (t = 1): the team's lanes split the dependencies; returns the team sum
// of coef_e * X[idx_e] on every lane of the team.
template <typename T, int LPV, bool PRODUCED>
__device__ __forceinline__ T team_dot1(const int32_t* __restrict__ idx, const T* __restrict__ val,
                                       const T* __restrict__ dscale, int beg, int end, const T* X, DevStatus* st,
                                       int row) {
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T acc = T(0);
  constexpr int K = 4;   // loads in flight per lane
  for (int e0 = beg + sl; e0 < end; e0 += LPV * K) {
    int j[K];
    T xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int e = e0 + u * LPV;
      j[u] = e < end ? idx[e] : -1;
      xv[u] = j[u] >= 0 ? (PRODUCED ? __ldcg(&X[j[u]]) : __ldg(&X[j[u]])) : T(0);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) {
      if (j[u] < 0) continue;
      acc += val[e0 + u * LPV] * (dscale ? dscale[j[u]] : T(1)) * xv[u];
    }
  }
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  return acc;
}

// ----------------------------------------------------------------------------- B X
// Y_s = ys_s (X_s - sum_c A[s,c] X_{nbr[s,c]})   (ys == nullptr: 1)
// Rows of a product kernel's team: CH = 0 interleaves the teams of the whole grid over the rows;
// CH = 1 gives each block one contiguous range of rows, so that the neighbour rows it gathers
// (near in Morton order) are reused from the SM's L1 across the range. Either way each row is
// one team's, so the results are the same.
template <int CH>
struct TeamRows {
  int s, end, step;
  template <int LPV>
  __device__ __forceinline__ static TeamRows make(int n) {
    constexpr int RPW = 32 / LPV;
    TeamRows r;
    if (CH == 0) {
      r.s = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + (threadIdx.x & 31) / LPV;
      r.end = n;
      r.step = ((gridDim.x * blockDim.x) >> 5) * RPW;
    } else {
      const int per = (n + gridDim.x - 1) / gridDim.x;
      const int b0 = blockIdx.x * per;
      r.s = b0 + (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
      r.end = min(n, b0 + per);
      r.step = (blockDim.x >> 5) * RPW;
    }
    return r;
  }
};

template <typename T, int LPV, int NV, int UNR, int CH = 0>
__global__ void __launch_bounds__(256) spmv_B_kernel(int n, int m, const int32_t* __restrict__ nbr,
                                                     const T* __restrict__ A, const T* __restrict__ X, int ld,
                                                     const T* __restrict__ ys, T* __restrict__ Y) {
  const TeamRows<CH> rows = TeamRows<CH>::template make<LPV>(n);
  T acc[NV * VecT<T>::n];
  for (int s = rows.s; s < rows.end; s += rows.step) {
    team_init<T, LPV, NV>(acc, s, ld, T(1), X, T(0), nullptr);
    team_gather<T, LPV, NV, UNR, false>(acc, nbr, A, nullptr, T(-1), s * m, s * m + m, X, ld, nullptr, s);
    team_store<T, LPV, NV>(Y, s, ld, ys ? ys[s] : T(1), acc);
  }
}

// Staged products (plan: build_halo_plan). Block b copies the rows of its list (its own rows and
// their dependencies) into shared memory with coalesced 16-byte loads, then each team takes a row
// of the block and accumulates exactly as team_gather does (entries in order, coefficient
// sgn * val * dscale), reading the rows from shared memory: the same numbers as the unstaged
// kernels.
struct HaloArgs {
  const int32_t* brow;
  const int32_t* uoff;
  const int32_t* ulist;
  const uint16_t* lidx;
  const uint16_t* lself;
};

// The block's rows into shared memory by asynchronous 16-byte copies (cp.async: every copy of
// the thread in flight at once, no registers held), then a wait and a block barrier.
template <typename T>
__device__ __forceinline__ void halo_stage(const HaloArgs& H, int b, const T* __restrict__ X, int ld, T* xs) {
  constexpr int VEC = VecT<T>::n;
  const int nw = ld / VEC;
  const int u0 = H.uoff[b], U = H.uoff[b + 1] - u0;
  const unsigned base = (unsigned)__cvta_generic_to_shared(xs);
  for (int w = threadIdx.x; w < U * nw; w += blockDim.x) {
    const int k = w / nw, v = w - k * nw;
    const T* src = X + (int64_t)H.ulist[u0 + k] * ld + v * VEC;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16u * (unsigned)w), "l"(src) : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
}

// acc (the lane's words) += sum_e sgn * val[e] * dscale[j_e] * xs[lidx[e], :] over [beg, end)
template <typename T, int LPV, int NV>
__device__ __forceinline__ void halo_gather(T* acc, const HaloArgs& H, const int32_t* __restrict__ idx,
                                            const T* __restrict__ val, const T* __restrict__ dscale, T sgn,
                                            int64_t beg, int64_t end, const T* xs, int ld) {
  constexpr int VEC = VecT<T>::n;
  using V = typename VecT<T>::type;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  for (int64_t e0 = beg; e0 < end; e0 += LPV) {
    const int cnt = (int)min((int64_t)LPV, end - e0);
    int jl = -1, pl = 0;
    T al = T(0);
    if (sl < cnt) {
      jl = idx[e0 + sl];
      if (jl >= 0) {
        al = sgn * val[e0 + sl] * (dscale ? dscale[jl] : T(1));
        pl = H.lidx[e0 + sl];
      }
    }
    for (int q = 0; q < cnt; ++q) {
      const int j = __shfl_sync(mask, jl, q, LPV);
      const int pq = __shfl_sync(mask, pl, q, LPV);
      const T a = __shfl_sync(mask, al, q, LPV);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int col = (sl + LPV * v) * VEC;
        const V xv = (j >= 0 && col < ld) ? *reinterpret_cast<const V*>(xs + (int64_t)pq * ld + col) : V{};
        fma_vec(acc + v * VEC, j >= 0 ? a : T(0), xv);
      }
    }
  }
}

template <typename T, int LPV, int NV>
__global__ void __launch_bounds__(256) spmv_B_staged_kernel(HaloArgs H, int m, const int32_t* __restrict__ nbr,
                                                            const T* __restrict__ A, const T* __restrict__ X, int ld,
                                                            const T* __restrict__ ys, T* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char vl_smem[];
  T* xs = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV, VEC = VecT<T>::n;
  const int b = blockIdx.x;
  halo_stage<T>(H, b, X, ld, xs);
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  T acc[NV * VEC];
  for (int s = H.brow[b] + tib; s < H.brow[b + 1]; s += tpb) {
    const int ps = H.lself[s];
#pragma unroll
    for (int i = 0; i < NV * VEC; ++i) acc[i] = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int col = (sl + LPV * v) * VEC;
      if (col < ld) fma_vec(acc + v * VEC, T(1), *reinterpret_cast<const typename VecT<T>::type*>(xs + (int64_t)ps * ld + col));
    }
    halo_gather<T, LPV, NV>(acc, H, nbr, A, nullptr, T(-1), (int64_t)s * m, (int64_t)s * m + m, xs, ld);
    team_store<T, LPV, NV>(Y, s, ld, ys ? ys[s] : T(1), acc);
  }
}

template <typename T, int LPV, int NV>
__global__ void __launch_bounds__(256) spmv_Bt_staged_kernel(HaloArgs H, const int32_t* __restrict__ rowptrT,
                                                             const int32_t* __restrict__ colT,
                                                             const T* __restrict__ valT, const T* __restrict__ Y,
                                                             const T* __restrict__ ys, const T* __restrict__ X,
                                                             const T* __restrict__ wx, int ld, T* __restrict__ Z) {
  extern __shared__ __align__(16) unsigned char vl_smem[];
  T* xs = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV, VEC = VecT<T>::n;
  const int b = blockIdx.x;
  halo_stage<T>(H, b, Y, ld, xs);
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  T acc[NV * VEC];
  for (int s = H.brow[b] + tib; s < H.brow[b + 1]; s += tpb) {
    const int ps = H.lself[s];
    const T s1 = ys ? ys[s] : T(1), s2 = X ? wx[s] : T(0);
#pragma unroll
    for (int i = 0; i < NV * VEC; ++i) acc[i] = T(0);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int col = (sl + LPV * v) * VEC;
      if (col < ld) {
        fma_vec(acc + v * VEC, s1, *reinterpret_cast<const typename VecT<T>::type*>(xs + (int64_t)ps * ld + col));
        if (X) fma_vec(acc + v * VEC, s2, ldg_vec(X + (int64_t)s * ld + col));
      }
    }
    halo_gather<T, LPV, NV>(acc, H, colT, valT, ys, T(-1), rowptrT[s], rowptrT[s + 1], xs, ld);
    team_store<T, LPV, NV>(Z, s, ld, T(1), acc);
  }
}

template <typename T, int LPV>
__global__ void __launch_bounds__(256) spmv_B_t1_kernel(int n, int m, const int32_t* __restrict__ nbr,
                                                        const T* __restrict__ A, const T* __restrict__ X,
                                                        const T* __restrict__ ys, T* __restrict__ Y) {
  constexpr int RPW = 32 / LPV;
  const int G = ((gridDim.x * blockDim.x) >> 5) * RPW;
  const int g = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + (threadIdx.x & 31) / LPV;
  for (int s = g; s < n; s += G) {
    const T acc = team_dot1<T, LPV, false>(nbr, A, nullptr, s * m, s * m + m, X, nullptr, s);
    if ((threadIdx.x & 31) % LPV == 0) Y[s] = (ys ? ys[s] : T(1)) * (X[s] - acc);
  }
}

// ----------------------------------------------------------------------------- W X + B^T Y
// Z_s = wx_s X_s + ys_s Y_s - sum_{e in row s of B^T} valT[e] ys_{i} Y_{i},  i = colT[e]
// (X == nullptr: no diagonal term; ys == nullptr: 1)
template <typename T, int LPV, int NV, int UNR, int CH = 0>
__global__ void __launch_bounds__(256) spmv_Bt_kernel(int n, const int32_t* __restrict__ rowptrT,
                                                      const int32_t* __restrict__ colT, const T* __restrict__ valT,
                                                      const T* __restrict__ Y, const T* __restrict__ ys,
                                                      const T* __restrict__ X, const T* __restrict__ wx, int ld,
                                                      T* __restrict__ Z) {
  const TeamRows<CH> rows = TeamRows<CH>::template make<LPV>(n);
  T acc[NV * VecT<T>::n];
  for (int s = rows.s; s < rows.end; s += rows.step) {
    team_init<T, LPV, NV>(acc, s, ld, ys ? ys[s] : T(1), Y, X ? wx[s] : T(0), X);
    team_gather<T, LPV, NV, UNR, false>(acc, colT, valT, ys, T(-1), rowptrT[s], rowptrT[s + 1], Y, ld, nullptr, s);
    team_store<T, LPV, NV>(Z, s, ld, T(1), acc);
  }
}

template <typename T, int LPV>
__global__ void __launch_bounds__(256) spmv_Bt_t1_kernel(int n, const int32_t* __restrict__ rowptrT,
                                                         const int32_t* __restrict__ colT, const T* __restrict__ valT,
                                                         const T* __restrict__ Y, const T* __restrict__ ys,
                                                         const T* __restrict__ X, const T* __restrict__ wx,
                                                         T* __restrict__ Z) {
  constexpr int RPW = 32 / LPV;
  const int G = ((gridDim.x * blockDim.x) >> 5) * RPW;
  const int g = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW + (threadIdx.x & 31) / LPV;
  for (int s = g; s < n; s += G) {
    const T acc = team_dot1<T, LPV, false>(colT, valT, ys, rowptrT[s], rowptrT[s + 1], Y, nullptr, s);
    if ((threadIdx.x & 31) % LPV == 0) Z[s] = (X ? wx[s] * X[s] : T(0)) + (ys ? ys[s] : T(1)) * Y[s] - acc;
  }
}

// ----------------------------------------------------------------------------- solves
// Level-synchronous triangular solve in one cooperative launch. Rows are taken
// in the level order of the task list (lptr[l] .. lptr[l+1] is level l); a row
// only reads rows of earlier levels, so a level's rows are independent.
//   head  levels [0, l_head):     block 0 alone, one __syncthreads per level
//   body  levels [l_head, l_tail): every block, one grid barrier per level
//   tail  levels [l_tail, nlev):   block 0 alone again
// The head and tail are the narrow ends of the level profile (random orderings
// give a long thin head), where a block barrier is far cheaper than a grid one.
// Values of x produced in this launch are read through L2 (ld.global.cg).
//   FWD (B^{-1}):   x_s = q_s r_s + sum_{c} A[s,c] x_{nbr[s,c]}
//   BWD (B^{-T}):   x_s = q_s r_s + sum_{e in row s of B^T} valT[e] x_{colT[e]}
// A piece of a heavy row's dependency list: the grid walk splits every heavy row of a level
// into chunks of at most CH dependencies that separate teams gather at the same time; each
// writes its partial row to a level-local slot and the team that completes the row's last
// chunk (an arrival counter per row) adds q_s rhs_s and the partials in slot order, so the
// result does not depend on which team finishes last.
struct HeavyChunk {
  int32_t p;       // task index of the row (its storage row is task[p])
  int32_t beg, end;   // dependency range in idx / val
  int32_t slot;    // level-local slot of this chunk's partial row
  int32_t base;    // slot of the row's first chunk; the row has nch consecutive slots
  int32_t nch;
  int32_t hrow;    // level-local index of the row (its arrival counter)
  int32_t pad;
};

struct LevelPlan {
  const int32_t* task;
  const int32_t* lptr;
  const int32_t* hptr;         // heavy rows of level l are task[lptr[l] .. hptr[l])
  int l_head, l_tail, nlev;
  unsigned* bar;               // {count, generation}, count == 0 at launch
  DevStatus* st;
  long long* trace;            // optional: block 0's clock at each level boundary (nlev + 1)
  // grid body only (null: heavy rows by whole blocks): the heavy rows of level l as the
  // chunks chunk[cptr[l] .. cptr[l+1]), partial rows in `part`, per-row arrival counters
  // in `cnt` (zero at launch; each row's finishing team sets its counter back to zero).
  // A level without chunks keeps a whole block per heavy row (one round of loads, no
  // partials): chunks only pay off when a level has more heavy rows than blocks.
  const HeavyChunk* chunk;
  const int32_t* cptr;
  void* part;
  int* cnt;
  int head_done;               // levels [0, l_head) were solved by sptrsv_t1_head_kernel before
};

// Grid barrier with a bounded wait on a monotonic arrival counter (zero at launch):
// barrier number e of the launch is passed once the counter reaches e * gridDim.x.
// Each block adds 1 with release semantics (after a block barrier, so the add
// publishes the whole block's writes) and polls with acquire loads; nothing has to
// be written after the last arrival, so waiters leave as soon as it lands in L2.
// `epoch` counts the barriers this block has passed (kept by thread 0). A timeout
// records VL_ERR_TIMEOUT; after an abort every barrier returns at once so the
// launch still ends.
// Measured at n = 1e6: 10 % faster scalar (t = 1) solves than the generation-word
// barrier below, but slower block (t = 50) solves, which therefore keep the latter.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void grid_barrier_counter(unsigned* bar, DevStatus* st, unsigned& epoch) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    if (!ld_volatile(&st->abort)) {
      const unsigned target = epoch * gridDim.x;
      red_release_add(&bar[0], 1u);
      int spins = 0;
      // a few tight polls, then back off so the polls do not crowd the arrivals
      // that land on the same word
      while (ld_acquire(&bar[0]) < target && ++spins < 4096) {
        if (spins > 4) __nanosleep(40);
      }
      if (spins >= 4096) bounded_wait([&] { return ld_acquire(&bar[0]) >= target; }, st, -1);
    }
  }
  __syncthreads();
}

// Grid barrier with a bounded wait: the last block to arrive resets the arrival
// counter and bumps the generation word the others poll (bar[1]; zero at launch).
__device__ __forceinline__ void grid_barrier_generation(unsigned* bar, DevStatus* st) {
  __syncthreads();
  if (threadIdx.x == 0 && !ld_volatile(&st->abort)) {
    const unsigned gen = ld_acquire(&bar[1]);
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      st_release(&bar[1], gen + 1);
    } else {
      int spins = 0;
      while (ld_acquire(&bar[1]) == gen && ++spins < 4096) {
      }
      if (spins >= 4096) bounded_wait([&] { return ld_acquire(&bar[1]) != gen; }, st, -1);
    }
  }
  __syncthreads();
}

// Grid barrier in two stages for a grid launched in thread-block clusters: the hardware
// cluster barrier (release / acquire at cluster scope), then one arrival per cluster on the
// monotonic counter (release at gpu scope, after the cluster barrier, so it publishes the whole
// cluster's writes), polled by the cluster's first thread; the cluster barrier again releases
// the cluster. A grid of C clusters makes C arrivals on the counter per level instead of one
// per block. Bounded like grid_barrier_counter; after an abort the counter is skipped.
__device__ __forceinline__ void grid_barrier_cluster(unsigned* bar, DevStatus* st, unsigned& epoch) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  if (cl.block_rank() == 0 && threadIdx.x == 0) {
    ++epoch;
    if (!ld_volatile(&st->abort)) {
      const unsigned target = epoch * (gridDim.x / cl.num_blocks());
      red_release_add(&bar[0], 1u);
      int spins = 0;
      while (ld_acquire(&bar[0]) < target && ++spins < 4096) {
        if (spins > 4) __nanosleep(40);
      }
      if (spins >= 4096) bounded_wait([&] { return ld_acquire(&bar[0]) >= target; }, st, -1);
    }
  }
  cl.sync();
}

// BAR: 0 generation word, 1 monotonic counter, 2 counter per thread-block cluster
template <int BAR>
__device__ __forceinline__ void grid_barrier(unsigned* bar, DevStatus* st, unsigned& epoch) {
  if constexpr (BAR == 2)
    grid_barrier_cluster(bar, st, epoch);
  else if constexpr (BAR == 1)
    grid_barrier_counter(bar, st, epoch);
  else
    grid_barrier_generation(bar, st);
}

// Row state loaded ahead of time: everything a team needs before it reads x
// (task, dependency range, its first chunk of dependency indices and weights,
// the scaled right-hand side). Prefetching it for the next level before a
// barrier leaves only the x gathers on the critical path.
template <typename T, int LPV, int NV>
struct RowPre {
  int s, beg, end, jl;
  T al;
  T acc[NV * VecT<T>::n];
};

// xpf != nullptr: the lane also asks L2 for the x row of the dependency it holds (every 128-byte
// line of it). Issued before the level barrier, this turns the DRAM misses of the gathers after
// it into L2 hits for the dependencies solved at earlier levels; a line a later level rewrites is
// simply updated in L2, so a prefetch never makes a load see stale data.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename T, bool FWD, int LPV, int NV>
__device__ __forceinline__ void row_pre_s(RowPre<T, LPV, NV>& r, int s, int m, const int32_t* __restrict__ idx,
                                          const T* __restrict__ val, const int32_t* __restrict__ rowptr,
                                          const T* __restrict__ rhs, const T* __restrict__ q, int ld,
                                          const T* xpf = nullptr) {
  const int sl = (threadIdx.x & 31) % LPV;
  r.s = s;
  r.beg = FWD ? r.s * m : rowptr[r.s];
  r.end = FWD ? r.s * m + m : rowptr[r.s + 1];
  const int e = r.beg + sl;
  r.jl = e < r.end ? idx[e] : -1;
  r.al = r.jl >= 0 ? val[e] : T(0);
  if (xpf && r.jl >= 0) {
    const char* row = reinterpret_cast<const char*>(xpf + (int64_t)r.jl * ld);
    const int bytes = ld * (int)sizeof(T);
    for (int o = 0; o < bytes; o += 128) prefetch_l2(row + o);
    prefetch_l2(row + bytes - 1);
  }
  team_init<T, LPV, NV>(r.acc, r.s, ld, q ? q[r.s] : T(1), rhs, T(0), nullptr);
}

template <typename T, bool FWD, int LPV, int NV>
__device__ __forceinline__ void row_pre(RowPre<T, LPV, NV>& r, int p, int m, const LevelPlan& L,
                                        const int32_t* __restrict__ idx, const T* __restrict__ val,
                                        const int32_t* __restrict__ rowptr, const T* __restrict__ rhs,
                                        const T* __restrict__ q, int ld, const T* xpf = nullptr) {
  row_pre_s<T, FWD, LPV, NV>(r, L.task[p], m, idx, val, rowptr, rhs, q, ld, xpf);
}

// Finishes a prefetched row: gathers its dependencies (first chunk already in
// registers) and stores x_s.
// acc += sum over one chunk of <= LPV dependencies (index jl / weight al held by
// lane sl of the team) of al * x[jl, :], UNR rows' loads in flight per lane.
template <typename T, int LPV, int NV, int UNR>
__device__ __forceinline__ void chunk_gather(T* acc, int jl, T al, int cnt, const T* x, int ld) {
  constexpr int VEC = VecT<T>::n;
  using V = typename VecT<T>::type;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  for (int q0 = 0; q0 < cnt; q0 += UNR) {
    int j[UNR];
    T a[UNR];
#pragma unroll
    for (int u = 0; u < UNR; ++u) {
      const int qq = q0 + u;
      const int src = qq < LPV ? qq : LPV - 1;
      const int jj = __shfl_sync(mask, jl, src, LPV);
      const T aa = __shfl_sync(mask, al, src, LPV);
      j[u] = (qq < cnt) ? jj : -1;
      a[u] = aa;
    }
    V xv[UNR][NV];
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int col = (sl + LPV * v) * VEC;
        xv[u][v] = (j[u] >= 0 && col < ld) ? ldcg_vec(x + (int64_t)j[u] * ld + col) : V{};
      }
#pragma unroll
    for (int u = 0; u < UNR; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) fma_vec(acc + v * VEC, j[u] >= 0 ? a[u] : T(0), xv[u][v]);
  }
}

template <typename T, int LPV, int NV, int UNR>
__device__ __forceinline__ void row_run(RowPre<T, LPV, NV>& r, const int32_t* __restrict__ idx,
                                        const T* __restrict__ val, T* x, int ld) {
  const int sl = (threadIdx.x & 31) % LPV;
  for (int e0 = r.beg; e0 < r.end; e0 += LPV) {
    const int cnt = min(LPV, r.end - e0);
    int jl = r.jl;
    T al = r.al;
    if (e0 != r.beg) {
      jl = sl < cnt ? idx[e0 + sl] : -1;
      al = jl >= 0 ? val[e0 + sl] : T(0);
    }
    chunk_gather<T, LPV, NV, UNR>(r.acc, jl, al, cnt, x, ld);
  }
  team_store<T, LPV, NV>(x, r.s, ld, T(1), r.acc);
}

// A heavy row (many dependencies) by the whole block: team k takes dependency
// chunks k, k + teams, ...; the teams' partial rows meet in shared memory and
// are summed in team order (deterministic). Every thread of the block calls it.
template <typename T, bool FWD, int LPV, int NV, int UNR>
__device__ void heavy_row(int p, int m, const LevelPlan& L, const int32_t* __restrict__ idx, const T* __restrict__ val,
                          const int32_t* __restrict__ rowptr, const T* __restrict__ rhs, const T* __restrict__ q, T* x,
                          int ld, T* part) {
  constexpr int VEC = VecT<T>::n;
  constexpr int RPW = 32 / LPV;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  const int s = L.task[p];
  const int beg = FWD ? s * m : rowptr[s];
  const int end = FWD ? s * m + m : rowptr[s + 1];
  T acc[NV * VEC];
#pragma unroll
  for (int i = 0; i < NV * VEC; ++i) acc[i] = T(0);
  for (int e0 = beg + tib * LPV; e0 < end; e0 += tpb * LPV) {
    const int cnt = min(LPV, end - e0);
    const int jl = sl < cnt ? idx[e0 + sl] : -1;
    const T al = jl >= 0 ? val[e0 + sl] : T(0);
    chunk_gather<T, LPV, NV, UNR>(acc, jl, al, cnt, x, ld);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = (sl + LPV * v) * VEC;
    if (col < ld)
#pragma unroll
      for (int i = 0; i < VEC; ++i) part[tib * ld + col + i] = acc[v * VEC + i];
  }
  __syncthreads();
  const T qs = q ? q[s] : T(1);
  for (int col = threadIdx.x; col < ld; col += blockDim.x) {
    T sum = qs * rhs[(int64_t)s * ld + col];
    for (int k = 0; k < tpb; ++k) sum += part[k * ld + col];
    x[(int64_t)s * ld + col] = sum;
  }
  __syncthreads();
}

// Scalar rows (t = 1): the team's lanes split the dependencies, K loads each in flight.
template <typename T, int LPV>
struct RowPre1 {
  static constexpr int K = 4;
  int s, beg, end;
  int j[K];
  T a[K];
  T b;   // q_s r_s
};

template <typename T, bool FWD, int LPV>
__device__ __forceinline__ void row_pre1(RowPre1<T, LPV>& r, int p, int m, const LevelPlan& L,
                                         const int32_t* __restrict__ idx, const T* __restrict__ val,
                                         const int32_t* __restrict__ rowptr, const T* __restrict__ rhs,
                                         const T* __restrict__ q) {
  const int sl = (threadIdx.x & 31) % LPV;
  r.s = L.task[p];
  r.beg = FWD ? r.s * m : rowptr[r.s];
  r.end = FWD ? r.s * m + m : rowptr[r.s + 1];
#pragma unroll
  for (int u = 0; u < RowPre1<T, LPV>::K; ++u) {
    const int e = r.beg + sl + u * LPV;
    r.j[u] = e < r.end ? idx[e] : -1;
    r.a[u] = r.j[u] >= 0 ? val[e] : T(0);
  }
  r.b = (q ? q[r.s] : T(1)) * rhs[r.s];
}

template <typename T, int LPV>
__device__ __forceinline__ void row_run1(RowPre1<T, LPV>& r, const int32_t* __restrict__ idx,
                                         const T* __restrict__ val, T* x) {
  constexpr int K = RowPre1<T, LPV>::K;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T acc = T(0);
  for (int e0 = r.beg + sl; e0 < r.end; e0 += LPV * K) {
    int j[K];
    T a[K], xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int e = e0 + u * LPV;
      if (e0 == r.beg + sl) {
        j[u] = r.j[u];
        a[u] = r.a[u];
      } else {
        j[u] = e < r.end ? idx[e] : -1;
        a[u] = j[u] >= 0 ? val[e] : T(0);
      }
      xv[u] = j[u] >= 0 ? __ldcg(&x[j[u]]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) acc += a[u] * xv[u];
  }
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  if (sl == 0) x[r.s] = r.b + acc;
}

// A heavy scalar row by the whole block: each team takes K dependency chunks of
// LPV at a stride, reduces in registers, and thread 0 sums the team partials in
// order (deterministic). Every thread of the block calls it.
template <typename T, bool FWD, int LPV>
__device__ void heavy_row1(int p, int m, const LevelPlan& L, const int32_t* __restrict__ idx,
                           const T* __restrict__ val, const int32_t* __restrict__ rowptr, const T* __restrict__ rhs,
                           const T* __restrict__ q, T* x, T* part) {
  constexpr int RPW = 32 / LPV, K = 4;
  const unsigned mask = team_mask<LPV>();
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  const int s = L.task[p];
  const int beg = FWD ? s * m : rowptr[s];
  const int end = FWD ? s * m + m : rowptr[s + 1];
  T acc = T(0);
  for (int e0 = beg + tib * LPV * K + sl; e0 < end; e0 += tpb * LPV * K) {
    int j[K];
    T a[K], xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int e = e0 + u * LPV;
      j[u] = e < end ? idx[e] : -1;
      a[u] = j[u] >= 0 ? val[e] : T(0);
      xv[u] = j[u] >= 0 ? __ldcg(&x[j[u]]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) acc += a[u] * xv[u];
  }
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  if (sl == 0) part[tib] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    T sum = (q ? q[s] : T(1)) * rhs[s];
    for (int k = 0; k < tpb; ++k) sum += part[k];
    x[s] = sum;
  }
  __syncthreads();
}

// One chunk of a heavy row (block rows, t > 1): the team gathers its dependencies, stores the
// partial row, and the team that completes the row's last chunk finishes the row.
template <typename T, int LPV, int NV, int UNR>
__device__ __forceinline__ void chunk_run(const HeavyChunk& hc, const LevelPlan& L, const int32_t* __restrict__ idx,
                                          const T* __restrict__ val, const T* __restrict__ rhs,
                                          const T* __restrict__ q, T* x, int ld) {
  constexpr int VEC = VecT<T>::n;
  using V = typename VecT<T>::type;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T* part = static_cast<T*>(L.part);
  T acc[NV * VEC];
#pragma unroll
  for (int i = 0; i < NV * VEC; ++i) acc[i] = T(0);
  for (int e0 = hc.beg; e0 < hc.end; e0 += LPV) {
    const int cnt = min(LPV, hc.end - e0);
    const int jl = sl < cnt ? idx[e0 + sl] : -1;
    const T al = jl >= 0 ? val[e0 + sl] : T(0);
    chunk_gather<T, LPV, NV, UNR>(acc, jl, al, cnt, x, ld);
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const int col = (sl + LPV * v) * VEC;
    if (col < ld) store_vec(part + (int64_t)hc.slot * ld + col, acc + v * VEC);
  }
  __threadfence();
  __syncwarp(mask);
  int last = 0;
  if (sl == 0) last = atomicAdd(&L.cnt[hc.hrow], 1) == hc.nch - 1;
  last = __shfl_sync(mask, last, 0, LPV);
  if (!last) return;
  __threadfence();
  const int s = L.task[hc.p];
  team_init<T, LPV, NV>(acc, s, ld, q ? q[s] : T(1), rhs, T(0), nullptr);
  for (int k = 0; k < hc.nch; ++k)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int col = (sl + LPV * v) * VEC;
      if (col < ld) fma_vec(acc + v * VEC, T(1), ldcg_vec(part + (int64_t)(hc.base + k) * ld + col));
    }
  team_store<T, LPV, NV>(x, s, ld, T(1), acc);
  if (sl == 0) L.cnt[hc.hrow] = 0;
}

// One chunk of a heavy scalar row (t = 1): the team's lanes split the chunk's dependencies
// (K loads each in flight), lane 0 stores the partial; the last chunk's team finishes the row.
template <typename T, int LPV>
__device__ __forceinline__ void chunk_run1(const HeavyChunk& hc, const LevelPlan& L, const int32_t* __restrict__ idx,
                                           const T* __restrict__ val, const T* __restrict__ rhs,
                                           const T* __restrict__ q, T* x) {
  constexpr int K = 4;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T* part = static_cast<T*>(L.part);
  T acc = T(0);
  for (int e0 = hc.beg + sl; e0 < hc.end; e0 += LPV * K) {
    int j[K];
    T a[K], xv[K];
#pragma unroll
    for (int u = 0; u < K; ++u) {
      const int e = e0 + u * LPV;
      j[u] = e < hc.end ? idx[e] : -1;
      a[u] = j[u] >= 0 ? val[e] : T(0);
      xv[u] = j[u] >= 0 ? __ldcg(&x[j[u]]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < K; ++u) acc += a[u] * xv[u];
  }
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  int last = 0;
  if (sl == 0) {
    part[hc.slot] = acc;
    __threadfence();
    last = atomicAdd(&L.cnt[hc.hrow], 1) == hc.nch - 1;
    if (last) {
      __threadfence();
      const int s = L.task[hc.p];
      T sum = (q ? q[s] : T(1)) * rhs[s];
      for (int k = 0; k < hc.nch; ++k) sum += __ldcg(&part[hc.base + k]);
      x[s] = sum;
      L.cnt[hc.hrow] = 0;
    }
  }
  __syncwarp(mask);
}

// Walks the levels with the head/body/tail split; each team prefetches its next
// light row (pre) before the barrier that precedes it and finishes it after
// (run); the heavy rows that lead each level are done first, a block per row
// (heavy(p), called by every thread of the block).
template <int LPV, int BAR, typename Pre, typename Run, typename Heavy, typename Chunk>
__device__ __forceinline__ void level_walk(const LevelPlan& L, Pre pre, Run run, Heavy heavy, Chunk chunk) {
  constexpr int RPW = 32 / LPV;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int G = gridDim.x * tpb, g = blockIdx.x * tpb + tib;
  const bool tr = L.trace && blockIdx.x == 0 && threadIdx.x == 0;
  auto first_light = [&](int l, int start, int& p) {
    p = L.hptr[l] + start;
    return p < L.lptr[l + 1];
  };
  // one block: levels [l0, l1) with a block barrier after each
  auto solo = [&](int l0, int l1) {
    int p = 0;
    bool has = l0 < l1 && first_light(l0, tib, p);
    if (has) pre(p);
    for (int l = l0; l < l1; ++l) {
      if (tr) L.trace[l] = clock64();
      for (int h = L.lptr[l]; h < L.hptr[l]; ++h) heavy(h);
      while (has) {
        run();
        p += tpb;
        has = p < L.lptr[l + 1];
        if (has) pre(p);
      }
      if (l + 1 < l1) {
        has = first_light(l + 1, tib, p);
        if (has) pre(p);
      }
      __syncthreads();
    }
  };
  unsigned epoch = 0;
  if (!L.head_done) {
    if (blockIdx.x == 0) solo(0, L.l_head);
    if (L.l_head > 0 && L.l_head < L.nlev) grid_barrier<BAR>(L.bar, L.st, epoch);
  }
  {
    int p = 0;
    bool has = L.l_head < L.l_tail && first_light(L.l_head, g, p);
    if (has) pre(p);
    for (int l = L.l_head; l < L.l_tail; ++l) {
      if (tr) L.trace[l] = clock64();
      if (L.chunk && L.cptr[l + 1] > L.cptr[l]) {
        // chunks from the last team down, light rows from the first team up
        for (int c = L.cptr[l] + (G - 1 - g); c < L.cptr[l + 1]; c += G) chunk(L.chunk[c]);
      } else {
        for (int h = L.lptr[l] + blockIdx.x; h < L.hptr[l]; h += gridDim.x) heavy(h);
      }
      while (has) {
        run();
        p += G;
        has = p < L.lptr[l + 1];
        if (has) pre(p);
      }
      if (l + 1 < L.l_tail) {
        has = first_light(l + 1, g, p);
        if (has) pre(p);
      }
      grid_barrier<BAR>(L.bar, L.st, epoch);
    }
  }
  if (blockIdx.x == 0) solo(L.l_tail, L.nlev);
  if (tr) L.trace[L.nlev] = clock64();
}

// Scalar-row (t = 1) solve by one thread-block cluster: the cluster walks every
// level with the hardware cluster barrier between levels (release/acquire at
// cluster scope). A t = 1 solve moves a few megabytes, so its time is the level
// chain; a cluster barrier is far cheaper than a grid-wide one, and the rest of
// the GPU stays free. Each team prefetches its next row before the barrier.
template <typename T, bool FWD, int LPV>
__global__ void __launch_bounds__(1024) sptrsv_t1_cluster_kernel(LevelPlan L, int m, const int32_t* __restrict__ idx,
                                                                 const T* __restrict__ val,
                                                                 const int32_t* __restrict__ rowptr,
                                                                 const T* __restrict__ rhs, const T* __restrict__ q,
                                                                 T* x) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  constexpr int RPW = 32 / LPV;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int G = (int)cl.num_blocks() * tpb, g = (int)cl.block_rank() * tpb + tib;
  const bool tr = L.trace && cl.block_rank() == 0 && threadIdx.x == 0;
  RowPre1<T, LPV> r;
  int p = L.lptr[0] + g;
  bool has = L.nlev > 0 && p < L.lptr[1];
  if (has) row_pre1<T, FWD, LPV>(r, p, m, L, idx, val, rowptr, rhs, q);
  for (int l = 0; l < L.nlev; ++l) {
    if (tr) L.trace[l] = clock64();
    while (has) {
      row_run1<T, LPV>(r, idx, val, x);
      p += G;
      has = p < L.lptr[l + 1];
      if (has) row_pre1<T, FWD, LPV>(r, p, m, L, idx, val, rowptr, rhs, q);
    }
    if (l + 1 < L.nlev) {
      p = L.lptr[l + 1] + g;
      has = p < L.lptr[l + 2];
      if (has) row_pre1<T, FWD, LPV>(r, p, m, L, idx, val, rowptr, rhs, q);
    }
    cl.sync();
  }
  if (tr) L.trace[L.nlev] = clock64();
}

// Scalar-row (t = 1) solve of a small system by one block with x resident in
// shared memory (n * sizeof(T) bytes of dynamic shared memory): a level costs
// shared-memory gathers and one block barrier, nothing goes through L2 between
// levels, and the solve occupies a single SM so that independent problems run
// side by side. Each team keeps its rows (indices, weights, scaled right-hand side)
// for the next few levels in registers, so their loads are issued levels before
// they are used; x is written out once at the end.
template <typename T, int LPV>
__device__ __forceinline__ void row_run1_smem(RowPre1<T, LPV>& r, const int32_t* __restrict__ idx,
                                              const T* __restrict__ val, T* xs) {
  constexpr int K = RowPre1<T, LPV>::K;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T acc = T(0);
#pragma unroll
  for (int u = 0; u < K; ++u) acc += r.j[u] >= 0 ? r.a[u] * xs[r.j[u]] : T(0);
  for (int e = r.beg + sl + LPV * K; e < r.end; e += LPV) acc += val[e] * xs[idx[e]];
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  if (sl == 0) xs[r.s] = r.b + acc;
}

template <typename T, bool FWD, int LPV>
__global__ void __launch_bounds__(1024) sptrsv_t1_smem_kernel(LevelPlan L, int n, int m, const int32_t* __restrict__ idx,
                                                              const T* __restrict__ val,
                                                              const int32_t* __restrict__ rowptr,
                                                              const T* __restrict__ rhs, const T* __restrict__ q, T* x) {
  extern __shared__ unsigned char vl_smem[];
  T* xs = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV;
  // levels of look-ahead (a level is too short to hide one L2 round trip); two for float64
  // rows, which need twice the registers of the 64-register budget of 1024-thread blocks
  constexpr int D = sizeof(T) == 4 ? 3 : 2;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const bool tr = L.trace && threadIdx.x == 0;
  // r[d]: this team's first row of level l + d, loaded D levels before it is needed
  RowPre1<T, LPV> r[D];
  bool h[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int p = d < L.nlev ? L.lptr[d] + tib : 0;
    h[d] = d < L.nlev && p < L.lptr[d + 1];
    if (h[d]) row_pre1<T, FWD, LPV>(r[d], p, m, L, idx, val, rowptr, rhs, q);
  }
  // the level loop is unrolled by D so that every ring slot has a fixed index: a
  // register move from slot to slot would wait for the slot's loads and undo the
  // look-ahead
  for (int l0 = 0; l0 < L.nlev; l0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int l = l0 + d;
      if (l < L.nlev) {   // uniform across the block
        if (tr) L.trace[l] = clock64();
        if (h[d]) {
          row_run1_smem<T, LPV>(r[d], idx, val, xs);
          // levels wider than the block's teams: the further rows are loaded on the spot
          for (int p = L.lptr[l] + tib + tpb; p < L.lptr[l + 1]; p += tpb) {
            RowPre1<T, LPV> e;
            row_pre1<T, FWD, LPV>(e, p, m, L, idx, val, rowptr, rhs, q);
            row_run1_smem<T, LPV>(e, idx, val, xs);
          }
        }
        const int ln = l + D;
        const int p = ln < L.nlev ? L.lptr[ln] + tib : 0;
        h[d] = ln < L.nlev && p < L.lptr[ln + 1];
        if (h[d]) row_pre1<T, FWD, LPV>(r[d], p, m, L, idx, val, rowptr, rhs, q);
        __syncthreads();
      }
    }
  }
  if (tr) L.trace[L.nlev] = clock64();
  for (int s = threadIdx.x; s < n; s += blockDim.x) x[s] = xs[s];
}

// The leading levels [0, L.l_head) of a scalar forward solve by one block with x in shared
// memory, indexed by task position (the head's rows depend only on rows of earlier head
// levels): hpos[p * m + c] is the task position of dependency c of the row at position p (-1:
// none), its weight val[s * m + c] (s = task[p]). Rows of the next D levels are loaded D levels
// ahead into ring slots with fixed indices, as in sptrsv_t1_smem_kernel; every row is also
// written to x for the levels after the head (the grid kernel that follows).
template <typename T, int LPV>
__device__ __forceinline__ void head_pre(RowPre1<T, LPV>& r, int p, int m, const LevelPlan& L,
                                         const int32_t* __restrict__ hpos, const T* __restrict__ val,
                                         const T* __restrict__ rhs, const T* __restrict__ q) {
  const int sl = (threadIdx.x & 31) % LPV;
  r.s = L.task[p];
  r.beg = p * m;
  r.end = p * m + m;
#pragma unroll
  for (int u = 0; u < RowPre1<T, LPV>::K; ++u) {
    const int c = sl + u * LPV;
    r.j[u] = c < m ? hpos[r.beg + c] : -1;
    r.a[u] = r.j[u] >= 0 ? val[(int64_t)r.s * m + c] : T(0);
  }
  r.b = (q ? q[r.s] : T(1)) * rhs[r.s];
}

template <typename T, int LPV>
__device__ __forceinline__ void head_run(RowPre1<T, LPV>& r, int p, int m, const int32_t* __restrict__ hpos,
                                         const T* __restrict__ val, T* xs, T* x) {
  constexpr int K = RowPre1<T, LPV>::K;
  const unsigned mask = team_mask<LPV>();
  const int sl = (threadIdx.x & 31) % LPV;
  T acc = T(0);
#pragma unroll
  for (int u = 0; u < K; ++u) acc += r.j[u] >= 0 ? r.a[u] * xs[r.j[u]] : T(0);
  for (int c = sl + LPV * K; c < m; c += LPV) {
    const int j = hpos[r.beg + c];
    if (j >= 0) acc += val[(int64_t)r.s * m + c] * xs[j];
  }
#pragma unroll
  for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
  if (sl == 0) {
    const T v = r.b + acc;
    xs[p] = v;
    x[r.s] = v;
  }
}

template <typename T, int LPV>
__global__ void __launch_bounds__(1024) sptrsv_t1_head_kernel(LevelPlan L, int m, const int32_t* __restrict__ hpos,
                                                              const T* __restrict__ val, const T* __restrict__ rhs,
                                                              const T* __restrict__ q, T* x) {
  extern __shared__ unsigned char vl_smem[];
  T* xs = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV;
  constexpr int D = sizeof(T) == 4 ? 3 : 2;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int nl = L.l_head;
  const bool tr = L.trace && threadIdx.x == 0;
  RowPre1<T, LPV> r[D];
  bool h[D];
  int pr[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    pr[d] = d < nl ? L.lptr[d] + tib : 0;
    h[d] = d < nl && pr[d] < L.lptr[d + 1];
    if (h[d]) head_pre<T, LPV>(r[d], pr[d], m, L, hpos, val, rhs, q);
  }
  for (int l0 = 0; l0 < nl; l0 += D) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int l = l0 + d;
      if (l < nl) {   // uniform across the block
        if (tr) L.trace[l] = clock64();
        if (h[d]) {
          head_run<T, LPV>(r[d], pr[d], m, hpos, val, xs, x);
          for (int p = pr[d] + tpb; p < L.lptr[l + 1]; p += tpb) {
            RowPre1<T, LPV> e;
            head_pre<T, LPV>(e, p, m, L, hpos, val, rhs, q);
            head_run<T, LPV>(e, p, m, hpos, val, xs, x);
          }
        }
        const int ln = l + D;
        pr[d] = ln < nl ? L.lptr[ln] + tib : 0;
        h[d] = ln < nl && pr[d] < L.lptr[ln + 1];
        if (h[d]) head_pre<T, LPV>(r[d], pr[d], m, L, hpos, val, rhs, q);
        __syncthreads();
      }
    }
  }
}

// Block (t > 1) solve by one thread-block cluster: the level walk of the grid
// kernel with the hardware cluster barrier in place of the grid barrier. Heavy
// rows go to whole blocks of the cluster (one row per block at a time), light
// rows to teams, each prefetched before the barrier.
template <typename T, bool FWD, int LPV, int NV, int UNR>
__global__ void __launch_bounds__(1024) sptrsv_cluster_kernel(LevelPlan L, int m, const int32_t* __restrict__ idx,
                                                              const T* __restrict__ val,
                                                              const int32_t* __restrict__ rowptr,
                                                              const T* __restrict__ rhs, const T* __restrict__ q, T* x,
                                                              int ld) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ unsigned char vl_smem[];
  T* part = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV;
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int nb = (int)cl.num_blocks(), br = (int)cl.block_rank();
  const int G = nb * tpb, g = br * tpb + tib;
  const bool tr = L.trace && br == 0 && threadIdx.x == 0;
  RowPre<T, LPV, NV> r;
  int p = 0;
  bool has = L.nlev > 0 && (p = L.hptr[0] + g) < L.lptr[1];
  if (has) row_pre<T, FWD, LPV, NV>(r, p, m, L, idx, val, rowptr, rhs, q, ld);
  for (int l = 0; l < L.nlev; ++l) {
    if (tr) L.trace[l] = clock64();
    for (int h = L.lptr[l] + br; h < L.hptr[l]; h += nb)
      heavy_row<T, FWD, LPV, NV, UNR>(h, m, L, idx, val, rowptr, rhs, q, x, ld, part);
    while (has) {
      row_run<T, LPV, NV, UNR>(r, idx, val, x, ld);
      p += G;
      has = p < L.lptr[l + 1];
      if (has) row_pre<T, FWD, LPV, NV>(r, p, m, L, idx, val, rowptr, rhs, q, ld);
    }
    if (l + 1 < L.nlev) {
      p = L.hptr[l + 1] + g;
      has = p < L.lptr[l + 2];
      if (has) row_pre<T, FWD, LPV, NV>(r, p, m, L, idx, val, rowptr, rhs, q, ld);
    }
    cl.sync();
  }
  if (tr) L.trace[L.nlev] = clock64();
}

template <typename T, bool FWD, int LPV, int NV, int UNR, int BAR = 0, int PF = 0>
__global__ void __launch_bounds__(512) sptrsv_kernel(LevelPlan L, int m, const int32_t* __restrict__ idx,
                                                     const T* __restrict__ val, const int32_t* __restrict__ rowptr,
                                                     const T* __restrict__ rhs, const T* __restrict__ q, T* x, int ld) {
  extern __shared__ unsigned char vl_smem[];
  T* part = reinterpret_cast<T*>(vl_smem);
  RowPre<T, LPV, NV> r;
  level_walk<LPV, BAR>(
      L, [&](int p) { row_pre<T, FWD, LPV, NV>(r, p, m, L, idx, val, rowptr, rhs, q, ld, PF ? x : nullptr); },
      [&]() { row_run<T, LPV, NV, UNR>(r, idx, val, x, ld); },
      [&](int p) { heavy_row<T, FWD, LPV, NV, UNR>(p, m, L, idx, val, rowptr, rhs, q, x, ld, part); },
      [&](const HeavyChunk& hc) { chunk_run<T, LPV, NV, UNR>(hc, L, idx, val, rhs, q, x, ld); });
}

template <typename T, bool FWD, int LPV, int BAR = 1>
__global__ void __launch_bounds__(512) sptrsv_t1_kernel(LevelPlan L, int m, const int32_t* __restrict__ idx,
                                                        const T* __restrict__ val, const int32_t* __restrict__ rowptr,
                                                        const T* __restrict__ rhs, const T* __restrict__ q, T* x) {
  extern __shared__ unsigned char vl_smem[];
  T* part = reinterpret_cast<T*>(vl_smem);
  RowPre1<T, LPV> r;
  level_walk<LPV, BAR>(
      L, [&](int p) { row_pre1<T, FWD, LPV>(r, p, m, L, idx, val, rowptr, rhs, q); },
      [&]() { row_run1<T, LPV>(r, idx, val, x); },
      [&](int p) { heavy_row1<T, FWD, LPV>(p, m, L, idx, val, rowptr, rhs, q, x, part); },
      [&](const HeavyChunk& hc) { chunk_run1<T, LPV>(hc, L, idx, val, rhs, q, x); });
}

// ----------------------------------------------------------------------------- tiled solves
// Triangular solve by storage-row tiles with no barrier at all (plan: tile_plan.h). Tile b (one
// block) owns the storage rows [b R, min(n, (b + 1) R)); the block's teams take the tile's rows,
// listed by level, round robin, and a row waits only for its own dependencies: a dependency in
// the tile through shared memory, one in another tile through global memory. In a random
// ordering the dependency chain is hundreds of rows long but most of its links stay inside a
// tile (the rows are in Morton order, a tile is a compact patch), so most links cost a
// shared-memory hand-off instead of a grid-wide barrier. Every wait is bounded (a timeout
// records VL_ERR_TIMEOUT and every other wait then returns at once).
struct TileArgs {
  const int32_t* ttask;      // n: each tile's rows by level, tiles in order
  const int32_t* toff;       // G + 1
  const uint8_t* exported;   // n: a row of another tile depends on this row (t > 1 flags)
  int* flag;                 // n: epoch of the last solve that finished the row (t > 1)
  DevStatus* st;
  int n, R;
  int epoch;
};

// float / double "not yet solved" marker: all bits set (a NaN no solve produces: results equal
// to it are replaced by the canonical quiet NaN)
__device__ __forceinline__ bool is_unsolved(float v) { return __float_as_uint(v) == 0xffffffffu; }
__device__ __forceinline__ bool is_unsolved(double v) { return __double_as_longlong(v) == -1LL; }
__device__ __forceinline__ float unsolved_value(float) { return __uint_as_float(0xffffffffu); }
__device__ __forceinline__ double unsolved_value(double) { return __longlong_as_double(-1LL); }
__device__ __forceinline__ float solved_value(float v) { return is_unsolved(v) ? __uint_as_float(0x7fc00000u) : v; }
__device__ __forceinline__ double solved_value(double v) {
  return is_unsolved(v) ? __longlong_as_double(0x7ff8000000000000LL) : v;
}

// Value of a dependency once it is solved (bounded: after a timeout or an abort the value read
// last is returned and the solve's result is void).
template <typename T>
__device__ __forceinline__ T tile_wait_value(const T* p, DevStatus* st, int row) {
  T v = *(volatile const T*)p;
  if (!is_unsolved(v)) return v;
  long long t0 = 0, limit = 0;
  for (int it = 1;; ++it) {
    __nanosleep(20);   // leave issue slots to the warps that produce the value
    v = *(volatile const T*)p;
    if (!is_unsolved(v)) return v;
    if ((it & 63) == 0) {
      if (ld_volatile(&st->abort)) return v;
      if (t0 == 0) {
        t0 = clock64();
        const long long set = *(volatile const long long*)&st->limit;
        limit = set > 0 ? set : kSpinLimitCycles;
      } else if (clock64() - t0 > limit) {
        raise_error(st, VL_ERR_TIMEOUT, row);
        return v;
      }
    }
  }
}

// Scalar rows (t = 1): the tile's x in shared memory, every row also stored to x for the other
// tiles; x starts "unsolved" (all bits set by the host before the launch) except on the rows a
// kernel before this one solved, so a value is its own ready flag and no fence is needed. Team lanes split a row's dependencies (K loads each).
template <typename T, bool FWD, int LPV>
__global__ void __launch_bounds__(1024) sptrsv_tile1_kernel(TileArgs A, int m, const int32_t* __restrict__ idx,
                                                            const T* __restrict__ val,
                                                            const int32_t* __restrict__ rowptr,
                                                            const T* __restrict__ rhs, const T* __restrict__ q, T* x) {
  extern __shared__ unsigned char vl_smem[];
  T* xs = reinterpret_cast<T*>(vl_smem);
  constexpr int RPW = 32 / LPV, K = 4;
  const unsigned mask = team_mask<LPV>();
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  const int b = blockIdx.x;
  const int r0 = b * A.R, r1 = min(A.n, r0 + A.R);
  // x holds "unsolved" everywhere but on the rows solved before the walk (the forward head)
  for (int i = threadIdx.x; i < r1 - r0; i += blockDim.x) xs[i] = __ldcg(x + r0 + i);
  __syncthreads();
  for (int p = A.toff[b] + tib; p < A.toff[b + 1]; p += tpb) {
    const int s = A.ttask[p];
    const int beg = FWD ? s * m : rowptr[s];
    const int end = FWD ? s * m + m : rowptr[s + 1];
    const T bs = (q ? q[s] : T(1)) * rhs[s];
    T acc = T(0);
    for (int e0 = beg + sl; e0 < end; e0 += LPV * K) {
      int j[K];
      T a[K], xv[K];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const int e = e0 + u * LPV;
        j[u] = e < end ? idx[e] : -1;
        a[u] = j[u] >= 0 ? val[e] : T(0);
      }
      // the K loads go out together; only a value still unsolved is waited for
      const T* src[K];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        src[u] = j[u] < 0 ? nullptr : ((j[u] >= r0 && j[u] < r1) ? xs + (j[u] - r0) : x + j[u]);
        xv[u] = src[u] ? *(volatile const T*)src[u] : T(0);
      }
#pragma unroll
      for (int u = 0; u < K; ++u)
        if (src[u] && is_unsolved(xv[u])) xv[u] = tile_wait_value(src[u], A.st, s);
#pragma unroll
      for (int u = 0; u < K; ++u) acc += a[u] * xv[u];
    }
#pragma unroll
    for (int off = LPV / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(mask, acc, off, LPV);
    if (sl == 0) {
      const T v = solved_value(bs + acc);
      *(volatile T*)(xs + (s - r0)) = v;
      *(volatile T*)(x + s) = v;
    }
  }
}

// Block rows (t > 1): x in global memory (a tile's rows are too wide for shared memory), ready
// flags per row: in shared memory for the tile, and in global memory (the launch's epoch) for
// the rows that another tile depends on, written after a gpu-scope fence of the team's stores.
// Each lane waits for the dependency it holds, the team meets (__syncwarp), then every lane
// gathers its words of the chunk's rows as in the grid walk.
template <typename T, bool FWD, int LPV, int NV, int UNR>
__global__ void __launch_bounds__(512) sptrsv_tile_kernel(TileArgs A, int m,
                                                          const int32_t* __restrict__ idx, const T* __restrict__ val,
                                                          const int32_t* __restrict__ rowptr,
                                                          const T* __restrict__ rhs, const T* __restrict__ q, T* x,
                                                          int ld) {
  extern __shared__ unsigned char vl_smem[];
  int* rf = reinterpret_cast<int*>(vl_smem);
  constexpr int RPW = 32 / LPV;
  const unsigned mask = team_mask<LPV>();
  const int tpb = (blockDim.x >> 5) * RPW;
  const int tib = (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / LPV;
  const int sl = (threadIdx.x & 31) % LPV;
  const int b = blockIdx.x;
  const int r0 = b * A.R, r1 = min(A.n, r0 + A.R);
  for (int i = threadIdx.x; i < r1 - r0; i += blockDim.x) rf[i] = 0;
  __syncthreads();
  for (int p = A.toff[b] + tib; p < A.toff[b + 1]; p += tpb) {
    const int s = A.ttask[p];
    RowPre<T, LPV, NV> r;
    row_pre_s<T, FWD, LPV, NV>(r, s, m, idx, val, rowptr, rhs, q, ld);
    for (int e0 = r.beg; e0 < r.end; e0 += LPV) {
      const int cnt = min(LPV, r.end - e0);
      int jl = r.jl;
      T al = r.al;
      if (e0 != r.beg) {
        jl = sl < cnt ? idx[e0 + sl] : -1;
        al = jl >= 0 ? val[e0 + sl] : T(0);
      }
      if (jl >= 0) {
        if (jl >= r0 && jl < r1) {
          const int* f = rf + (jl - r0);
          bounded_wait([&] { return *(volatile const int*)f != 0; }, A.st, s);
        } else {
          const int* f = A.flag + jl;
          bounded_wait([&] { return ld_acquire(f) == A.epoch; }, A.st, s);
        }
      }
      __syncwarp(mask);
      chunk_gather<T, LPV, NV, UNR>(r.acc, jl, al, cnt, x, ld);
    }
    team_store<T, LPV, NV>(x, r.s, ld, T(1), r.acc);
    const bool ex = A.exported[s] != 0;
    if (ex) __threadfence();
    else __threadfence_block();
    __syncwarp(mask);
    if (sl == 0) {
      *(volatile int*)(rf + (s - r0)) = 1;
      if (ex) st_release(A.flag + s, A.epoch);
    }
  }
}

// ----------------------------------------------------------------------------- column reductions
// Rows are swept by reduction blocks of blockDim = (cx, 256 / cx), cx = 1 for t == 1, else a
// multiple of 32 covering t. Block b covers rows [row0(b), row1(b)) of segment seg(b): the
// problems of a batch are segments of the storage rows, a single problem is one segment with
// blocks of rpb rows. A block never straddles segments, so a per-(segment, column) sum is a
// sum of whole blocks taken in block order, and results do not depend on scheduling.
struct BlockRows {
  int n, rpb, nblk, nseg;
  const int32_t* r0;    // per block first row (null: b * rpb)
  const int32_t* r1;    // per block end row (null: min(n, (b + 1) * rpb))
  const int32_t* seg;   // per block segment (null: 0)
  const int32_t* sb0;   // per segment first block, nseg + 1 entries (null: 0, nblk)
  __device__ __forceinline__ int row0(int b) const { return r0 ? r0[b] : b * rpb; }
  __device__ __forceinline__ int row1(int b) const { return r1 ? r1[b] : min(n, (b + 1) * rpb); }
  __device__ __forceinline__ int segment(int b) const { return seg ? seg[b] : 0; }
  __device__ __forceinline__ int blk0(int k) const { return sb0 ? sb0[k] : 0; }
  __device__ __forceinline__ int blk1(int k) const { return sb0 ? sb0[k + 1] : nblk; }
};

// ----------------------------------------------------------------------------- PCG scalars
// Per (segment, column) q = k * t + c, ncol = nseg * t entries each.
struct PcgScalars {
  double* rz;          // r_l^T z_l
  double* rz0;         // r_0^T z_0 = ||P^{-1/2} b||^2
  double* alpha;       // alpha_{l+1}
  double* beta;        // beta_{l+1}
  double* alpha_prev;  // alpha_l   (alpha_0 = 1)
  double* beta_prev;   // beta_l    (beta_0 = 0)
  double* bnorm2;
  double* rnorm2;
  double* relres;
  const double* tol2;  // per column squared relative tolerance (null: the scalar of the call)
  int* active;
  int* stop;
  int* iters;
  double* Tdiag;       // ncol x lmax
  double* Toff;        // ncol x lmax
  int lmax;
  int* count;          // number of active columns after the update
};

// r_0 = b, z_0 = P^{-1} r_0: set rz, rz0, bnorm2 (already reduced into rz/bnorm2) and flags.
static __global__ void pcg_init_kernel(int ncol, PcgScalars S) {
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    S.rz0[c] = S.rz[c];
    S.alpha_prev[c] = 1.0;
    S.beta_prev[c] = 0.0;
    S.iters[c] = 0;
    S.stop[c] = 0;
    S.alpha[c] = 0.0;
    S.beta[c] = 0.0;
    const bool act = S.bnorm2[c] > 0.0 && S.rz[c] > 0.0;
    S.active[c] = act ? 1 : 0;
    S.relres[c] = act ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) *S.count = 1;
}

// What the last block of a column reduction does with the sums (Appendix, PCG algorithm):
enum ReduceEpilogue {
  EPI_NONE = 0,   // out = the sums
  EPI_ALPHA = 1,  // alpha_{l+1} = r_l^T z_l / h_l^T v_l (active columns; 0 otherwise)
  EPI_STOP = 2,   // ||r_{l+1}||^2 and the stopping test (before the T update, as in the algorithm)
  EPI_BETA = 3    // beta_{l+1}, the T entries, the freeze of finished columns, the active count
};

struct ReduceTail {
  int epi;
  double* out;          // EPI_NONE: ncol sums
  PcgScalars S;
  double tol2;          // EPI_STOP: squared relative tolerance (when S.tol2 is null)
  int max_iter;         // EPI_BETA
  unsigned* done;       // arrival counter of the launch's blocks (zero at launch, reset by the last)
};

// Column sums of a block's per-thread values acc (thread (c, y) of blockDim (cx, ry)) into
// sh[c] by a fixed pairwise tree over y; ry is a power of two. Every thread calls it.
__device__ __forceinline__ double block_col_sum(double acc, double* sh) {
  const int cx = blockDim.x, c = threadIdx.x, y = threadIdx.y;
  sh[y * cx + c] = acc;
  __syncthreads();
  for (int h = blockDim.y >> 1; h > 0; h >>= 1) {
    if (y < h) sh[y * cx + c] += sh[(y + h) * cx + c];
    __syncthreads();
  }
  return sh[c];
}

// Runs in the last block to finish: per (segment, column) sums of the block partials, each
// by one warp (lanes take the segment's blocks at a stride of 32, then a fixed shuffle tree,
// so the order does not depend on scheduling), then the epilogue. Every thread calls it.
__device__ __forceinline__ void reduce_tail(const BlockRows& br, int t, const double* __restrict__ partial,
                                            const ReduceTail& rt) {
  __shared__ int last;
  __shared__ int cnt;
  __syncthreads();
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  if (tid == 0) {
    __threadfence();
    last = atomicAdd(rt.done, 1u) == gridDim.x - 1;
    cnt = 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const PcgScalars& S = rt.S;
  int local = 0;
  const int ncol = br.nseg * t;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nth >> 5;
  for (int q = warp; q < ncol; q += nwarp) {
    const int k = q / t, c = q - k * t;
    double sum = 0.0;
    for (int b = br.blk0(k) + lane; b < br.blk1(k); b += 32) sum += __ldcg(&partial[(int64_t)b * t + c]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane != 0) continue;
    if (rt.epi == EPI_NONE) {
      rt.out[q] = sum;
    } else if (rt.epi == EPI_ALPHA) {
      const double a = S.active[q] ? S.rz[q] / sum : 0.0;
      S.alpha[q] = (S.active[q] && isfinite(a)) ? a : 0.0;
    } else if (rt.epi == EPI_STOP) {
      if (!S.active[q]) continue;
      S.rnorm2[q] = sum;
      S.relres[q] = sqrt(sum / S.bnorm2[q]);
      const double tl = S.tol2 ? S.tol2[q] : rt.tol2;
      S.stop[q] = (sum <= tl * S.bnorm2[q]) ? 1 : 0;
    } else {   // EPI_BETA
      if (!S.active[q]) continue;
      const int l = S.iters[q];
      const double a = S.alpha[q], ap = S.alpha_prev[q], bp = S.beta_prev[q];
      const double bt = sum / S.rz[q];
      if (l < S.lmax) {
        S.Tdiag[(int64_t)q * S.lmax + l] = 1.0 / a + bp / ap;
        if (l > 0) S.Toff[(int64_t)q * S.lmax + l - 1] = sqrt(bp) / ap;
      }
      S.beta[q] = bt;
      S.alpha_prev[q] = a;
      S.beta_prev[q] = bt;
      S.rz[q] = sum;
      S.iters[q] = l + 1;
      if (S.stop[q] || l + 1 >= rt.max_iter || l + 1 >= S.lmax || !(a > 0.0) || !isfinite(bt))
        S.active[q] = 0;
      else
        ++local;
    }
  }
  if (rt.epi == EPI_BETA) {
    atomicAdd(&cnt, local);
    __syncthreads();
    if (tid == 0) *S.count = cnt;
  }
  if (tid == 0) *rt.done = 0u;
}

// partial[b * t + c] = sum over block b's rows of w_s X[s,c] Y[s,c] (w == nullptr: 1), then
// the last block's reduce_tail. Accumulation: float64 for float64 data; float32 partials of
// 16 rows each, flushed to float64.
template <typename T>
__global__ void coldot_kernel(BlockRows br, int t, int ld, const T* __restrict__ X, const T* __restrict__ Y,
                              const T* __restrict__ w, double* __restrict__ partial, ReduceTail rt) {
  const int ry = blockDim.y;
  const int c = threadIdx.x;
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  double acc = 0.0;
  if (c < t) {
    T a = T(0);
    int cntf = 0;
    for (int s = r0 + threadIdx.y; s < r1; s += ry) {
      const int64_t o = (int64_t)s * ld + c;
      T v = X[o] * Y[o];
      if (w) v *= w[s];
      a += v;
      if (++cntf == 16) {   // flush the working-precision partial every 16 rows
        acc += (double)a;
        a = T(0);
        cntf = 0;
      }
    }
    acc += (double)a;
  }
  extern __shared__ double sh[];
  const double sum = block_col_sum(acc, sh);
  if (threadIdx.y == 0 && c < t) {
    partial[(int64_t)blockIdx.x * t + c] = sum;
    __threadfence();
  }
  reduce_tail(br, t, partial, rt);
}

// u += alpha h, r -= alpha v (alpha = 0 for frozen columns) with ||r||^2 partials, then the
// stopping test in the last block.
template <typename T>
__global__ void pcg_update1_kernel(BlockRows br, int t, int ld, T* __restrict__ u, T* __restrict__ r,
                                   const T* __restrict__ h, const T* __restrict__ v, double* __restrict__ partial,
                                   ReduceTail rt) {
  const int ry = blockDim.y;
  const int c = threadIdx.x;
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  const int k = br.segment(blockIdx.x);
  double acc = 0.0;
  if (c < t) {
    const T a = (T)rt.S.alpha[k * t + c];
    T part = T(0);
    int cntf = 0;
    for (int s = r0 + threadIdx.y; s < r1; s += ry) {
      const int64_t o = (int64_t)s * ld + c;
      if (a != T(0)) {
        u[o] += a * h[o];
        r[o] -= a * v[o];
      }
      const T rv = r[o];
      part += rv * rv;
      if (++cntf == 16) {
        acc += (double)part;
        part = T(0);
        cntf = 0;
      }
    }
    acc += (double)part;
  }
  extern __shared__ double sh[];
  const double sum = block_col_sum(acc, sh);
  if (threadIdx.y == 0 && c < t) {
    partial[(int64_t)blockIdx.x * t + c] = sum;
    __threadfence();
  }
  reduce_tail(br, t, partial, rt);
}

// h = z + beta h for active columns.
template <typename T>
__global__ void pcg_update2_kernel(BlockRows br, int t, int ld, const double* __restrict__ beta,
                                   const int* __restrict__ active, const T* __restrict__ z, T* __restrict__ h) {
  const int c = threadIdx.x;
  if (c >= t) return;
  const int q = br.segment(blockIdx.x) * t + c;
  if (!active[q]) return;
  const T bt = (T)beta[q];
  const int r1 = br.row1(blockIdx.x);
  for (int s = br.row0(blockIdx.x) + threadIdx.y; s < r1; s += blockDim.y) {
    const int64_t o = (int64_t)s * ld + c;
    h[o] = z[o] + bt * h[o];
  }
}

// ----------------------------------------------------------------------------- vector sweeps
// The column sweeps of block vectors (t > 1, ld a multiple of 8) with 16-byte loads: a thread
// holds one float4 / double2 word of a row (CX words per row, CX the power of two covering
// ld / VEC), a 1024-thread block sweeps 1024 / CX rows at a time, two rows per thread in flight.
// Per-word column sums are float32 partials of 16 rows flushed to float64 (float64 data: float64
// throughout), then a fixed tree over the block's row lanes in shared memory (1024 * VEC doubles),
// so the result does not depend on scheduling. The scalar (t = 1) sweeps keep the kernels above.
template <typename T>
struct VecSweep {
  static constexpr int VEC = VecT<T>::n;
  int cx, ry, w, y;   // words per row lane group, rows per sweep, this thread's word and row lane
  __device__ __forceinline__ VecSweep(int ld) {
    const int nw = ld / VEC;
    cx = nw <= 8 ? 8 : (nw <= 16 ? 16 : (nw <= 32 ? 32 : 64));
    ry = blockDim.x / cx;
    w = threadIdx.x % cx;
    y = threadIdx.x / cx;
  }
};

// acc[i] of every thread (its word's VEC columns) -> column sums over the block's row lanes into
// partial[blockIdx.x * t + c] for c < t. Every thread calls it.
template <typename T>
__device__ __forceinline__ void vec_block_sums(const VecSweep<T>& V, const double* acc, int t, double* sh,
                                               double* __restrict__ partial) {
  constexpr int VEC = VecSweep<T>::VEC;
  const int width = V.cx * VEC;
#pragma unroll
  for (int i = 0; i < VEC; ++i) sh[V.y * width + V.w * VEC + i] = acc[i];
  __syncthreads();
  for (int hh = V.ry >> 1; hh > 0; hh >>= 1) {
    if (V.y < hh)
#pragma unroll
      for (int i = 0; i < VEC; ++i) sh[V.y * width + V.w * VEC + i] += sh[(V.y + hh) * width + V.w * VEC + i];
    __syncthreads();
  }
  for (int c = threadIdx.x; c < t; c += blockDim.x) partial[(int64_t)blockIdx.x * t + c] = sh[c];
  __threadfence();
}

template <typename T>
__device__ __forceinline__ typename VecT<T>::type ld_word(const T* p) {
  return *reinterpret_cast<const typename VecT<T>::type*>(p);
}
template <typename T>
__device__ __forceinline__ void st_word(T* p, const T* a) {
  store_vec(p, a);
}
__device__ __forceinline__ void unpack(float4 v, float* a) {
  a[0] = v.x; a[1] = v.y; a[2] = v.z; a[3] = v.w;
}
__device__ __forceinline__ void unpack(double2 v, double* a) {
  a[0] = v.x; a[1] = v.y;
}

// partial[b * t + c] = sum over block b's rows of w_s X[s,c] Y[s,c] (w == nullptr: 1), then the
// last block's reduce_tail (as coldot_kernel).
template <typename T>
__global__ void __launch_bounds__(1024, 1) coldot_vec_kernel(BlockRows br, int t, int ld, const T* __restrict__ X,
                                                             const T* __restrict__ Y, const T* __restrict__ w,
                                                             double* __restrict__ partial, ReduceTail rt) {
  constexpr int VEC = VecT<T>::n;
  extern __shared__ double sh[];
  const VecSweep<T> V(ld);
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  double acc[VEC];
  T part[VEC];
#pragma unroll
  for (int i = 0; i < VEC; ++i) acc[i] = 0.0, part[i] = T(0);
  if (V.w * VEC < ld) {
    const int col = V.w * VEC;
    int cntf = 0;
    for (int s = r0 + V.y; s < r1; s += 2 * V.ry) {
      const int s2 = s + V.ry;
      const bool two = s2 < r1;
      T x0[VEC], y0[VEC], x1[VEC], y1[VEC];
      unpack(ld_word(X + (int64_t)s * ld + col), x0);
      unpack(ld_word(Y + (int64_t)s * ld + col), y0);
      if (two) {
        unpack(ld_word(X + (int64_t)s2 * ld + col), x1);
        unpack(ld_word(Y + (int64_t)s2 * ld + col), y1);
      }
      const T w0 = w ? w[s] : T(1), w1 = (w && two) ? w[s2] : T(1);
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        part[i] += w0 * x0[i] * y0[i];
        if (two) part[i] += w1 * x1[i] * y1[i];
      }
      cntf += two ? 2 : 1;
      if (cntf >= 16) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] += (double)part[i], part[i] = T(0);
        cntf = 0;
      }
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc[i] += (double)part[i];
  }
  vec_block_sums<T>(V, acc, t, sh, partial);
  reduce_tail(br, t, partial, rt);
}

// u += alpha h, r -= alpha v (alpha = 0 for frozen and padding columns) with ||r||^2 partials,
// then the stopping test in the last block (as pcg_update1_kernel).
template <typename T>
__global__ void __launch_bounds__(1024, 1) pcg_update1_vec_kernel(BlockRows br, int t, int ld, T* __restrict__ u,
                                                                  T* __restrict__ r, const T* __restrict__ h,
                                                                  const T* __restrict__ v,
                                                                  double* __restrict__ partial, ReduceTail rt) {
  constexpr int VEC = VecT<T>::n;
  extern __shared__ double sh[];
  const VecSweep<T> V(ld);
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  const int k = br.segment(blockIdx.x);
  double acc[VEC];
  T part[VEC];
#pragma unroll
  for (int i = 0; i < VEC; ++i) acc[i] = 0.0, part[i] = T(0);
  if (V.w * VEC < ld) {
    const int col = V.w * VEC;
    T a[VEC];
    bool any = false;
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
      a[i] = col + i < t ? (T)rt.S.alpha[k * t + col + i] : T(0);
      any = any || a[i] != T(0);
    }
    int cntf = 0;
    for (int s = r0 + V.y; s < r1; s += 2 * V.ry) {
      const int s2 = s + V.ry;
      const bool two = s2 < r1;
      const int64_t o0 = (int64_t)s * ld + col, o1 = (int64_t)s2 * ld + col;
      T r0v[VEC], r1v[VEC];
      unpack(ld_word(r + o0), r0v);
      if (two) unpack(ld_word(r + o1), r1v);
      if (any) {
        T u0[VEC], h0[VEC], v0[VEC], u1[VEC], h1[VEC], v1[VEC];
        unpack(ld_word(u + o0), u0);
        unpack(ld_word(h + o0), h0);
        unpack(ld_word(v + o0), v0);
        if (two) {
          unpack(ld_word(u + o1), u1);
          unpack(ld_word(h + o1), h1);
          unpack(ld_word(v + o1), v1);
        }
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
          u0[i] += a[i] * h0[i];
          r0v[i] -= a[i] * v0[i];
          if (two) {
            u1[i] += a[i] * h1[i];
            r1v[i] -= a[i] * v1[i];
          }
        }
        st_word(u + o0, u0);
        st_word(r + o0, r0v);
        if (two) {
          st_word(u + o1, u1);
          st_word(r + o1, r1v);
        }
      }
#pragma unroll
      for (int i = 0; i < VEC; ++i) {
        part[i] += r0v[i] * r0v[i];
        if (two) part[i] += r1v[i] * r1v[i];
      }
      cntf += two ? 2 : 1;
      if (cntf >= 16) {
#pragma unroll
        for (int i = 0; i < VEC; ++i) acc[i] += (double)part[i], part[i] = T(0);
        cntf = 0;
      }
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) acc[i] += (double)part[i];
  }
  vec_block_sums<T>(V, acc, t, sh, partial);
  reduce_tail(br, t, partial, rt);
}

// h = z + beta h on active columns (as pcg_update2_kernel).
template <typename T>
__global__ void __launch_bounds__(1024, 1) pcg_update2_vec_kernel(BlockRows br, int t, int ld,
                                                                  const double* __restrict__ beta,
                                                                  const int* __restrict__ active,
                                                                  const T* __restrict__ z, T* __restrict__ h) {
  constexpr int VEC = VecT<T>::n;
  const VecSweep<T> V(ld);
  if (V.w * VEC >= ld) return;
  const int col = V.w * VEC;
  const int k = br.segment(blockIdx.x);
  T bt[VEC];
  bool act[VEC], any = false;
#pragma unroll
  for (int i = 0; i < VEC; ++i) {
    const int c = col + i;
    act[i] = c < t && active[k * t + c];
    bt[i] = act[i] ? (T)beta[k * t + c] : T(0);
    any = any || act[i];
  }
  if (!any) return;
  const int r0 = br.row0(blockIdx.x), r1 = br.row1(blockIdx.x);
  for (int s = r0 + V.y; s < r1; s += 2 * V.ry) {
    const int s2 = s + V.ry;
    const bool two = s2 < r1;
    const int64_t o0 = (int64_t)s * ld + col, o1 = (int64_t)s2 * ld + col;
    T z0[VEC], h0[VEC], z1[VEC], h1[VEC];
    unpack(ld_word(z + o0), z0);
    unpack(ld_word(h + o0), h0);
    if (two) {
      unpack(ld_word(z + o1), z1);
      unpack(ld_word(h + o1), h1);
    }
#pragma unroll
    for (int i = 0; i < VEC; ++i) {
      if (act[i]) h0[i] = z0[i] + bt[i] * h0[i];
      if (two && act[i]) h1[i] = z1[i] + bt[i] * h1[i];
    }
    st_word(h + o0, h0);
    if (two) st_word(h + o1, h1);
  }
}

// out[c] = sum_b partial[b * t + c] (fixed order)
static __global__ void reduce_partials_kernel(int nblk, int t, const double* __restrict__ partial,
                                              double* __restrict__ out) {
  for (int c = threadIdx.x; c < t; c += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * t + c];
    out[c] = s;
  }
}

// ----------------------------------------------------------------------------- SLQ quadrature
// e1^T log(T) e1 for the l x l symmetric positive definite tridiagonal T of one probe (Eq.
// def_SLQ; the Gauss quadrature sum_j q_{1j}^2 log(theta_j) of its eigenpairs) from the identity
//   log(theta) = integral over s > 0 of [1 / (1 + s) - 1 / (theta + s)] ds,
// which gives e1^T log(T) e1 = integral of [1 / (1 + s) - e1^T (T + s I)^{-1} e1] ds with no
// eigen-decomposition. With s = e^u the integrand is analytic in the strip |Im u| < pi, so the
// trapezoidal rule in u converges geometrically (error ~ exp(-2 pi^2 / h)); h = 0.4 leaves it far
// below float64 rounding. e1^T (T + s I)^{-1} e1 = 1 / D_0(s) with the pivots of T + s I taken from
// the bottom row up, D_{l-1} = d_{l-1} + s, D_k = d_k + s - e_k^2 / D_{k+1}: all positive for a
// positive definite T and s >= 0, so the recurrence is stable, and clustered or repeated Ritz
// values (which Lanczos without reorthogonalisation produces) need no special care. Every node
// is independent: the float64 work spreads over many warps (float64 issues at a small fraction of
// the float32 rate on this GPU; one thread running implicit QR sweeps over a 519-row T took half
// a second). The u range covers [log(theta_lo) - 40, log(theta_hi) + 40], where the integrand is
// below 1e-17: theta_hi a Gershgorin bound, theta_lo within a factor 16 below the smallest
// eigenvalue (Sturm counts, Wilkinson's sign-count bisection). Host-callable.
constexpr double kQuadStep = 0.4;
constexpr int kQuadMaxNodes = 1024;

// Eigenvalues of T below x (the negative pivots of T - x I from the top).
__host__ __device__ inline int tridiag_count_below(int l, const double* d, const double* e, double x) {
  const double pivmin = 1e-290;
  double q = d[0] - x;
  int cnt = q < 0.0;
  for (int k = 1; k < l; ++k) {
    if (fabs(q) < pivmin) q = -pivmin;
    q = (d[k] - x) - e[k - 1] * e[k - 1] / q;
    cnt += q < 0.0;
  }
  return cnt;
}

// First node u0 and node count of T's quadrature; false when T is not positive definite (or its
// eigenvalues span more than the node budget).
__host__ __device__ inline bool slq_quad_range(int l, const double* d, const double* e, double* u0, int* nodes) {
  *u0 = 0.0;
  *nodes = 0;
  if (l <= 0) return true;
  double hi = 0.0;
  for (int k = 0; k < l; ++k) {
    const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k + 1 < l ? fabs(e[k]) : 0.0);
    hi = k == 0 ? d[k] + r : fmax(hi, d[k] + r);
  }
  if (!(hi > 0.0) || tridiag_count_below(l, d, e, 0.0) > 0) return false;
  double lo = hi;
  for (int it = 0; it < 300 && tridiag_count_below(l, d, e, lo) > 0; ++it) lo *= 0.0625;
  if (!(lo > 0.0)) return false;
  *u0 = log(lo) - 40.0;
  const int n = (int)ceil((log(hi) + 40.0 - *u0) / kQuadStep) + 1;
  if (n > kQuadMaxNodes) return false;
  *nodes = n;
  return true;
}

// Integrand at node u: s / (1 + s) - s e1^T (T + s I)^{-1} e1, s = e^u (the factor s is ds / du).
__host__ __device__ inline double slq_quad_node(int l, const double* d, const double* e, double u) {
  const double s = exp(u);
  double D = d[l - 1] + s;
  for (int k = l - 2; k >= 0; --k) D = (d[k] + s) - e[k] * e[k] / D;
  return s / (1.0 + s) - s / D;
}

// One thread per column: the node range (u0[c], nodes[c]); a T that is not positive definite
// is counted in *bad.
static __global__ void slq_range_kernel(int t, int lmax, const double* __restrict__ Tdiag,
                                        const double* __restrict__ Toff, const int* __restrict__ iters,
                                        double* __restrict__ u0, int* __restrict__ nodes, int* __restrict__ bad) {
  const int c = blockIdx.x;
  if (c >= t || threadIdx.x != 0) return;
  const int l = min(iters[c], lmax);
  if (!slq_quad_range(l, Tdiag + (int64_t)c * lmax, Toff + (int64_t)c * lmax, &u0[c], &nodes[c])) {
    nodes[c] = 0;
    atomicAdd(bad, 1);
  }
}

// Block (x, c): nodes i = x * blockDim.x + threadIdx.x of column c, T_c staged in shared memory
// when it fits (staged != 0).
static __global__ void slq_node_kernel(int t, int lmax, const double* __restrict__ Tdiag,
                                       const double* __restrict__ Toff, const int* __restrict__ iters,
                                       const double* __restrict__ u0, const int* __restrict__ nodes,
                                       double* __restrict__ term, int staged) {
  extern __shared__ double vl_qsh[];
  const int c = blockIdx.y;
  if (c >= t || (int)(blockIdx.x * blockDim.x) >= nodes[c]) return;
  const int l = min(iters[c], lmax);
  const double* d = Tdiag + (int64_t)c * lmax;
  const double* e = Toff + (int64_t)c * lmax;
  if (staged) {
    for (int k = threadIdx.x; k < l; k += blockDim.x) {
      vl_qsh[k] = d[k];
      vl_qsh[lmax + k] = k + 1 < l ? e[k] : 0.0;
    }
    __syncthreads();
    d = vl_qsh;
    e = vl_qsh + lmax;
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nodes[c]) term[(int64_t)c * kQuadMaxNodes + i] = slq_quad_node(l, d, e, u0[c] + i * kQuadStep);
}

// gamma_c = w_c * h * sum_i term[c, i], in node order.
static __global__ void slq_sum_kernel(int t, const int* __restrict__ nodes, const double* __restrict__ w,
                                      const double* __restrict__ term, double* __restrict__ gamma) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= t) return;
  double g = 0.0;
  for (int i = 0; i < nodes[c]; ++i) g += term[(int64_t)c * kQuadMaxNodes + i];
  gamma[c] = w[c] * kQuadStep * g;
}

// ----------------------------------------------------------------------------- likelihood
// mu = F + b; g = d log p / d mu; W = -d^2 log p / d mu^2; logp; rhs = W b + g.
// lik_terms is host-callable for checks on the CPU.
// Gamma (shape a, rate a e^{-mu}), u = y e^{-mu}: log p = a log a - lgamma(a) + (a - 1) log y
// - a mu - a u, d log p / d mu = a (u - 1), W = a u.
__host__ __device__ __forceinline__ void lik_terms(int lik, double shape, double y, double mu, double& lp, double& g,
                                                   double& W) {
  if (lik == VL_LIK_GAMMA_LOG) {
    const double u = y * exp(-mu);
    g = shape * (u - 1.0);
    W = shape * u;
    lp = shape * log(shape) - lgamma(shape) + (shape - 1.0) * log(y) - shape * mu - shape * u;
  } else if (lik == VL_LIK_BERNOULLI_LOGIT) {
    const double p = 1.0 / (1.0 + exp(-mu));
    g = y - p;
    W = p * (1.0 - p);
    const double sp = fmax(mu, 0.0) + log1p(exp(-fabs(mu)));   // log(1 + e^mu)
    lp = y * mu - sp;
  } else {
    const double lam = exp(mu);
    g = y - lam;
    W = lam;
    lp = y * mu - lam - lgamma(y + 1.0);
  }
}

static __global__ void lik_kernel(int n, int lik, double shape, const double* __restrict__ y, const double* __restrict__ F,
                           const double* __restrict__ b, double* __restrict__ W, double* __restrict__ g,
                           double* __restrict__ rhs, double* __restrict__ logp) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    double lp, gg, ww;
    lik_terms(lik, shape, y[s], F[s] + b[s], lp, gg, ww);
    if (W) W[s] = ww;
    if (g) g[s] = gg;
    if (rhs) rhs[s] = ww * b[s] + gg;
    if (logp) logp[s] = lp;
  }
}

// ----------------------------------------------------------------------------- probes
// Rademacher r[s, j] = 1 - 2 * bit j of Philox4x64-10(counter = (p, j / 256, stream, 0),
// key = (seed, 0)), p = the caller index of storage row s; bit j % 256 is bit
// (j % 64) of output word (j % 256) / 64.
template <typename T>
__global__ void rademacher_kernel(int n, int t, int ld, const int32_t* __restrict__ s2u, uint64_t seed, int stream,
                                  int64_t idx_offset, T* __restrict__ R) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint64_t p = s2u ? (uint64_t)s2u[s] : (uint64_t)(s + idx_offset);
  for (int blk = 0; blk * 256 < ld; ++blk) {
    const Philox4 w = philox4x64_10(p, (uint64_t)blk, (uint64_t)stream, 0, seed, 0);
    for (int j = blk * 256; j < min(ld, blk * 256 + 256); ++j) {
      const int bit = j - blk * 256;
      const uint64_t v = (w.v[bit >> 6] >> (bit & 63)) & 1ULL;
      R[(int64_t)s * ld + j] = (j < t) ? (T)(1.0 - 2.0 * (double)v) : T(0);
    }
  }
}

// Gaussian z[s, j] by Box-Muller: block j / 4, words (2q, 2q + 1), q = (j % 4) / 2:
// u1 = ((w >> 11) + 1) 2^-53, u2 = (w >> 11) 2^-53, sqrt(-2 ln u1) cos / sin (2 pi u2).
// Fills columns j = col0 .. col0 + t - 1 into Z[s, j - col0]; padding columns get 0.
static __global__ void gaussian_kernel(int n, int t, int ld, int col0, const int32_t* __restrict__ s2u, uint64_t seed,
                                int stream, double* __restrict__ Z) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint64_t p = (uint64_t)s2u[s];
  const double two_m53 = 1.1102230246251565e-16;
  const double two_pi = 6.283185307179586;
  for (int k = t; k < ld; ++k) Z[(int64_t)s * ld + k] = 0.0;
  if (t <= 0) return;
  for (int blk = col0 / 4; blk <= (col0 + t - 1) / 4; ++blk) {
    const Philox4 w = philox4x64_10(p, (uint64_t)blk, (uint64_t)stream, 0, seed, 0);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const double u1 = ((double)(w.v[2 * q] >> 11) + 1.0) * two_m53;
      const double u2 = (double)(w.v[2 * q + 1] >> 11) * two_m53;
      const double rad = sqrt(-2.0 * log(u1));
      const double ang = two_pi * u2;
      const int j0 = blk * 4 + 2 * q;
      if (j0 >= col0 && j0 < col0 + t) Z[(int64_t)s * ld + (j0 - col0)] = rad * cos(ang);
      if (j0 + 1 >= col0 && j0 + 1 < col0 + t) Z[(int64_t)s * ld + (j0 + 1 - col0)] = rad * sin(ang);
    }
  }
}

}  // namespace vl
