// Plan of the tiled triangular solves (sptrsv_tile1_kernel, sptrsv_tile_kernel): plain host
// C++ with no CUDA dependency, so that a host test can build plans and replay the walk.
//
// Tile b owns the storage rows [b R, min(n, (b + 1) R)), R = ceil(n / G); the storage order
// is the Morton order of the locations, so a tile is a compact patch of the domain and most
// dependencies of its rows lie inside it. The tile's rows are listed in task order (sorted by
// level). In the kernels the block's teams take the listed rows round robin, each team in list
// order, and a row waits only for its own dependencies: every dependency has a lower level and so
// an earlier place in its tile's list, which makes the walk free of deadlock whatever the number
// of teams (the unfinished row with the lowest (level, place) can always proceed).
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace vl {

struct TilePlanHost {
  int G = 0, R = 0;
  std::vector<int32_t> ttask;     // n - first: each tile's rows in task order, tiles in order
  std::vector<int32_t> toff;      // G + 1: tile b's rows are ttask[toff[b] .. toff[b + 1])
  std::vector<uint8_t> exported;  // n: 1 when a row of another tile depends on this row
};

// Dependencies of storage row s: ELL (nbr[s m .. s m + m), -1 padding) when rp is null, else
// CSR (col[rp[s] .. rp[s + 1])). task: storage rows sorted by level; the rows task[0 .. first)
// are solved before the walk (the leading levels, by another kernel) and are not listed.
inline TilePlanHost build_tile_plan(int n, int G, const int32_t* task, int m, const int32_t* nbr,
                                    const int32_t* rp, const int32_t* col, int first = 0) {
  TilePlanHost P;
  P.G = G;
  P.R = n > 0 ? (n + G - 1) / G : 1;
  const int R = P.R;
  P.toff.assign(G + 1, 0);
  for (int p = first; p < n; ++p) ++P.toff[task[p] / R + 1];
  for (int b = 0; b < G; ++b) P.toff[b + 1] += P.toff[b];
  P.ttask.resize(n - first);
  {
    std::vector<int32_t> fill(P.toff.begin(), P.toff.end() - 1);
    for (int p = first; p < n; ++p) P.ttask[fill[task[p] / R]++] = task[p];
  }
  P.exported.assign(n, 0);
  for (int s = 0; s < n; ++s) {
    const int beg = rp ? rp[s] : s * m, end = rp ? rp[s + 1] : s * m + m;
    for (int k = beg; k < end; ++k) {
      const int j = rp ? col[k] : nbr[k];
      if (j >= 0 && j / R != s / R) P.exported[j] = 1;
    }
  }
  return P;
}

}  // namespace vl

namespace vl {

// Plan of the staged products (spmv_B_staged_kernel, spmv_Bt_staged_kernel): consecutive storage
// rows are grouped into blocks, each with the sorted list of the rows it reads (its own rows and
// their dependencies), at most ucap of them and at most rmax rows per block. A block copies its
// list's rows into shared memory with independent coalesced loads and gathers from there, so the
// products stream instead of chasing one dependency at a time. lidx gives each dependency entry
// its place in its block's list (0xffff for a padding entry), lself each row's own place.
struct HaloPlanHost {
  std::vector<int32_t> brow;    // nb + 1
  std::vector<int32_t> uoff;    // nb + 1
  std::vector<int32_t> ulist;
  std::vector<uint16_t> lidx;   // one per dependency entry (ELL n * m, or CSR nnz)
  std::vector<uint16_t> lself;  // n
  bool ok = false;              // false: some row alone reads more than ucap rows
};

inline HaloPlanHost build_halo_plan(int n, int m, const int32_t* nbr, const int32_t* rp, const int32_t* col,
                                    int ucap, int rmax) {
  HaloPlanHost P;
  if (ucap < 2 || ucap > 65535) return P;
  const int64_t nent = rp ? (int64_t)rp[n] : (int64_t)n * m;
  P.lidx.assign(nent, 0xffff);
  P.lself.assign(n, 0);
  P.brow.push_back(0);
  P.uoff.push_back(0);
  std::vector<int32_t> mark(n, -1), cur;
  int nb = 0;
  auto deps = [&](int s, auto fn) {
    const int64_t beg = rp ? rp[s] : (int64_t)s * m, end = rp ? rp[s + 1] : (int64_t)s * m + m;
    for (int64_t k = beg; k < end; ++k) {
      const int j = rp ? col[k] : nbr[k];
      if (j >= 0) fn(j, k);
    }
  };
  int s = 0;
  while (s < n) {
    cur.clear();
    const int r0 = s;
    while (s < n && s - r0 < rmax) {
      int add = 0;
      if (mark[s] != nb) ++add;
      int extra = 0;
      deps(s, [&](int j, int64_t) {
        if (mark[j] != nb && j != s) ++extra;
      });
      // dependencies may repeat only across rows, never within one row
      if ((int)cur.size() + add + extra > ucap) {
        if (s == r0) return P;   // one row alone does not fit
        break;
      }
      if (mark[s] != nb) {
        mark[s] = nb;
        cur.push_back(s);
      }
      deps(s, [&](int j, int64_t) {
        if (mark[j] != nb) {
          mark[j] = nb;
          cur.push_back(j);
        }
      });
      ++s;
    }
    std::sort(cur.begin(), cur.end());
    for (size_t k = 0; k < cur.size(); ++k) mark[cur[k]] = -2 - (int32_t)k;   // place, encoded
    for (int r = r0; r < s; ++r) {
      P.lself[r] = (uint16_t)(-2 - mark[r]);
      deps(r, [&](int j, int64_t k) { P.lidx[k] = (uint16_t)(-2 - mark[j]); });
    }
    for (int32_t j : cur) mark[j] = -1;
    P.ulist.insert(P.ulist.end(), cur.begin(), cur.end());
    P.brow.push_back(s);
    P.uoff.push_back((int32_t)P.ulist.size());
    ++nb;
    // rows of later blocks must not see this block's marks
  }
  P.ok = true;
  return P;
}

}  // namespace vl
