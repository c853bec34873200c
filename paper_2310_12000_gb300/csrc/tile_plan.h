// Plan of the tiled triangular solves (sptrsv_tile1_kernel, sptrsv_tile_kernel): plain host
// C++ with no CUDA dependency, so that a host test can build plans and replay the walk.
//
// Tile b owns the storage rows [b R, min(n, (b + 1) R)), R = ceil(n / G). Its rows are listed
// in task order (the task list is sorted by level), and each run of one level is a segment.
// Before segment k the tile waits until every other tile B that a row of the segment depends on
// has published progress >= need (one more than the highest level of those dependencies in B);
// a wait is dropped when an earlier segment of the same tile already waited for as much.
#pragma once

#include <algorithm>
#include <cstdint>
#include <vector>

namespace vl {

struct TilePlanHost {
  int G = 0, R = 0;
  std::vector<int32_t> ttask;     // n: each tile's rows in task order, tiles in order
  std::vector<int32_t> sp;        // G + 1: segments of tile b are [sp[b], sp[b + 1])
  std::vector<int32_t> seg_lev;   // level of each segment
  std::vector<int32_t> seg_beg;   // nseg + 1: ttask range of each segment (last entry n)
  std::vector<int32_t> wptr;      // nseg + 1: waits of each segment
  std::vector<int32_t> wtile, wneed;
};

// Dependencies of storage row s: ELL (nbr[s m .. s m + m), -1 padding) when rp is null, else
// CSR (col[rp[s] .. rp[s + 1])). lptr: first task of each level (nlev + 1 entries).
inline TilePlanHost build_tile_plan(int n, int G, const int32_t* task, const int32_t* lptr, int nlev, int m,
                                    const int32_t* nbr, const int32_t* rp, const int32_t* col) {
  TilePlanHost P;
  P.G = G;
  P.R = n > 0 ? (n + G - 1) / G : 1;
  const int R = P.R;
  std::vector<int32_t> lev(n);
  for (int l = 0; l < nlev; ++l)
    for (int p = lptr[l]; p < lptr[l + 1]; ++p) lev[task[p]] = l;
  std::vector<int32_t> toff(G + 1, 0);
  for (int p = 0; p < n; ++p) ++toff[task[p] / R + 1];
  for (int b = 0; b < G; ++b) toff[b + 1] += toff[b];
  P.ttask.resize(n);
  {
    std::vector<int32_t> fill(toff.begin(), toff.end() - 1);
    for (int p = 0; p < n; ++p) P.ttask[fill[task[p] / R]++] = task[p];
  }
  P.sp.assign(G + 1, 0);
  P.wptr.assign(1, 0);
  std::vector<int32_t> waited(G, 0), cur(G, 0), touched;
  for (int b = 0; b < G; ++b) {
    P.sp[b] = (int32_t)P.seg_lev.size();
    std::fill(waited.begin(), waited.end(), 0);
    for (int p = toff[b]; p < toff[b + 1];) {
      const int l = lev[P.ttask[p]];
      int e = p;
      while (e < toff[b + 1] && lev[P.ttask[e]] == l) ++e;
      P.seg_lev.push_back(l);
      P.seg_beg.push_back(p);
      for (int q = p; q < e; ++q) {
        const int s = P.ttask[q];
        const int beg = rp ? rp[s] : s * m, end = rp ? rp[s + 1] : s * m + m;
        for (int k = beg; k < end; ++k) {
          const int j = rp ? col[k] : nbr[k];
          if (j < 0) continue;
          const int B = j / R;
          if (B == b) continue;
          if (cur[B] == 0) touched.push_back(B);
          cur[B] = std::max(cur[B], lev[j] + 1);
        }
      }
      std::sort(touched.begin(), touched.end());
      for (int B : touched) {
        if (cur[B] > waited[B]) {
          P.wtile.push_back(B);
          P.wneed.push_back(cur[B]);
          waited[B] = cur[B];
        }
        cur[B] = 0;
      }
      touched.clear();
      P.wptr.push_back((int32_t)P.wtile.size());
      p = e;
    }
  }
  P.sp[G] = (int32_t)P.seg_lev.size();
  P.seg_beg.push_back(n);
  return P;
}

}  // namespace vl
