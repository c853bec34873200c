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
