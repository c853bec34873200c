// Host check of the staged-product plan (build_halo_plan in tile_plan.h) for both directions:
// the blocks cover the rows in order, each holds at most rmax rows and reads at most ucap rows,
// its list is sorted and unique, and every row's own place and every dependency entry's place
// point at that row in the block's list. stdin: n m ucap rmax, then n*m neighbour storage
// indices (-1 padding). stdout: "fwd ok" / "bwd ok", or "fwd refused" when a row alone reads more
// than ucap rows, or a message naming the failure.
#include <cstdio>
#include <vector>

#include "tile_plan.h"

static bool check(const char* name, int n, int m, const int32_t* nbr, const int32_t* rp, const int32_t* col,
                  int ucap, int rmax) {
  const vl::HaloPlanHost P = vl::build_halo_plan(n, m, nbr, rp, col, ucap, rmax);
  if (!P.ok) {
    printf("%s refused\n", name);
    return true;
  }
  const int nb = (int)P.brow.size() - 1;
  if (P.brow[0] != 0 || P.brow[nb] != n || (int)P.uoff.size() != nb + 1) {
    printf("%s: blocks do not cover the rows\n", name);
    return false;
  }
  for (int b = 0; b < nb; ++b) {
    const int r0 = P.brow[b], r1 = P.brow[b + 1], u0 = P.uoff[b], U = P.uoff[b + 1] - u0;
    if (r1 <= r0 || r1 - r0 > rmax || U > ucap) {
      printf("%s: block %d out of bounds\n", name, b);
      return false;
    }
    for (int k = 1; k < U; ++k)
      if (P.ulist[u0 + k] <= P.ulist[u0 + k - 1]) {
        printf("%s: list of block %d not sorted and unique\n", name, b);
        return false;
      }
    for (int r = r0; r < r1; ++r) {
      if (P.lself[r] >= U || P.ulist[u0 + P.lself[r]] != r) {
        printf("%s: own place of row %d wrong\n", name, r);
        return false;
      }
      const long beg = rp ? rp[r] : (long)r * m, end = rp ? rp[r + 1] : (long)r * m + m;
      for (long e = beg; e < end; ++e) {
        const int j = rp ? col[e] : nbr[e];
        if (j < 0) continue;
        if (P.lidx[e] >= U || P.ulist[u0 + P.lidx[e]] != j) {
          printf("%s: place of entry %ld wrong\n", name, e);
          return false;
        }
      }
    }
  }
  printf("%s ok\n", name);
  return true;
}

int main() {
  int n, m, ucap, rmax;
  if (scanf("%d %d %d %d", &n, &m, &ucap, &rmax) != 4) return 2;
  std::vector<int32_t> nbr((size_t)n * m);
  for (auto& v : nbr)
    if (scanf("%d", &v) != 1) return 2;
  std::vector<int32_t> rp(n + 1, 0), col;
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < m; ++c)
      if (nbr[(size_t)i * m + c] >= 0) ++rp[nbr[(size_t)i * m + c] + 1];
  for (int s = 0; s < n; ++s) rp[s + 1] += rp[s];
  col.resize(rp[n] > 0 ? rp[n] : 1);
  std::vector<int32_t> fill(rp.begin(), rp.end() - 1);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < m; ++c)
      if (nbr[(size_t)i * m + c] >= 0) col[fill[nbr[(size_t)i * m + c]]++] = i;
  bool ok = check("fwd", n, m, nbr.data(), nullptr, nullptr, ucap, rmax);
  ok = check("bwd", n, m, nullptr, rp.data(), col.data(), ucap, rmax) && ok;
  return ok ? 0 : 1;
}
