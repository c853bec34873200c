// Host replay of the tiled triangular solves: builds the plans of tile_plan.h for both
// directions, checks that every cross-tile dependency is covered by a wait of its segment or an
// earlier one, and replays the walk with the tiles advancing in a random interleaving under
// the kernels' rules (a tile runs its next segment once every wait of that segment is met, then
// publishes the level of its following segment). Every dependency must be solved when it is
// read, the walk must never stall, and x must equal the sequential substitution.
// stdin: n m G seed, then n*m neighbour storage indices (-1 padding).
// stdout: "fwd ok" / "bwd ok" lines (or a message naming the failure).
#include <cstdio>
#include <random>
#include <vector>

#include "tile_plan.h"

using vl::TilePlanHost;

static bool replay(const char* name, int n, int G, int nlev, const std::vector<int32_t>& task,
                   const std::vector<int32_t>& lptr, const std::vector<int32_t>& lev, int m,
                   const std::vector<int32_t>& nbr, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                   const std::vector<double>& w, const std::vector<double>& rhs, unsigned seed) {
  const bool ell = rp.empty();
  TilePlanHost P = vl::build_tile_plan(n, G, task.data(), lptr.data(), nlev, m, ell ? nbr.data() : nullptr,
                                       ell ? nullptr : rp.data(), ell ? nullptr : col.data());
  auto deps = [&](int s, auto fn) {
    const int beg = ell ? s * m : rp[s], end = ell ? s * m + m : rp[s + 1];
    for (int k = beg; k < end; ++k) {
      const int j = ell ? nbr[k] : col[k];
      if (j >= 0) fn(j, k);
    }
  };
  // sequential substitution in task order
  std::vector<double> xref(n, 0.0);
  for (int p = 0; p < n; ++p) {
    const int s = task[p];
    double acc = 0.0;
    deps(s, [&](int j, int k) { acc += w[k] * xref[j]; });
    xref[s] = rhs[s] + acc;
  }
  // coverage: a cross-tile dependency of a row in segment k is waited for by segment k or earlier
  const int R = P.R;
  for (int b = 0; b < G; ++b) {
    std::vector<int> waited(G, 0);
    for (int k = P.sp[b]; k < P.sp[b + 1]; ++k) {
      for (int w_ = P.wptr[k]; w_ < P.wptr[k + 1]; ++w_) waited[P.wtile[w_]] = std::max(waited[P.wtile[w_]], P.wneed[w_]);
      for (int p = P.seg_beg[k]; p < P.seg_beg[k + 1]; ++p) {
        const int s = P.ttask[p];
        if (s / R != b || lev[s] != P.seg_lev[k]) {
          printf("%s: row %d misplaced\n", name, s);
          return false;
        }
        bool ok = true;
        deps(s, [&](int j, int) {
          if (lev[j] >= lev[s]) ok = false;
          if (j / R != b && waited[j / R] < lev[j] + 1) ok = false;
        });
        if (!ok) {
          printf("%s: dependency of row %d not covered\n", name, s);
          return false;
        }
      }
    }
  }
  // replay in a random interleaving
  std::mt19937 rng(seed);
  std::vector<int> prog(G, 0), next(G);
  for (int b = 0; b < G; ++b) next[b] = P.sp[b];
  std::vector<char> done(n, 0);
  std::vector<double> x(n, 0.0);
  int left = 0;
  for (int b = 0; b < G; ++b) left += P.sp[b] < P.sp[b + 1];
  std::vector<int> order(G);
  for (int b = 0; b < G; ++b) order[b] = b;
  while (left > 0) {
    std::shuffle(order.begin(), order.end(), rng);
    bool moved = false;
    for (int b : order) {
      const int k = next[b];
      if (k >= P.sp[b + 1]) continue;
      bool ready = true;
      for (int w_ = P.wptr[k]; w_ < P.wptr[k + 1]; ++w_) ready = ready && prog[P.wtile[w_]] >= P.wneed[w_];
      if (!ready) continue;
      for (int p = P.seg_beg[k]; p < P.seg_beg[k + 1]; ++p) {
        const int s = P.ttask[p];
        double acc = 0.0;
        bool ok = true;
        deps(s, [&](int j, int kk) {
          ok = ok && done[j];
          acc += w[kk] * x[j];
        });
        if (!ok) {
          printf("%s: row %d read an unsolved dependency\n", name, s);
          return false;
        }
        x[s] = rhs[s] + acc;
      }
      for (int p = P.seg_beg[k]; p < P.seg_beg[k + 1]; ++p) done[P.ttask[p]] = 1;
      prog[b] = k + 1 < P.sp[b + 1] ? P.seg_lev[k + 1] : 0x7fffffff;
      next[b] = k + 1;
      if (next[b] >= P.sp[b + 1]) --left;
      moved = true;
    }
    if (!moved) {
      printf("%s: the walk stalled with %d tiles left\n", name, left);
      return false;
    }
  }
  for (int s = 0; s < n; ++s)
    if (!done[s] || x[s] != xref[s]) {
      printf("%s: row %d differs from the sequential substitution\n", name, s);
      return false;
    }
  printf("%s ok\n", name);
  return true;
}

int main() {
  int n, m, G;
  unsigned seed;
  if (scanf("%d %d %d %u", &n, &m, &G, &seed) != 4) return 2;
  std::vector<int32_t> nbr((size_t)n * m);
  for (auto& v : nbr)
    if (scanf("%d", &v) != 1) return 2;
  // forward levels (longest path over the ELL dependencies) and task list sorted by (level, row)
  auto levels = [&](auto deps_of, std::vector<int32_t>& lev, std::vector<int32_t>& task, std::vector<int32_t>& lptr,
                    const std::vector<int32_t>& topo) {
    lev.assign(n, 0);
    int nlev = 0;
    for (int s : topo) {
      int l = 0;
      deps_of(s, [&](int j) { l = std::max(l, lev[j] + 1); });
      lev[s] = l;
      nlev = std::max(nlev, l + 1);
    }
    lptr.assign(nlev + 1, 0);
    for (int s = 0; s < n; ++s) ++lptr[lev[s] + 1];
    for (int l = 0; l < nlev; ++l) lptr[l + 1] += lptr[l];
    std::vector<int32_t> fill(lptr.begin(), lptr.end() - 1);
    task.assign(n, 0);
    for (int s = 0; s < n; ++s) task[fill[lev[s]]++] = s;
    return nlev;
  };
  // a topological order of the forward DAG: rows by their depth-first finishing order
  std::vector<int32_t> topo_f, state(n, 0);
  for (int s0 = 0; s0 < n; ++s0) {
    if (state[s0]) continue;
    std::vector<std::pair<int, int>> st{{s0, 0}};
    state[s0] = 1;
    while (!st.empty()) {
      auto& [s, c] = st.back();
      if (c < m) {
        const int j = nbr[(size_t)s * m + c++];
        if (j >= 0 && !state[j]) {
          state[j] = 1;
          st.push_back({j, 0});
        }
      } else {
        topo_f.push_back(s);
        st.pop_back();
      }
    }
  }
  std::vector<int32_t> levf, taskf, lptrf, levb, taskb, lptrb;
  const int nlevf = levels([&](int s, auto fn) {
    for (int c = 0; c < m; ++c)
      if (nbr[(size_t)s * m + c] >= 0) fn(nbr[(size_t)s * m + c]);
  }, levf, taskf, lptrf, topo_f);
  // transpose (row j lists the rows i with j in N(i)) for the backward solve
  std::vector<int32_t> rp(n + 1, 0), col;
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < m; ++c)
      if (nbr[(size_t)i * m + c] >= 0) ++rp[nbr[(size_t)i * m + c] + 1];
  for (int s = 0; s < n; ++s) rp[s + 1] += rp[s];
  col.resize(std::max(rp[n], 1));
  {
    std::vector<int32_t> fill(rp.begin(), rp.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < m; ++c)
        if (nbr[(size_t)i * m + c] >= 0) col[fill[nbr[(size_t)i * m + c]]++] = i;
  }
  std::vector<int32_t> topo_b(topo_f.rbegin(), topo_f.rend());
  const int nlevb = levels([&](int s, auto fn) {
    for (int k = rp[s]; k < rp[s + 1]; ++k) fn(col[k]);
  }, levb, taskb, lptrb, topo_b);
  std::mt19937 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::vector<double> wf((size_t)n * m), wb(std::max(rp[n], 1)), rhs(n);
  for (auto& v : wf) v = U(rng);
  for (auto& v : wb) v = U(rng);
  for (auto& v : rhs) v = U(rng);
  bool ok = replay("fwd", n, G, nlevf, taskf, lptrf, levf, m, nbr, {}, {}, wf, rhs, seed + 1);
  ok = replay("bwd", n, G, nlevb, taskb, lptrb, levb, m, nbr, rp, col, wb, rhs, seed + 2) && ok;
  return ok ? 0 : 1;
}
