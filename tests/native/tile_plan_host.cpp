// Host replay of the tiled triangular solves: builds the plans of tile_plan.h for both
// directions, checks the tile lists (every row in its own tile, in task order) and the marks of
// the rows other tiles depend on, and replays the walk under the kernels' rule (each tile's
// teams take its rows round robin, each team in list order, a row runs once its dependencies
// are solved) with the teams advancing in a random interleaving, for 1, 3 and 64 teams per
// tile. The walk must never stall and x must equal the sequential substitution.
// stdin: n m G seed, then n*m neighbour storage indices (-1 padding).
// stdout: one "fwd ok" / "bwd ok" line per team count (or a message naming the failure).
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>

#include "tile_plan.h"

using vl::TilePlanHost;

static bool replay(const char* name, int n, int G, int teams, const std::vector<int32_t>& task, int m,
                   const std::vector<int32_t>& nbr, const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                   const std::vector<double>& w, const std::vector<double>& rhs, unsigned seed, int first) {
  const bool ell = rp.empty();
  TilePlanHost P = vl::build_tile_plan(n, G, task.data(), m, ell ? nbr.data() : nullptr, ell ? nullptr : rp.data(),
                                       ell ? nullptr : col.data(), first);
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
  // every row in its own tile, each tile's rows in task order, and the exported marks exact
  const int R = P.R;
  std::vector<int> pos(n, -1);
  for (int p = 0; p < n; ++p) pos[task[p]] = p;
  std::vector<uint8_t> ex(n, 0);
  for (int s = 0; s < n; ++s) deps(s, [&](int j, int) { if (j / R != s / R) ex[j] = 1; });
  if (ex != P.exported) {
    printf("%s: exported marks differ\n", name);
    return false;
  }
  if ((int)P.ttask.size() != n - first || P.toff[G] != n - first) {
    printf("%s: the tile lists do not hold the rows after the first %d\n", name, first);
    return false;
  }
  for (int b = 0; b < G; ++b)
    for (int p = P.toff[b]; p < P.toff[b + 1]; ++p)
      if (P.ttask[p] / R != b || pos[P.ttask[p]] < first ||
          (p > P.toff[b] && pos[P.ttask[p]] < pos[P.ttask[p - 1]])) {
        printf("%s: tile list of tile %d out of order\n", name, b);
        return false;
      }
  // replay: `teams` teams per tile take the tile's rows round robin, each in list order; a team
  // runs its next row once every dependency of that row is solved
  std::mt19937 rng(seed);
  std::vector<std::pair<int, int>> cursor;   // (tile, team) -> next place
  std::vector<int> next;
  for (int b = 0; b < G; ++b)
    for (int tm = 0; tm < teams; ++tm) {
      cursor.push_back({b, tm});
      next.push_back(P.toff[b] + tm);
    }
  std::vector<char> done(n, 0);
  std::vector<double> x(n, 0.0);
  for (int p = 0; p < first; ++p) {   // solved before the walk, in task order
    const int s = task[p];
    double acc = 0.0;
    deps(s, [&](int j, int k) { acc += w[k] * x[j]; });
    x[s] = rhs[s] + acc;
    done[s] = 1;
  }
  int left = n - first;
  std::vector<int> order(cursor.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  while (left > 0) {
    std::shuffle(order.begin(), order.end(), rng);
    bool moved = false;
    for (int i : order) {
      const int b = cursor[i].first;
      int& p = next[i];
      while (p < P.toff[b + 1]) {
        const int s = P.ttask[p];
        bool ready = true;
        deps(s, [&](int j, int) { ready = ready && done[j]; });
        if (!ready) break;
        double acc = 0.0;
        deps(s, [&](int j, int k) { acc += w[k] * x[j]; });
        x[s] = rhs[s] + acc;
        done[s] = 1;
        --left;
        p += teams;
        moved = true;
        if (rng() % 3 == 0) break;   // let other teams interleave
      }
    }
    if (!moved) {
      printf("%s: the walk stalled with %d rows left\n", name, left);
      return false;
    }
  }
  for (int s = 0; s < n; ++s)
    if (x[s] != xref[s]) {
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
  (void)nlevb;
  bool ok = true;
  for (int teams : {1, 3, 64}) {
    // forward: also with the rows of the first levels solved before the walk
    const int first = teams == 3 ? lptrf[std::min(nlevf, 6)] : 0;
    ok = replay("fwd", n, G, teams, taskf, m, nbr, {}, {}, wf, rhs, seed + teams, first) && ok;
    ok = replay("bwd", n, G, teams, taskb, m, nbr, rp, col, wb, rhs, seed + 2 * teams, 0) && ok;
  }
  return ok ? 0 : 1;
}
