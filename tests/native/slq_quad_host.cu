// Host-side run of the library's SLQ quadrature (csrc/kernels.cuh: e1^T log(T) e1 of a symmetric
// positive definite tridiagonal T as the trapezoidal sum, in u = log s, of
// s / (1 + s) - s e1^T (T + s I)^{-1} e1, each node by the bottom-up pivot recurrence), composed
// exactly as slq_range_kernel, slq_node_kernel and slq_sum_kernel take it. Reads cases from stdin
// as "l d_0 .. d_{l-1} e_0 .. e_{l-2}" and prints "value bad" per case. Host code only: no GPU.
#include <cstdio>
#include <vector>

#include "kernels.cuh"

int main() {
  int l;
  while (std::scanf("%d", &l) == 1) {
    std::vector<double> d(l > 0 ? l : 1), e(l > 0 ? l : 1, 0.0);
    for (int i = 0; i < l; ++i) std::scanf("%lf", &d[i]);
    for (int i = 0; i + 1 < l; ++i) std::scanf("%lf", &e[i]);
    double u0 = 0.0;
    int nodes = 0;
    const bool ok = vl::slq_quad_range(l, d.data(), e.data(), &u0, &nodes);
    std::vector<double> term(nodes > 0 ? nodes : 1);
    for (int i = 0; i < nodes; ++i) term[i] = vl::slq_quad_node(l, d.data(), e.data(), u0 + i * vl::kQuadStep);
    double g = 0.0;
    for (int i = 0; i < nodes; ++i) g += term[i];
    std::printf("%.17g %d\n", vl::kQuadStep * g, ok ? 0 : 1);
  }
  return 0;
}
