// Host-side run of the library's SLQ quadrature (vl::tridiag_log_quad in csrc/kernels.cuh:
// e1^T log(T) e1 of a symmetric tridiagonal T by implicit-shift QR). Reads cases from stdin as
// "l d_0 .. d_{l-1} e_0 .. e_{l-2}" and prints "value bad" per case. Host code only: no GPU.
#include <cstdio>
#include <vector>

#include "kernels.cuh"

int main() {
  int l;
  while (std::scanf("%d", &l) == 1) {
    std::vector<double> d(l > 0 ? l : 1), e(l > 0 ? l : 1, 0.0), z(l > 0 ? l : 1);
    for (int i = 0; i < l; ++i) std::scanf("%lf", &d[i]);
    for (int i = 0; i + 1 < l; ++i) std::scanf("%lf", &e[i]);
    bool bad = false;
    const double g = vl::tridiag_log_quad(l, d.data(), e.data(), z.data(), &bad);
    std::printf("%.17g %d\n", g, bad ? 1 : 0);
  }
  return 0;
}
