// Host-side run of the library's per-point likelihood terms (vl::lik_terms, csrc/kernels.cuh)
// and covariance function (vl::cov_eval, csrc/vl_device.cuh). Reads lines
// "L lik shape y mu" (prints "logp grad W") or "C cov h sigma2 rho" (prints "c(h)"). No GPU.
#include <cstdio>

#include "kernels.cuh"

int main() {
  char kind;
  while (std::scanf(" %c", &kind) == 1) {
    if (kind == 'L') {
      int lik;
      double shape, y, mu, lp, g, W;
      if (std::scanf("%d %lf %lf %lf", &lik, &shape, &y, &mu) != 4) return 1;
      vl::lik_terms(lik, shape, y, mu, lp, g, W);
      std::printf("%.17g %.17g %.17g\n", lp, g, W);
    } else {
      int cov;
      double h, s2, rho;
      if (std::scanf("%d %lf %lf %lf", &cov, &h, &s2, &rho) != 4) return 1;
      std::printf("%.17g\n", vl::cov_eval(h, cov, s2, rho));
    }
  }
  return 0;
}
