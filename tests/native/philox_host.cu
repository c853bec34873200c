// Host-side run of the library's Philox4x64-10 (vl::philox4x64_10 in csrc/vl_device.cuh, the
// generator behind the probe and simulation kernels). Reads lines "c0 c1 c2 c3 k0 k1" from
// stdin and prints the four output words of each. Host code only: needs no GPU.
#include <cstdio>

#include "vl_device.cuh"

int main() {
  unsigned long long c[4], k[2];
  while (std::scanf("%llu %llu %llu %llu %llu %llu", &c[0], &c[1], &c[2], &c[3], &k[0], &k[1]) == 6) {
    const vl::Philox4 o = vl::philox4x64_10(c[0], c[1], c[2], c[3], k[0], k[1]);
    std::printf("%llu %llu %llu %llu\n", (unsigned long long)o.v[0], (unsigned long long)o.v[1],
                (unsigned long long)o.v[2], (unsigned long long)o.v[3]);
  }
  return 0;
}
