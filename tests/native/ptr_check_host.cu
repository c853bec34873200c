// Host-side run of the library's pointer-placement rule (vl::device_memory_usable,
// csrc/vl_internal.h): which memory may be handed to kernels on the context's device.
// Reads lines "type device ctx_device" and prints 1 or 0. No GPU.
#include <cstdio>

#include "vl_internal.h"

int main() {
  int type, device, ctx;
  while (std::scanf("%d %d %d", &type, &device, &ctx) == 3)
    std::printf("%d\n", vl::device_memory_usable(type, device, ctx) ? 1 : 0);
  return 0;
}
