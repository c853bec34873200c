// Randomised check of the workspace arena (vl::Arena, a first-fit sub-allocator over one
// buffer), linked against libvl. Host code only: the "buffer" is a plain address range and
// is never dereferenced. Checks after every operation: live blocks never overlap and stay
// inside the buffer, offsets are 256-byte aligned, in_use equals the sum of live sizes, peak
// is the running maximum, and releasing everything coalesces the free space so that one
// allocation of the whole buffer succeeds again. Prints "ok" and returns 0 on success.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <random>

#include "vl_internal.h"

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s %lld %lld\n", what, a, b);
  return 1;
}

int main(int argc, char** argv) {
  const unsigned seed = argc > 1 ? (unsigned)std::atoi(argv[1]) : 1u;
  std::mt19937_64 rng(seed);
  const size_t size = (size_t)64 << 20;
  char* base = reinterpret_cast<char*>((uintptr_t)1 << 40);   // never dereferenced
  vl::Arena a;
  a.init(base, size);
  std::map<size_t, size_t> live;   // offset -> requested bytes
  size_t in_use = 0, peak = 0;
  for (int step = 0; step < 200000; ++step) {
    const bool do_alloc = live.empty() || (rng() % 100) < 55;
    if (do_alloc) {
      size_t req = (rng() % 4 == 0) ? (size_t)(rng() % 64) : (size_t)(rng() % (1 << 20));
      void* p = a.alloc(req);
      const size_t rounded = ((req ? req : 1) + 255) / 256 * 256;
      if (!p) {
        // first fit may fail only when no free hole is large enough: check the claim
        size_t prev_end = 0, biggest = 0;
        for (auto& kv : live) {
          size_t rs = ((kv.second ? kv.second : 1) + 255) / 256 * 256;
          if (kv.first > prev_end) biggest = std::max(biggest, kv.first - prev_end);
          prev_end = kv.first + rs;
        }
        biggest = std::max(biggest, size - prev_end);
        if (biggest >= rounded) return fail("spurious exhaustion", (long long)biggest, (long long)rounded);
        continue;
      }
      const size_t off = (size_t)(static_cast<char*>(p) - base);
      if (off % 256) return fail("misaligned", (long long)off, 0);
      if (off + rounded > size) return fail("out of range", (long long)off, (long long)rounded);
      auto nx = live.lower_bound(off);
      if (nx != live.end() && off + rounded > nx->first) return fail("overlap next", (long long)off, (long long)nx->first);
      if (nx != live.begin()) {
        auto pv = std::prev(nx);
        size_t rs = ((pv->second ? pv->second : 1) + 255) / 256 * 256;
        if (pv->first + rs > off) return fail("overlap prev", (long long)pv->first, (long long)off);
      }
      live[off] = req;
      in_use += rounded;
      peak = std::max(peak, in_use);
    } else {
      auto it = live.begin();
      std::advance(it, (long)(rng() % live.size()));
      a.release(base + it->first);
      in_use -= ((it->second ? it->second : 1) + 255) / 256 * 256;
      live.erase(it);
    }
    if (a.in_use() != in_use) return fail("in_use", (long long)a.in_use(), (long long)in_use);
    if (a.peak() != peak) return fail("peak", (long long)a.peak(), (long long)peak);
  }
  a.release(nullptr);                       // no-op
  a.release(base + 12345);                  // not a block: ignored
  for (auto& kv : live) a.release(base + kv.first);
  if (a.in_use() != 0) return fail("in_use after release", (long long)a.in_use(), 0);
  void* all = a.alloc(size);
  if (all != base) return fail("not coalesced", (long long)(static_cast<char*>(all) - base), 0);
  if (a.alloc(1) != nullptr) return fail("allocation beyond the buffer", 0, 0);
  std::printf("ok\n");
  return 0;
}
