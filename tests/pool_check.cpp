// Host check of the server's pool allocator (compiled and run by
// tests/test_pool_cpu.py).  Prints "ok" or the first failed condition.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "pgvimp_pool.h"

#define CHECK(c)                                          \
  do {                                                    \
    if (!(c)) {                                           \
      std::printf("failed line %d: %s\n", __LINE__, #c); \
      return 1;                                           \
    }                                                     \
  } while (0)

int main() {
  using pgv::RangeAllocator;
  RangeAllocator a;
  a.reset(4096);
  size_t o1, o2, o3, o4;
  CHECK(a.alloc(1, &o1) && o1 == 0);           // rounded up to one 256-byte granule
  CHECK(a.alloc(300, &o2) && o2 == 256);       // two granules
  CHECK(a.alloc(1024, &o3) && o3 == 768);
  CHECK(a.used() == 256 + 512 + 1024);
  CHECK(!a.alloc(4096, &o4));                  // larger than what is left
  a.release(o2, 300);                          // a hole of 512 between o1 and o3
  CHECK(a.free_ranges() == 2);
  CHECK(a.alloc(512, &o4) && o4 == 256);       // first fit reuses the hole
  a.release(o4, 512);
  a.release(o1, 1);                            // coalesces with the hole on its right
  CHECK(a.free_ranges() == 2 && a.largest_free() == 4096 - 1792);
  a.release(o3, 1024);                         // everything free again: one range
  CHECK(a.free_ranges() == 1 && a.largest_free() == 4096 && a.used() == 0);
  // random alloc / release never hands out overlapping ranges and ends whole
  std::srand(7);
  std::vector<std::pair<size_t, size_t>> live;
  a.reset(1 << 20);
  for (int it = 0; it < 20000; ++it) {
    if (live.empty() || std::rand() % 2) {
      size_t sz = 1 + std::rand() % 20000, off;
      if (a.alloc(sz, &off)) {
        size_t r = pgv::round_up(sz);
        for (auto& l : live) CHECK(off + r <= l.first || l.first + pgv::round_up(l.second) <= off);
        CHECK(off + r <= a.total());
        live.push_back({off, sz});
      }
    } else {
      size_t k = std::rand() % live.size();
      a.release(live[k].first, live[k].second);
      live.erase(live.begin() + k);
    }
  }
  for (auto& l : live) a.release(l.first, l.second);
  CHECK(a.used() == 0 && a.free_ranges() == 1 && a.largest_free() == a.total());
  std::printf("ok\n");
  return 0;
}
