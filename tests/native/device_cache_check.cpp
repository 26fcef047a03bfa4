// Host check of the per-device launch set-up cache (tfft_device_cache.h):
// each device id gets its own value, made once; ids outside the table are
// recomputed on every call; concurrent first calls make the value once.
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>

#include "tfft_device_cache.h"

extern "C" int check_device_cache() {
  tfft::PerDevice<int> cache;
  int made[tfft::kMaxDevices] = {};
  for (int rep = 0; rep < 3; ++rep)
    for (int dev = 0; dev < tfft::kMaxDevices; ++dev) {
      const int v = cache.get(dev, [&] {
        ++made[dev];
        return 1000 + dev;  // e.g. an SM count that differs per device
      });
      if (v != 1000 + dev) return 1;  // a value cached for another device
    }
  for (int dev = 0; dev < tfft::kMaxDevices; ++dev)
    if (made[dev] != 1) return 2;  // made more than once, or never
  int outside = 0;
  for (int rep = 0; rep < 3; ++rep) {
    if (cache.get(-1, [&] { ++outside; return 7; }) != 7) return 3;
    if (cache.get(tfft::kMaxDevices, [&] { ++outside; return 8; }) != 8) return 3;
  }
  if (outside != 6) return 4;  // out-of-range ids are not cached
  tfft::PerDevice<long> shared;
  std::atomic<int> calls{0};
  std::vector<std::thread> th;
  for (int t = 0; t < 8; ++t)
    th.emplace_back([&] {
      for (int i = 0; i < 1000; ++i) shared.get(3, [&] { calls.fetch_add(1); return 42L; });
    });
  for (auto& x : th) x.join();
  if (calls.load() != 1) return 5;  // concurrent first use made the value twice
  return 0;
}
