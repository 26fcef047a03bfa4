// Per-device caches of launch set-up.
//
// A kernel's maximum dynamic shared memory (cudaFuncSetAttribute) is set on
// the current device only, and occupancy and SM counts are properties of a
// device, so a process that binds plans on several GPUs must keep one value
// per device id: a value cached for the first device would leave the second
// device's large-shared-memory kernels without their attribute (the launch
// then fails) or size its persistent grids for the wrong SM count.
//
// Plain C++ (no CUDA headers), so the host tests can exercise the keying.
#pragma once

#include <atomic>
#include <mutex>

namespace tfft {

constexpr int kMaxDevices = 64;

// One value per device id, made by `make()` the first time that device asks
// (thread-safe; `make` runs at most once per device).  Ids outside
// [0, kMaxDevices) are not cached: `make()` runs on every call.
template <class T>
class PerDevice {
 public:
  template <class F>
  T get(int dev, F&& make) {
    if (dev < 0 || dev >= kMaxDevices) return make();
    if (ready_[dev].load(std::memory_order_acquire)) return val_[dev];
    std::lock_guard<std::mutex> lock(mutex_);
    if (!ready_[dev].load(std::memory_order_relaxed)) {
      val_[dev] = make();
      ready_[dev].store(true, std::memory_order_release);
    }
    return val_[dev];
  }

 private:
  std::mutex mutex_;
  std::atomic<bool> ready_[kMaxDevices] = {};
  T val_[kMaxDevices] = {};
};

}  // namespace tfft
