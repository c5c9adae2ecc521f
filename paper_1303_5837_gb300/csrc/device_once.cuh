// device_once.cuh -- one-time, per-device host setup that is safe under
// concurrent callers (the solve server calls the library from several host
// threads, each on its own stream).  Kernel attributes such as the dynamic
// shared-memory limit belong to a device, so each device is set up once.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

namespace cagb {

constexpr int kMaxDevices = 64;

inline std::mutex &device_setup_mutex() {
  static std::mutex mu;
  return mu;
}

// Runs fn() (returning cudaError_t) once per device for the call site that
// owns `done` (one bit per device).  A failed setup is not recorded, so the
// next call tries again.  Devices beyond kMaxDevices run fn() every time.
template <class F>
cudaError_t once_per_device(std::atomic<unsigned long long> &done, F &&fn) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return fn();
  const unsigned long long bit = 1ull << dev;
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  std::lock_guard<std::mutex> g(device_setup_mutex());
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = fn();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

// Number of SMs of the current device (cached per device).
inline cudaError_t device_sm_count(int *sms) {
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices) {
    const int v = cache[dev].load(std::memory_order_acquire);
    if (v > 0) {
      *sms = v;
      return cudaSuccess;
    }
  }
  int v = 0;
  if ((e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (v < 1) v = 1;
  if (dev >= 0 && dev < kMaxDevices) cache[dev].store(v, std::memory_order_release);
  *sms = v;
  return cudaSuccess;
}

}  // namespace cagb
