// Dynamic shared-memory opt-in of a kernel instantiation, shared by every context and host
// thread of the process.
#pragma once
#include <cuda_runtime.h>

#include <atomic>

namespace homb {

constexpr int kAttrDevices = 64;   // device ordinals with a "done" flag; others set it every call

// Raise the dynamic shared-memory limit of `kernel` on the current device to the most it can
// have (the device's opt-in maximum less the kernel's static shared memory), once per
// device. Every caller sets the same value, so concurrent callers cannot lower the limit for
// one another, and a set flag is never stale. `done` is a zero-initialised static array of
// kAttrDevices flags, one array per instantiation. Returns cudaErrorInvalidValue when
// `bytes` exceeds that limit.
template <typename K>
inline cudaError_t smem_attr(K kernel, size_t bytes, std::atomic<int>* done) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool flagged = dev >= 0 && dev < kAttrDevices;
  if (flagged && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa{};
  e = cudaFuncGetAttributes(&fa, kernel);
  if (e != cudaSuccess) return e;
  const long long room = (long long)optin - (long long)fa.sharedSizeBytes;
  if (room < (long long)bytes) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
  if (e == cudaSuccess && flagged) done[dev].store(1, std::memory_order_release);
  return e;
}

}  // namespace homb
