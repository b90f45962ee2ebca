// cg_setup.h -- per-device launch setup of a kernel (host code).
//
// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) applies to the current
// device only, and the resident CTAs per SM are a property of the device,
// so both are kept per device index, each filled once under a once-flag on
// the first launch on that device (safe when host threads launch at once).
#pragma once
#include <cuda_runtime.h>

#include <mutex>

namespace cgi {

constexpr int kSetupMaxDevices = 64;

struct KernelSetup {
  std::once_flag once[kSetupMaxDevices];
  cudaError_t err[kSetupMaxDevices];
  int per_sm[kSetupMaxDevices];
};

// On the current device: opt `kernel` in to `smem` bytes of dynamic shared
// memory (above the 48 KiB default) and find how many CTAs of `threads`
// threads fit on one SM (at least 1).  Returns the opt-in's error, which is
// kept: a later launch on the same device gets it again.
template <typename K>
cudaError_t kernel_setup(KernelSetup &s, K kernel, int threads, size_t smem, int *per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kSetupMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(s.once[dev], [&] {
    cudaError_t r = cudaSuccess;
    if (smem > 48 * 1024) {
      r = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (r != cudaSuccess) cudaGetLastError();
    }
    int n = 0;
    if (r == cudaSuccess &&
        (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess ||
         n < 1)) {
      cudaGetLastError();
      n = 1;
    }
    s.err[dev] = r;
    s.per_sm[dev] = n > 0 ? n : 1;
  });
  *per_sm = s.per_sm[dev];
  return s.err[dev];
}

}  // namespace cgi
