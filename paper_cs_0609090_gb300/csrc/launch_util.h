// launch_util.h -- host helpers shared by the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

namespace ldpc {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device, calling cudaFuncSetAttribute only when the limit must grow.
// Decoding calls can then be captured in a CUDA graph once the same request
// has run on the device before the capture (the attribute call is not a
// stream operation).
inline cudaError_t ensure_dynamic_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, int> done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  auto it = done[dev].find(kernel);
  if (it != done[dev].end() && it->second >= (int)bytes) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done[dev][kernel] = (int)bytes;
  return e;
}

}  // namespace ldpc
