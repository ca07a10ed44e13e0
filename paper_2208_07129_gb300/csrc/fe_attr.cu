// Per-device, thread-safe cache of the dynamic shared-memory attribute of the
// cell kernels (cudaFuncAttributeMaxDynamicSharedMemorySize).
#include <map>
#include <mutex>
#include <utility>

#include "fe_internal.h"

namespace fe {

cudaError_t ensure_dyn_smem(const void* kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> set;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = set[{kern, dev}];
  if (have >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

}  // namespace fe
