// Per-device, thread-safe cache of the dynamic shared-memory attribute of the
// cell kernels (cudaFuncAttributeMaxDynamicSharedMemorySize), and the
// per-thread record of the last CUDA runtime error behind a status.
#include <cstdio>
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

namespace {
thread_local cudaError_t last_cuda_error = cudaSuccess;
thread_local const char* last_cuda_where = nullptr;
thread_local char last_cuda_text[160];
}

fe_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return FE_OK;
  last_cuda_error = e;
  last_cuda_where = where;
  return e == cudaErrorMemoryAllocation ? FE_ENOMEM : FE_ECUDA;
}

}  // namespace fe

extern "C" const char* fe_last_cuda_error(void) {
  if (fe::last_cuda_error == cudaSuccess) return "none";
  if (!fe::last_cuda_where) return cudaGetErrorName(fe::last_cuda_error);
  std::snprintf(fe::last_cuda_text, sizeof(fe::last_cuda_text), "%s in %s", cudaGetErrorName(fe::last_cuda_error),
                fe::last_cuda_where);
  return fe::last_cuda_text;
}
