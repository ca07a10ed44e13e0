// fe_apply_host without any device allocation.
//
// fe_apply_host stages the host blocks in device memory that it allocates
// with cudaMalloc (and keeps in the context).  Some callers cannot allow a
// library to allocate device memory: a process whose memory manager has
// reserved the whole device up front, a real-time loop that must never block
// in the allocator, or an application with a strict, pre-measured memory
// budget.  For them this variant stages through one fixed, file-scope device
// array instead.  The array is `static __device__`, so every GPU that loads
// the library holds its kFeNoAllocStageBytes until the process exits.
//
// In host code the array's name stands for a host-side shadow, not for device
// memory; its device address is obtained once per device with
// cudaGetSymbolAddress (with that device current) and cached here.
//
// On a refined mesh with hanging nodes the product first writes a copy of X
// with the slave rows filled in; that block comes from the same array, so
// such a call needs room for three blocks instead of two.
#include <mutex>

#include "fe_internal.h"

namespace {

constexpr size_t kFeNoAllocStageBytes = FE_NOALLOC_STAGE_BYTES;   // X and Y staging together
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_stage[kFeNoAllocStageBytes];

std::mutex g_mu;
void* g_stage_ptr[kMaxDevices] = {};

// Device address of g_stage on the current device (looked up once per device).
cudaError_t stage_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_stage_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_stage);
    if (e != cudaSuccess) return e;
    g_stage_ptr[dev] = p;
  }
  *out = g_stage_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" size_t fe_noalloc_stage_bytes(void) { return kFeNoAllocStageBytes; }

extern "C" fe_status fe_apply_host_noalloc(fe_ctx* c, const void* Xh, void* Yh, int n_vec, void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!Xh || !Yh) return FE_EINVAL;
  // refuse what fe_apply would refuse before any copy is queued
  if (c->refined && c->mode != FE_FP64 && c->mode != FE_DF64 && c->mode != FE_FP32) return FE_EUNSUPPORTED;
  const size_t elem =
      (c->mode == FE_FP64 || c->mode == FE_DF64) ? sizeof(double) : c->mode == FE_BF16S ? (size_t)2 : sizeof(float);
  const size_t bytes = c->n_dofs * (size_t)n_vec * elem;
  // X, Y and (on a refined mesh with hanging nodes) the distribute step's copy
  // of X with the slave rows filled in, each block at a 256-byte boundary
  const size_t slot = (bytes + 255) / 256 * 256;
  const int blocks = (c->refined && c->n_slaves > 0) ? 3 : 2;
  if ((size_t)(blocks - 1) * slot + bytes > kFeNoAllocStageBytes) return FE_EINVAL;
  void* base = nullptr;
  cudaError_t e = stage_address(&base);
  if (e != cudaSuccess) return FE_ECUDA;
  char* dX = static_cast<char*>(base);
  char* dY = dX + slot;
  char* dXc = blocks == 3 ? dX + 2 * slot : nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  e = cudaMemcpyAsync(dX, Xh, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    return FE_ECUDA;
  }
  fe_status st;
  if (c->refined) {
    e = fe::apply_refined(c, dX, dY, n_vec, s, dXc);
    st = e == cudaSuccess ? FE_OK : FE_ECUDA;
  } else {
    st = fe_apply(c, dX, dY, n_vec, stream);
  }
  if (st != FE_OK) {
    // the copy of the caller's X may still be in flight: let it finish before
    // the caller reuses the buffer or another call touches the array
    cudaStreamSynchronize(s);
    return st;
  }
  e = cudaMemcpyAsync(Yh, dY, bytes, cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  return (e == cudaSuccess && e2 == cudaSuccess) ? FE_OK : FE_ECUDA;
}
