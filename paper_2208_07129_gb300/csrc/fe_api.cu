// C ABI of libfe: apply, host-buffer apply, diagonal, status.
#include <cstring>

#include "fe_internal.h"

using namespace fe;

namespace {
fe_status from_cuda(cudaError_t e) {
  return e == cudaSuccess ? FE_OK : (e == cudaErrorMemoryAllocation ? FE_ENOMEM : FE_ECUDA);
}
size_t elem_size(fe_mode m) { return m == FE_FP64 ? sizeof(double) : sizeof(float); }

bool overlaps(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}
}  // namespace

extern "C" fe_status fe_apply(fe_ctx* c, const void* X, void* Y, int n_vec, void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!X || !Y) return FE_EINVAL;
  const size_t bytes = c->n_dofs * (size_t)n_vec * elem_size(c->mode);
  if (overlaps(X, Y, bytes)) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (c->mode) {
    case FE_FP64: e = apply_cc_f64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, s); break;
    case FE_FP32: e = apply_cc_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, s); break;
    case FE_TF32:
    case FE_BF16:
      if ((size_t)3 * c->nq * c->nq * c->nq * 16 * sizeof(float) > 220 * 1024) return FE_EUNSUPPORTED;
      e = apply_mma_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, s, c->mode == FE_BF16);
      break;
    default: return FE_EUNSUPPORTED;
  }
  return from_cuda(e);
}

extern "C" fe_status fe_apply_host(fe_ctx* c, const void* Xh, void* Yh, int n_vec, void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!Xh || !Yh) return FE_EINVAL;
  const size_t bytes = c->n_dofs * (size_t)n_vec * elem_size(c->mode);
  if (c->stage_bytes < 2 * bytes) {
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_stage, 2 * bytes);
    if (e != cudaSuccess) return from_cuda(e);
    c->stage_bytes = 2 * bytes;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  char* dX = static_cast<char*>(c->d_stage);
  char* dY = dX + bytes;
  cudaError_t e = cudaMemcpyAsync(dX, Xh, bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return from_cuda(e);
  fe_status st = fe_apply(c, dX, dY, n_vec, stream);
  if (st != FE_OK) return st;
  e = cudaMemcpyAsync(Yh, dY, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

extern "C" fe_status fe_diagonal(fe_ctx* c, double* diag, void* stream) {
  if (!c || !diag) return FE_EINVAL;
  return from_cuda(diagonal_f64(c, diag, static_cast<cudaStream_t>(stream)));
}

extern "C" fe_status fe_last_device_status(fe_ctx* c) {
  if (!c) return FE_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return FE_ECUDA;
  int h = 0;
  e = cudaMemcpy(&h, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return FE_ECUDA;
  cudaMemset(c->d_status, 0, sizeof(int));
  return static_cast<fe_status>(h);
}

extern "C" const char* fe_status_str(fe_status s) {
  switch (s) {
    case FE_OK: return "ok";
    case FE_EINVAL: return "invalid argument";
    case FE_ENOMEM: return "out of memory";
    case FE_ECUDA: return "CUDA error";
    case FE_ENOTCONV: return "solver did not converge";
    case FE_EBREAKDOWN: return "Krylov breakdown";
    case FE_ENONFINITE: return "non-finite value";
    case FE_ETIMEOUT: return "bounded device wait timed out";
    case FE_EUNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}
