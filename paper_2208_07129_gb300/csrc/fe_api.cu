// C ABI of libfe: apply, host-buffer apply, diagonal, status.
#include <cstring>

#include "fe_internal.h"

using namespace fe;

namespace {
fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}
size_t elem_size(fe_mode m) {
  return (m == FE_FP64 || m == FE_DF64) ? sizeof(double) : m == FE_BF16S ? (size_t)2 : sizeof(float);
}

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
  if (c->refined) {
    if (c->mode != FE_FP64 && c->mode != FE_DF64 && c->mode != FE_FP32) return FE_EUNSUPPORTED;
    return from_cuda(apply_refined(c, X, Y, n_vec, s));
  }
  switch (c->mode) {
    case FE_FP64: e = apply_cc_f64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, s); break;
    case FE_DF64: e = apply_df64(c, static_cast<const double*>(X), static_cast<double*>(Y), n_vec, s); break;
    case FE_FP32: e = apply_cc_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, s); break;
    case FE_TF32:
    case FE_BF16:
      if (c->tc_variant != 1 && tc_supported(c)) {
        e = apply_tc(c, X, Y, n_vec, s, c->mode);
        break;
      }
      [[fallthrough]];
    case FE_TF32X3:
      if ((size_t)3 * c->nq * c->nq * c->nq * 16 * sizeof(float) > 220 * 1024) return FE_EUNSUPPORTED;
      e = apply_mma_f32(c, static_cast<const float*>(X), static_cast<float*>(Y), n_vec, s, c->mode);
      break;
    case FE_BF16S:
      if (!tc_supported(c)) return FE_EUNSUPPORTED;
      e = apply_tc(c, X, Y, n_vec, s, c->mode);
      break;
    default: return FE_EUNSUPPORTED;
  }
  return from_cuda(e);
}

namespace {
// Vectors per chunk of the host-buffer pipeline: rows of 128 bytes (16 FP64
// or 32 FP32 values) keep the strided host copies near full link speed.
// Fewer than two chunks' worth of vectors goes through one plain copy.
int host_chunk_vectors(int n_vec, size_t elem) {
  const int cv = (int)(128 / elem);
  return n_vec >= 2 * cv ? cv : n_vec;
}

cudaError_t host_pipeline_ready(fe_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (!c->copy_in) e = cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->copy_out) e = cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking);
  cudaEvent_t* evs[] = {&c->ev_start, &c->ev_in[0], &c->ev_in[1], &c->ev_comp[0], &c->ev_comp[1], &c->ev_out[0],
                        &c->ev_out[1]};
  for (cudaEvent_t* ev : evs)
    if (e == cudaSuccess && !*ev) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  return e;
}

// The pipeline proper: chunk k of cv vector columns is copied in on copy_in,
// applied on s and copied out on copy_out; two stage buffers per side let the
// copies of chunks k-1 and k+1 run under the product of chunk k.
fe_status apply_host_pipelined(fe_ctx* c, const char* Xh, char* Yh, int n_vec, int cv, cudaStream_t s) {
  const size_t elem = elem_size(c->mode);
  const size_t chunk_bytes = c->n_dofs * (size_t)cv * elem;
  const size_t pitch = (size_t)n_vec * elem;
  char* Xs[2] = {static_cast<char*>(c->d_stage), static_cast<char*>(c->d_stage) + chunk_bytes};
  char* Ys[2] = {Xs[0] + 2 * chunk_bytes, Xs[0] + 3 * chunk_bytes};
  cudaError_t e = cudaEventRecord(c->ev_start, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_in, c->ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_out, c->ev_start, 0);
  fe_status st = FE_OK;
  for (int k = 0, c0 = 0; c0 < n_vec && e == cudaSuccess && st == FE_OK; ++k, c0 += cv) {
    const int b = k & 1;
    const int w = n_vec - c0 < cv ? n_vec - c0 : cv;
    const size_t wb = (size_t)w * elem;
    // X stage b is free once the product of chunk k-2 has run
    if (k >= 2) e = cudaStreamWaitEvent(c->copy_in, c->ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Xs[b], wb, Xh + c0 * elem, pitch, wb, c->n_dofs, cudaMemcpyHostToDevice, c->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_in[b], c->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_in[b], 0);
    // Y stage b is free once chunk k-2 has been copied out
    if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(s, c->ev_out[b], 0);
    if (e != cudaSuccess) break;
    st = fe_apply(c, Xs[b], Ys[b], w, s);
    if (st != FE_OK) break;
    e = cudaEventRecord(c->ev_comp[b], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->copy_out, c->ev_comp[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(Yh + c0 * elem, pitch, Ys[b], wb, wb, c->n_dofs, cudaMemcpyDeviceToHost, c->copy_out);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out[b], c->copy_out);
  }
  if (e == cudaSuccess && st == FE_OK) {
    e = cudaEventRecord(c->ev_start, c->copy_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c->ev_start, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return from_cuda(e);
  }
  // leave no copy in flight into or out of the stage on an error
  cudaStreamSynchronize(c->copy_in);
  cudaStreamSynchronize(s);
  cudaStreamSynchronize(c->copy_out);
  return st != FE_OK ? st : from_cuda(e);
}
}  // namespace

namespace {
// Device address of a page-locked, device-mapped host buffer (cudaHostAlloc,
// cudaHostRegister, torch's pin_memory), or nullptr for any other pointer.
void* mapped_host(const void* h) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
    cudaGetLastError();   // clear the error of an unknown pointer
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}
}  // namespace

extern "C" fe_status fe_apply_host(fe_ctx* c, const void* Xh, void* Yh, int n_vec, void* stream) {
  if (!c || n_vec < 0) return FE_EINVAL;
  if (n_vec == 0) return FE_OK;
  if (!Xh || !Yh) return FE_EINVAL;
  // FP64 on pinned buffers: the cell kernel reads X and writes Y in host
  // memory directly over the host link (NVLink-C2C on GB300).  The FP64
  // product does about 28 flop per byte on a pipe 1/64 the FP32 rate, so the
  // link traffic hides under the arithmetic and no staging copy is needed.
  if (c->mode == FE_FP64) {
    void* dX = mapped_host(Xh);
    void* dY = dX ? mapped_host(Yh) : nullptr;
    if (dX && dY) {
      cudaStream_t s = static_cast<cudaStream_t>(stream);
      fe_status st = fe_apply(c, dX, dY, n_vec, stream);
      cudaError_t e = cudaStreamSynchronize(s);
      return st != FE_OK ? st : from_cuda(e);
    }
  }
  const size_t elem = elem_size(c->mode);
  const int cv = host_chunk_vectors(n_vec, elem);
  const bool pipelined = cv < n_vec;
  const size_t chunk_bytes = c->n_dofs * (size_t)cv * elem;
  const size_t need = (pipelined ? 4 : 2) * chunk_bytes;
  if (c->stage_bytes < need) {
    cudaFree(c->d_stage);
    c->d_stage = nullptr;
    c->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_stage, need);
    if (e != cudaSuccess) return from_cuda(e);
    c->stage_bytes = need;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (pipelined) {
    cudaError_t e = host_pipeline_ready(c);
    if (e != cudaSuccess) return from_cuda(e);
    return apply_host_pipelined(c, static_cast<const char*>(Xh), static_cast<char*>(Yh), n_vec, cv, s);
  }
  const size_t bytes = chunk_bytes;
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
  if (c->refined) return FE_EUNSUPPORTED;
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
