// Instantiation of the tensor-core cell kernel for one operand kind over every
// supported (p, n_q), uniform and trilinear cells.
#pragma once

#include "fe_dispatch.cuh"
#include "fe_mma_kernel.cuh"

namespace fe {

template <int KIND>
cudaError_t apply_mma_kind(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
#define FE_CASE(P, NQ)                                                          \
  if (c->p == P && c->nq == NQ) {                                               \
    return c->general ? launch_mma<P + 1, NQ, true, KIND>(c, X, Y, n_vec, s)    \
                      : launch_mma<P + 1, NQ, false, KIND>(c, X, Y, n_vec, s);  \
  }
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
