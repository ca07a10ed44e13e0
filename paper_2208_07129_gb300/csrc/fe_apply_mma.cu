// Tensor-core (TF32 / BF16 warp MMA) instantiations of the cell kernel.
#include "fe_dispatch.cuh"
#include "fe_mma_kernel.cuh"

namespace fe {

cudaError_t apply_mma_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s, bool bf16) {
#define FE_CASE(P, NQ)                                                                        \
  if (c->p == P && c->nq == NQ) {                                                             \
    if (c->general)                                                                           \
      return bf16 ? launch_mma<P + 1, NQ, true, true>(c, X, Y, n_vec, s)                     \
                  : launch_mma<P + 1, NQ, true, false>(c, X, Y, n_vec, s);                   \
    return bf16 ? launch_mma<P + 1, NQ, false, true>(c, X, Y, n_vec, s)                      \
                : launch_mma<P + 1, NQ, false, false>(c, X, Y, n_vec, s);                    \
  }
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
