// FP32 CUDA-core instantiations of the fused cell kernel.
#include "fe_dispatch.cuh"

namespace fe {

cudaError_t apply_cc_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
#define FE_CASE(P, NQ)                                                                        \
  if (c->p == P && c->nq == NQ)                                                               \
    return c->general ? launch_apply<float, P + 1, NQ, true>(c, X, Y, n_vec, s, c->vb32, c->nty32) \
                      : launch_apply<float, P + 1, NQ, false>(c, X, Y, n_vec, s, c->vb32, c->nty32);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
