// FP32 instantiations of the scaled product of the Chebyshev filter,
// Y = a M^-1/2 A M^-1/2 X + b X + c Y (even-odd line kernel).
#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"

namespace fe {

cudaError_t apply_scaled_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, const Scale<float>& sc,
                             cudaStream_t s) {
#define FE_CASE(P, NQ)                                                                                       \
  if (c->p == P && c->nq == NQ)                                                                              \
    return c->general ? launch_apply_eo<float, P + 1, NQ, true, true>(c, X, Y, n_vec, s, c->vb32, c->nty32, sc) \
                      : launch_apply_eo<float, P + 1, NQ, false, true>(c, X, Y, n_vec, s, c->vb32, c->nty32, sc);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
