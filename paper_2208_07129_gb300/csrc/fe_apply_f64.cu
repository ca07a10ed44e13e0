// FP64 CUDA-core instantiations of the fused cell kernel (even-odd by
// default, the plain line kernel as variant 1) and of the diagonal.
#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"

namespace fe {

cudaError_t apply_cc_f64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s) {
#define FE_CASE(P, NQ)                                                                              \
  if (c->p == P && c->nq == NQ) {                                                                   \
    if (c->fp64_variant == 1)                                                                       \
      return c->general ? launch_apply<double, P + 1, NQ, true>(c, X, Y, n_vec, s, c->vb64, c->nty64) \
                        : launch_apply<double, P + 1, NQ, false>(c, X, Y, n_vec, s, c->vb64, c->nty64); \
    return c->general ? launch_apply_eo<double, P + 1, NQ, true>(c, X, Y, n_vec, s, c->vb64, c->nty64) \
                      : launch_apply_eo<double, P + 1, NQ, false>(c, X, Y, n_vec, s, c->vb64, c->nty64); \
  }
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

cudaError_t diagonal_f64(const fe_ctx* c, double* diag, cudaStream_t s) {
#define FE_CASE(P, NQ) \
  if (c->p == P && c->nq == NQ) \
    return c->general ? launch_diag<P + 1, NQ, true>(c, diag, s) : launch_diag<P + 1, NQ, false>(c, diag, s);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
