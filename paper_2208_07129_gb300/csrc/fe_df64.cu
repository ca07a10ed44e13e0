// FE_DF64 instantiations of the double-float cell kernel on structured meshes.
#include "fe_ff_body.cuh"

namespace fe {

cudaError_t apply_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s) {
  const Scale<double> none{};
#define FE_CASE(P, NQ)                                                                  \
  if (c->p == P && c->nq == NQ)                                                         \
    return c->general ? launch_df64<P + 1, NQ, true, false>(c, X, Y, n_vec, s, none)   \
                      : launch_df64<P + 1, NQ, false, false>(c, X, Y, n_vec, s, none);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

cudaError_t apply_scaled_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, const Scale<double>& sc,
                              cudaStream_t s) {
#define FE_CASE(P, NQ)                                                                \
  if (c->p == P && c->nq == NQ)                                                       \
    return c->general ? launch_df64<P + 1, NQ, true, true>(c, X, Y, n_vec, s, sc)    \
                      : launch_df64<P + 1, NQ, false, true>(c, X, Y, n_vec, s, sc);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
