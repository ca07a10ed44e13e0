// FE_DF64 entry points of the double-float cell kernel on structured meshes;
// the kernels themselves are instantiated in fe_df64_{affine,general}.cu and
// fe_df64_scaled_{affine,general}.cu.
#include "fe_internal.h"

namespace fe {

template <bool GEN, bool SC>
cudaError_t apply_df64_variant(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s,
                               const Scale<double>& sc);

cudaError_t apply_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s) {
  const Scale<double> none{};
  return c->general ? apply_df64_variant<true, false>(c, X, Y, n_vec, s, none)
                    : apply_df64_variant<false, false>(c, X, Y, n_vec, s, none);
}

cudaError_t apply_scaled_df64(const fe_ctx* c, const double* X, double* Y, int n_vec, const Scale<double>& sc,
                              cudaStream_t s) {
  return c->general ? apply_df64_variant<true, true>(c, X, Y, n_vec, s, sc)
                    : apply_df64_variant<false, true>(c, X, Y, n_vec, s, sc);
}

}  // namespace fe
