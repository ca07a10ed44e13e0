// Dispatch of the double-float cell kernel over (p, n_q) for one (trilinear
// geometry, scaled epilogue) combination.  Each combination is instantiated
// in its own translation unit (fe_df64_*.cu) so that the 24 (p, n_q) kernels
// of each compile in parallel with the others.
#pragma once

#include "fe_ff_body.cuh"

namespace fe {

template <bool GEN, bool SC>
cudaError_t apply_df64_variant(const fe_ctx* c, const double* X, double* Y, int n_vec, cudaStream_t s,
                               const Scale<double>& sc) {
#define FE_CASE(P, NQ) \
  if (c->p == P && c->nq == NQ) return launch_df64<P + 1, NQ, GEN, SC>(c, X, Y, n_vec, s, sc);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
