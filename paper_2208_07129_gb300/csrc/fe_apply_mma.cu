// Tensor-core cell kernels: mode dispatch.  Each operand kind is compiled in
// its own translation unit (fe_apply_mma_<kind>.cu) so that the build runs
// them in parallel.
#include "fe_internal.h"

namespace fe {

template <int KIND>
cudaError_t apply_mma_kind(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s);

cudaError_t apply_mma_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s, fe_mode mode) {
  switch (mode) {
    case FE_TF32: return apply_mma_kind<0>(c, X, Y, n_vec, s);
    case FE_BF16: return apply_mma_kind<1>(c, X, Y, n_vec, s);
    case FE_TF32X3: return apply_mma_kind<2>(c, X, Y, n_vec, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fe
