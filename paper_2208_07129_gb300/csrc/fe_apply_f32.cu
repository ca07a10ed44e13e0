// FP32 CUDA-core instantiations: the line kernel, the line kernel with
// even-odd contractions, or the register-plane kernel (n_q <= 8), as
// selected with fe_set_tile.
#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"
#include "fe_plane_kernel.cuh"

namespace fe {

namespace {
template <int NP, int NQ, bool GEN>
cudaError_t pick(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
  if constexpr (NQ <= 8) {
    if (c->fp32_variant == 2) return launch_plane<NP, NQ, GEN>(c, X, Y, n_vec, s);
  }
  if (c->fp32_variant == 3) return launch_apply_eo<float, NP, NQ, GEN>(c, X, Y, n_vec, s, c->vb32, c->nty32);
  return launch_apply<float, NP, NQ, GEN>(c, X, Y, n_vec, s, c->vb32, c->nty32);
}
}  // namespace

cudaError_t apply_cc_f32(const fe_ctx* c, const float* X, float* Y, int n_vec, cudaStream_t s) {
#define FE_CASE(P, NQ) \
  if (c->p == P && c->nq == NQ) \
    return c->general ? pick<P + 1, NQ, true>(c, X, Y, n_vec, s) : pick<P + 1, NQ, false>(c, X, Y, n_vec, s);
  FE_FOR_EACH_P_NQ(FE_CASE)
#undef FE_CASE
  return cudaErrorInvalidValue;
}

}  // namespace fe
