// Double-float cell kernels, geometry per point (trilinear), scaled (Chebyshev filter) epilogue.
#include "fe_df64_variant.cuh"

namespace fe {
template cudaError_t apply_df64_variant<true, true>(const fe_ctx*, const double*, double*, int, cudaStream_t,
                                                    const Scale<double>&);
}  // namespace fe
