// Double-float cell kernels, geometry per cell (affine), plain product.
#include "fe_df64_variant.cuh"

namespace fe {
template cudaError_t apply_df64_variant<false, false>(const fe_ctx*, const double*, double*, int, cudaStream_t,
                                                    const Scale<double>&);
}  // namespace fe
