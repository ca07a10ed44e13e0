// Tensor-core cell kernels, operand kind bf16.
#include "fe_apply_mma_kind.cuh"

namespace fe {
template cudaError_t apply_mma_kind<kBF16>(const fe_ctx*, const float*, float*, int, cudaStream_t);
}  // namespace fe
