// Tensor-core cell kernels, operand kind tf32x3.
#include "fe_apply_mma_kind.cuh"

namespace fe {
template cudaError_t apply_mma_kind<kTF32x3>(const fe_ctx*, const float*, float*, int, cudaStream_t);
}  // namespace fe
