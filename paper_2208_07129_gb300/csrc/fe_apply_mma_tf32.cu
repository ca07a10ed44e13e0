// Tensor-core cell kernels, operand kind tf32.
#include "fe_apply_mma_kind.cuh"

namespace fe {
template cudaError_t apply_mma_kind<kTF32>(const fe_ctx*, const float*, float*, int, cudaStream_t);
}  // namespace fe
