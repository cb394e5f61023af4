// Block size 64 instantiation of the BF16 tensor-core sparse block step (see k_sparse_cta_bf16.cuh).
#include "k_sparse_cta_bf16.cuh"

namespace ials {
cudaError_t launch_sparse_bf16_b64(const StepArgs &a, cudaStream_t s) {
    return launch_sparse_cta_bf16_dispatch<64>(a, s);
}
}  // namespace ials
