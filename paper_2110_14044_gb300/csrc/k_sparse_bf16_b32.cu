// Block size 32 instantiation of the BF16 tensor-core sparse block step (see k_sparse_bf16.cuh).
#include "k_sparse_bf16.cuh"

namespace ials {
cudaError_t launch_sparse_bf16_b32(const StepArgs &a, cudaStream_t s) {
    if (a.alpha) return a.pos ? launch_sparse_bf16_all<32, true, true>(a, s) : launch_sparse_bf16_all<32, false, true>(a, s);
    return a.pos ? launch_sparse_bf16_all<32, true, false>(a, s) : launch_sparse_bf16_all<32, false, false>(a, s);
}
}  // namespace ials
