// Block size 64 instantiation of the BF16 tensor-core sparse block step: one
// row per pair of warps (k_sparse_pair64.cuh) for Algorithm 3, the CTA kernel
// (k_sparse_cta_bf16.cuh) for the direct solve of Algorithm 1 (b = d = 64).
#include "k_sparse_pair64.cuh"

namespace ials {
cudaError_t launch_sparse_bf16_b64(const StepArgs &a, cudaStream_t s) {
    if (a.direct) return launch_sparse_cta_bf16_dispatch<64>(a, s);
    if (a.alpha) return a.pos ? launch_sparse_pair64_bf16_all<true, true>(a, s) : launch_sparse_pair64_bf16_all<false, true>(a, s);
    return a.pos ? launch_sparse_pair64_bf16_all<true, false>(a, s) : launch_sparse_pair64_bf16_all<false, false>(a, s);
}
}  // namespace ials
