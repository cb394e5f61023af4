// Block size 64 instantiation of the BF16 tensor-core sparse block step: the
// batched warp-solve kernel (k_sparse_gj64.cuh) for Algorithm 3, the CTA kernel
// (k_sparse_cta_bf16.cuh) for the direct solve of Algorithm 1 (b = d = 64).
#include "k_sparse_gj64.cuh"

namespace ials {
cudaError_t launch_sparse_bf16_b64(const StepArgs &a, cudaStream_t s) {
    if (a.direct) return launch_sparse_cta_bf16_dispatch<64>(a, s);
    if (a.alpha) return a.pos ? launch_sparse_gj64_all<true, true, true>(a, s) : launch_sparse_gj64_all<false, true, true>(a, s);
    return a.pos ? launch_sparse_gj64_all<true, false, true>(a, s) : launch_sparse_gj64_all<false, false, true>(a, s);
}
}  // namespace ials
