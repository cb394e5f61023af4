// Block size 64 instantiation of the sparse block step: one row per pair of
// warps (k_sparse_pair64.cuh) for Algorithm 3, the register-tile kernel
// (k_sparse_rc.cuh) for the direct solve of Algorithm 1 (b = d = 64).
#include "k_sparse_pair64.cuh"

namespace ials {
cudaError_t launch_sparse_b64(const StepArgs &a, cudaStream_t s) {
    if (a.direct) return launch_sparse_rc_dispatch<64>(a, s);
    const bool perm = a.pos != nullptr, wa = a.alpha != nullptr;
    if (perm) return wa ? launch_sparse_pair64_all<true, true>(a, s) : launch_sparse_pair64_all<true, false>(a, s);
    return wa ? launch_sparse_pair64_all<false, true>(a, s) : launch_sparse_pair64_all<false, false>(a, s);
}
}  // namespace ials
