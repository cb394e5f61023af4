// Block size 64 instantiation of the sparse block step (see k_sparse_rc.cuh).
#include "k_sparse_rc.cuh"

namespace ials {
cudaError_t launch_sparse_b64(const StepArgs &a, cudaStream_t s) {
    return launch_sparse_rc_dispatch<64>(a, s);
}
}  // namespace ials
