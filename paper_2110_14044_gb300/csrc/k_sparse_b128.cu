// Block size 128 instantiation of the sparse block step (see k_sparse_rc.cuh).
#include "k_sparse_rc.cuh"

namespace ials {
cudaError_t launch_sparse_b128(const StepArgs &a, cudaStream_t s) {
    return launch_sparse_rc_dispatch<128>(a, s);
}
}  // namespace ials
