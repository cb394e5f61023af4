// Block size 8 instantiation of the sparse block step (see k_sparse_impl.cuh).
#include "k_sparse_impl.cuh"

namespace ials {
cudaError_t launch_sparse_b8(const StepArgs &a, cudaStream_t s) {
    return launch_sparse_dispatch<8>(a, s);
}
}  // namespace ials
