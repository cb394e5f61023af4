// Block size 256 instantiation of the sparse block step (register-tile kernel,
// k_sparse_rc.cuh: 528 tiles of 8 x 8, one CTA of 544 threads per row; FP32 only).
#include "k_sparse_rc.cuh"

namespace ials {
cudaError_t launch_sparse_b256(const StepArgs &a, cudaStream_t s) {
    return launch_sparse_rc_dispatch<256>(a, s);
}
int64_t sparse_retry_ws_doubles(int32_t b) { return b == 256 ? retry_ws_doubles<256>() : 0; }
}  // namespace ials
