// Block size 128 on the BF16 path: the statistics and solves run on the FP32
// register-tile kernel (k_sparse_rc.cuh), which reads the FP32 factors the BF16
// path keeps beside their hi/lo shadows and updates both.  It was measured faster
// than the compensated tensor-core CTA kernel (k_sparse_cta_bf16.cuh, bound by its
// CTA barriers) at every d tried (256, 512, 1024, 2048); the Gramian and row terms
// of this block size stay on the tcgen05 kernels.
#include "ials_internal.cuh"

namespace ials {
cudaError_t launch_sparse_bf16_b128(const StepArgs &a, cudaStream_t s) { return launch_sparse_b128(a, s); }
}  // namespace ials
