// ials_partial_gramian_noalloc: the split-K partial Gramian for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc / cudaFree at the point where they need
// a Gramian: code whose device memory is owned by another allocator (a
// framework's caching allocator or a fixed arena that must account for every
// byte), and latency-bound loops such as a serving path, where cudaMalloc and
// cudaFree may synchronise the device and take unbounded time.  This entry
// point keeps the split-K partial sums in a file-scope device array instead:
// kNoAllocScratchFloats floats (8 MiB), held by every GPU that loads the
// library until the process exits.  The caller still passes X and G.
#include "ials_internal.cuh"
#include "../../include/ials.h"

#include <mutex>
#include <string>

namespace {

constexpr int64_t kNoAllocScratchFloats = int64_t(2) << 20;  // 2 Mi floats = 8 MiB
constexpr int kMaxDevices = 64;

// Partial sums of the split-K Gramian.  Host code must not use this name as a
// pointer: it is a host-side stand-in.  Its device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) float g_gram_scratch[kNoAllocScratchFloats];

std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

namespace ials {
void set_last_error(const std::string &msg);
}

extern "C" ials_status ials_partial_gramian_noalloc(const float *X, int64_t n, int32_t d,
                                                    int32_t p0, int32_t bs, float *G,
                                                    void *cuda_stream) {
    if (!X || !G || n < 0 || d < 1 || bs < 1 || p0 < 0 || p0 + bs > d) {
        ials::set_last_error("bad Gramian arguments");
        return IALS_EINVAL;
    }
    if ((int64_t)d * bs > kNoAllocScratchFloats) {
        ials::set_last_error("d * bs = " + std::to_string((int64_t)d * bs) +
                             " exceeds the fixed Gramian scratch of " +
                             std::to_string(kNoAllocScratchFloats) + " floats");
        return IALS_EINVAL;
    }
    // X and G must be memory the GPU addresses directly: unlike the library's
    // other calls this one copies nothing, so a host array is refused here
    // rather than handed to the kernel.  cudaPointerGetAttributes allocates nothing.
    for (const void *p : {static_cast<const void *>(X), static_cast<const void *>(G)}) {
        cudaPointerAttributes at;
        const cudaError_t pe = cudaPointerGetAttributes(&at, p);
        if (pe != cudaSuccess) cudaGetLastError();
        if (pe != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            ials::set_last_error("X and G must be device (or managed) memory");
            return IALS_EINVAL;
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        ials::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return IALS_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        ials::set_last_error("device index " + std::to_string(dev) + " exceeds the " +
                             std::to_string(kMaxDevices) + " devices this entry point supports");
        return IALS_ECUDA;
    }
    float *ws = nullptr;
    {
        // Set-up on the first call on this device (the device is current here).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_gram_scratch);
            if (e != cudaSuccess || !p) {
                ials::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                cudaGetLastError();
                return IALS_ECUDA;
            }
            g_scratch_ptr[dev] = static_cast<float *>(p);
            e = ials::dense_prepare();  // kernel attributes, also once per device before any capture
            if (e != cudaSuccess) {
                ials::set_last_error(std::string("kernel attributes: ") + cudaGetErrorString(e));
                cudaGetLastError();
                g_scratch_ptr[dev] = nullptr;
                return IALS_ECUDA;
            }
        }
        ws = g_scratch_ptr[dev];
    }
    // Every partial slot the reduction reads is written by the tile kernel
    // first, so nothing in the scratch has to start at zero.
    e = ials::launch_gram_capped(X, n, d, p0, bs, G, ws, kNoAllocScratchFloats,
                                 static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) {
        ials::set_last_error(std::string("partial Gramian: ") + cudaGetErrorString(e));
        cudaGetLastError();
        return IALS_ECUDA;
    }
    return IALS_OK;
}
