// Partial Gramian G^{pi} = X^T X[:, pi] (Eq. 10) on the 5th-generation tensor
// cores (tcgen05), for precision IALS_PREC_BF16.
//
// X is the fixed side, held as BF16 hi/lo shadows (x = hi + lo); the product is
// compensated, G = Xh^T Xh_pi + Xh^T Xl_pi + Xl^T Xh_pi, all three chained into
// one FP32 accumulator in tensor memory.  One CTA computes a 128 x b tile of G
// (128 coordinates of d, all b columns of the block) over a range of rows of X
// (split-K); partial tiles go to a workspace and k_gram_reduce sums them in
// split order.
//
// Operands: D[m][j] = sum_k A[m][k] B[j][k] with A[m][k] = X[k][m] and
// B[j][k] = X[k][p0 + j].  X is row-major, so both operands are MN-major: TMA
// copies boxes of 64 rows of X (64 coordinates = 128 B per row for A, b
// coordinates = 2b bytes per row for B) with the matching 128B / 64B / 32B
// swizzle, which is the canonical MN-major layout: atoms of 8 rows, leading
// byte offset = distance between 64-coordinate atoms of A, stride byte offset
// = distance between 8-row groups.  Warp 0 lane 0 issues the TMA copies, warp 1
// lane 0 issues the MMAs, four stages in flight; all four warps read the
// accumulator back with tcgen05.ld.  Every wait is bounded: on timeout the
// kernel records an error code, waits (bounded) for its own copies and MMAs,
// releases tensor memory and returns.
#include "ials_internal.cuh"

#include <cuda.h>

#include <mutex>

namespace ials {

namespace {

constexpr int TC_BK = 64;      // rows of X per stage
constexpr int TC_STAGES = 4;
constexpr int TC_M = 128;      // coordinates of d per CTA
constexpr uint32_t TC_MAXIT = 1u << 22;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < TC_MAXIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start, leading / stride byte
// offsets (16-byte units), descriptor version 1, swizzle mode.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(swz & 7u) << 61;
    return d;
}

constexpr uint32_t SWZ_128B = 2, SWZ_64B = 4, SWZ_32B = 6;

// Instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both MN-major.
constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int N>
struct TcGramCfg {
    static constexpr int A_BOX = 64 * TC_BK * 2;       // one 64-coordinate box: 8 KB
    static constexpr int A_BYTES = 2 * A_BOX;          // 128 coordinates
    static constexpr int B_BYTES = N * TC_BK * 2;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;  // hi and lo of A and B
    static constexpr int RB = 2 * N;                   // bytes per row of a B box
    static constexpr uint32_t B_SWZ = N == 64 ? SWZ_128B : (N == 32 ? SWZ_64B : SWZ_32B);
    static constexpr int SMEM = TC_STAGES * STAGE + 1024 + 256;
};

template <int N>
__global__ void __launch_bounds__(128, 1)
    k_tc_gram(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
              const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
              int64_t n, int32_t d, int32_t p0, int32_t bs, int32_t ktiles_per_split,
              float *__restrict__ ws, int32_t *err) {
    using C = TcGramCfg<N>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + TC_STAGES * C::STAGE);
    uint64_t *empty = full + TC_STAGES;
    uint64_t *done = empty + TC_STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * TC_M;
    const int64_t kt0 = (int64_t)blockIdx.y * ktiles_per_split;
    const int64_t kt_total = (n + TC_BK - 1) / TC_BK;
    const int nk = (int)max((int64_t)0, min((int64_t)ktiles_per_split, kt_total - kt0));
    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (tid == 0) {  // TMA producer
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TC_STAGES;
            if (kt >= TC_STAGES && !mbar_wait(&empty[s], ((kt / TC_STAGES) - 1) & 1)) {
                atomicExch(err, 1);
                break;
            }
            uint8_t *st = base + s * C::STAGE;
            mbar_expect_tx(&full[s], C::STAGE);
            const int y = (int)((kt0 + kt) * TC_BK);
            tma_load_2d(st, &mAh, m0, y, &full[s]);
            tma_load_2d(st + C::A_BOX, &mAh, m0 + 64, y, &full[s]);
            tma_load_2d(st + C::A_BYTES, &mAl, m0, y, &full[s]);
            tma_load_2d(st + C::A_BYTES + C::A_BOX, &mAl, m0 + 64, y, &full[s]);
            tma_load_2d(st + 2 * C::A_BYTES, &mBh, p0, y, &full[s]);
            tma_load_2d(st + 2 * C::A_BYTES + C::B_BYTES, &mBl, p0, y, &full[s]);
        }
    } else if (tid == 32) {  // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_mn(TC_M, N);
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % TC_STAGES;
            if (!mbar_wait(&full[s], (kt / TC_STAGES) & 1)) {
                atomicExch(err, 2);
                break;
            }
            tc_fence_after();
            const uint32_t ah = smem_u32(base + s * C::STAGE), al = ah + C::A_BYTES;
            const uint32_t bh = ah + 2 * C::A_BYTES, bl = bh + C::B_BYTES;
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j) {
                const uint64_t dah = smem_desc(ah + j * 16 * 128, C::A_BOX, 8 * 128, SWZ_128B);
                const uint64_t dal = smem_desc(al + j * 16 * 128, C::A_BOX, 8 * 128, SWZ_128B);
                const uint64_t dbh = smem_desc(bh + j * 16 * C::RB, C::B_BYTES, 8 * C::RB, C::B_SWZ);
                const uint64_t dbl = smem_desc(bl + j * 16 * C::RB, C::B_BYTES, 8 * C::RB, C::B_SWZ);
                const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p, q;\n setp.ne.b32 p, %4, 0;\n setp.eq.b32 q, %4, %4;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %3, q;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %2, %3, q;\n}\n" ::"r"(tmem),
                    "l"(dah), "l"(dbh), "r"(idesc), "r"(acc), "l"(dbl), "l"(dal)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(done, 0);
    if (!ok && (tid & 31) == 0) atomicExch(err, 3);
    tc_fence_after();
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int m = m0 + warp * 32 + (tid & 31);
    if (m < d) {
        float *out = ws + (int64_t)blockIdx.y * d * bs + (int64_t)m * bs;
#pragma unroll
        for (int j = 0; j < N; ++j)
            if (j < bs) out[j] = (nk > 0 && ok) ? __uint_as_float(r[j]) : 0.f;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ row terms
// R[r, f] = alpha0 * sum_k X[r, k] G[k, f] + lambda (1 + nu n_r) X[r, p0 + f]
// (Algorithm 3 gradient initialisation; dense part of Eq. 11) on tcgen05:
// D (128 rows x N) = A (rows x d) B^T with A[m][k] = X[r0+m][k] and
// B[f][k] = G[k][f] = G^T[f][k].  Both operands are K-major (X rows and the rows
// of G^T are contiguous in k): TMA boxes of 64 k x 128 rows (A) and 64 k x N
// rows (B) with the 128B swizzle, i.e. atoms of 8 rows x 128 B, stride byte
// offset 1024 between atoms; a K step of 16 advances the start address by 32 B
// inside the atom.  hi/lo compensation as in the Gramian.
template <int N>
struct TcRowCfg {
    static constexpr int A_BYTES = 128 * 64 * 2;   // 16 KB
    static constexpr int B_BYTES = N * 64 * 2;
    static constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;
    static constexpr int STAGES = 2;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

constexpr uint32_t idesc_bf16_k(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int N>
__global__ void __launch_bounds__(128, 1)
    k_tc_rowterm(const __grid_constant__ CUtensorMap mXh, const __grid_constant__ CUtensorMap mXl,
                 const __grid_constant__ CUtensorMap mGh, const __grid_constant__ CUtensorMap mGl,
                 const float *__restrict__ X, const int64_t *__restrict__ ptr, int32_t n_rows, int32_t d,
                 int32_t p0, float alpha0, float lambda, float nu, float *__restrict__ R, int32_t ldr,
                 int32_t *err) {
    using C = TcRowCfg<N>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *full = reinterpret_cast<uint64_t *>(base + C::STAGES * C::STAGE);
    uint64_t *empty = full + C::STAGES;
    uint64_t *done = empty + C::STAGES;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r0 = blockIdx.x * 128;
    const int nk = d / 64 + (d % 64 ? 1 : 0);
    if (tid == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    if (tid == 0) {
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % C::STAGES;
            if (kt >= C::STAGES && !mbar_wait(&empty[s], ((kt / C::STAGES) - 1) & 1)) {
                atomicExch(err, 11);
                break;
            }
            uint8_t *st = base + s * C::STAGE;
            mbar_expect_tx(&full[s], C::STAGE);
            tma_load_2d(st, &mXh, kt * 64, r0, &full[s]);
            tma_load_2d(st + C::A_BYTES, &mXl, kt * 64, r0, &full[s]);
            tma_load_2d(st + 2 * C::A_BYTES, &mGh, kt * 64, 0, &full[s]);
            tma_load_2d(st + 2 * C::A_BYTES + C::B_BYTES, &mGl, kt * 64, 0, &full[s]);
        }
    } else if (tid == 32) {
        constexpr uint32_t idesc = idesc_bf16_k(128, N);
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % C::STAGES;
            if (!mbar_wait(&full[s], (kt / C::STAGES) & 1)) {
                atomicExch(err, 12);
                break;
            }
            tc_fence_after();
            const uint32_t xh = smem_u32(base + s * C::STAGE), xl = xh + C::A_BYTES;
            const uint32_t gh = xh + 2 * C::A_BYTES, gl = gh + C::B_BYTES;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t dxh = smem_desc(xh + 32 * j, 16, 1024, SWZ_128B);
                const uint64_t dxl = smem_desc(xl + 32 * j, 16, 1024, SWZ_128B);
                const uint64_t dgh = smem_desc(gh + 32 * j, 16, 1024, SWZ_128B);
                const uint64_t dgl = smem_desc(gl + 32 * j, 16, 1024, SWZ_128B);
                const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p, q;\n setp.ne.b32 p, %4, 0;\n setp.eq.b32 q, %4, %4;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %3, q;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %2, %3, q;\n}\n" ::"r"(tmem),
                    "l"(dxh), "l"(dgh), "r"(idesc), "r"(acc), "l"(dgl), "l"(dxl)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             smem_u32(&empty[s]))
                         : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(done))
                     : "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait(done, 0);
    if (!ok && (tid & 31) == 0) atomicExch(err, 13);
    tc_fence_after();
    uint32_t r[32];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    const int row = r0 + warp * 32 + (tid & 31);
    if (row < n_rows && ok) {
        const float lam = lambda * (1.0f + nu * (float)(ptr[row + 1] - ptr[row]));
        const float *x = X + (int64_t)row * d + p0;
        float *out = R + (int64_t)row * ldr;
#pragma unroll
        for (int f = 0; f < N; f += 4) {
            const float4 xv = *reinterpret_cast<const float4 *>(x + f);
            *reinterpret_cast<float4 *>(out + f) =
                make_float4(alpha0 * __uint_as_float(r[f]) + lam * xv.x, alpha0 * __uint_as_float(r[f + 1]) + lam * xv.y,
                            alpha0 * __uint_as_float(r[f + 2]) + lam * xv.z, alpha0 * __uint_as_float(r[f + 3]) + lam * xv.w);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem) : "memory");
}

// Columns col0 .. col0+b-1 of G (d x ldg, FP32) -> their transpose, hi and lo (b x d, BF16)
__global__ void k_transpose_split(const float *__restrict__ G, int32_t ldg, int32_t col0, int32_t d, int32_t b,
                                  __nv_bfloat16 *__restrict__ th, __nv_bfloat16 *__restrict__ tl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d * b) return;
    const int f = i / d, k = i % d;
    const float x = G[(int64_t)k * ldg + col0 + f];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    th[i] = h;
    tl[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// ------------------------------------------------------------------ host side
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled get_encode() {
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
        cudaGetLastError();
    });
    return fn;
}

bool encode_2d(CUtensorMap *map, const __nv_bfloat16 *ptr, int64_t rows, int32_t cols, int box_cols,
               int box_rows, CUtensorMapSwizzle swz) {
    EncodeTiled enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int tc_splits(int64_t n, int32_t d, int &kper) {
    const int mt = (d + TC_M - 1) / TC_M;
    const int64_t kt = (n + TC_BK - 1) / TC_BK;
    int64_t ns = (152 + mt - 1) / mt;  // about one CTA per SM
    if (ns > kt) ns = kt;
    if (ns < 1) ns = 1;
    kper = (int)((kt + ns - 1) / ns);
    if (kper < 1) kper = 1;
    return (int)((kt + kper - 1) / kper);
}

}  // namespace

// Tensor maps of one BF16 hi/lo pair for the tcgen05 Gramian: A boxes
// (64 coordinates x 64 rows, 128B swizzle) and B boxes (b coordinates x 64 rows).
// Blocks wider than 32 columns (b = 64, 128) are processed as 32-column slabs:
// the accumulator holds 32 TMEM columns.
static int tc_slab(int32_t b) { return b <= 32 ? b : 32; }

bool make_gram_maps(GramMaps &g, const __nv_bfloat16 *hi, const __nv_bfloat16 *lo, int64_t rows, int32_t d,
                    int32_t b_full) {
    const int32_t b = tc_slab(b_full);
    if (d % 8 != 0 || (b != 16 && b != 32) || b_full % b != 0) return false;
    const CUtensorMapSwizzle bsw = b == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                           : (b == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    static_assert(sizeof(CUtensorMap) == sizeof(g.ah), "tensor map size");
    return encode_2d(reinterpret_cast<CUtensorMap *>(g.ah), hi, rows, d, 64, TC_BK, CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(g.al), lo, rows, d, 64, TC_BK, CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(g.bh), hi, rows, d, b, TC_BK, bsw) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(g.bl), lo, rows, d, b, TC_BK, bsw);
}

bool make_row_maps(RowMaps &m, const __nv_bfloat16 *xh, const __nv_bfloat16 *xl, int64_t rows, int32_t d,
                   const __nv_bfloat16 *gth, const __nv_bfloat16 *gtl, int32_t b_full) {
    const int32_t b = tc_slab(b_full);
    if (d % 8 != 0 || (b != 16 && b != 32) || b_full % b != 0) return false;
    static_assert(sizeof(CUtensorMap) == sizeof(m.xh), "tensor map size");
    return encode_2d(reinterpret_cast<CUtensorMap *>(m.xh), xh, rows, d, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(m.xl), xl, rows, d, 64, 128, CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(m.gh), gth, b, d, 64, b, CU_TENSOR_MAP_SWIZZLE_128B) &&
           encode_2d(reinterpret_cast<CUtensorMap *>(m.gl), gtl, b, d, 64, b, CU_TENSOR_MAP_SWIZZLE_128B);
}

cudaError_t launch_rowterm_tc(const RowMaps &m, const float *G, __nv_bfloat16 *gth, __nv_bfloat16 *gtl,
                              const float *X, const int64_t *ptr, int32_t n_rows, int32_t d, int32_t p0, int32_t b,
                              float alpha0, float lambda, float nu, float *R, int32_t *err, cudaStream_t s) {
    if (n_rows == 0) return cudaSuccess;
    const int32_t bs = tc_slab(b);
    if ((bs != 16 && bs != 32) || b % bs != 0) return cudaErrorInvalidValue;
    const CUtensorMap *xh = reinterpret_cast<const CUtensorMap *>(m.xh);
    const CUtensorMap *xl = reinterpret_cast<const CUtensorMap *>(m.xl);
    const CUtensorMap *gh = reinterpret_cast<const CUtensorMap *>(m.gh);
    const CUtensorMap *gl = reinterpret_cast<const CUtensorMap *>(m.gl);
    const int grid = (n_rows + 127) / 128;
    static bool a16 = false, a32 = false;
    cudaError_t e = cudaSuccess;
    if (bs == 16 && !a16) {
        e = cudaFuncSetAttribute(k_tc_rowterm<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcRowCfg<16>::SMEM);
        if (e != cudaSuccess) return e;
        a16 = true;
    }
    if (bs == 32 && !a32) {
        e = cudaFuncSetAttribute(k_tc_rowterm<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcRowCfg<32>::SMEM);
        if (e != cudaSuccess) return e;
        a32 = true;
    }
    // one slab of bs columns at a time: its G^T columns, then R[:, c0 : c0 + bs]
    for (int32_t c0 = 0; c0 < b; c0 += bs) {
        k_transpose_split<<<(d * bs + 255) / 256, 256, 0, s>>>(G, b, c0, d, bs, gth, gtl);
        if (bs == 16)
            k_tc_rowterm<16><<<grid, 128, TcRowCfg<16>::SMEM, s>>>(*xh, *xl, *gh, *gl, X, ptr, n_rows, d, p0 + c0,
                                                                   alpha0, lambda, nu, R + c0, b, err);
        else
            k_tc_rowterm<32><<<grid, 128, TcRowCfg<32>::SMEM, s>>>(*xh, *xl, *gh, *gl, X, ptr, n_rows, d, p0 + c0,
                                                                   alpha0, lambda, nu, R + c0, b, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int64_t gram_tc_ws_floats(int64_t n, int32_t d, int32_t bs) {
    int kper = 0;
    return (int64_t)tc_splits(n, d, kper) * d * bs;
}

cudaError_t launch_gram_tc(const GramMaps &g, int64_t n, int32_t d, int32_t p0, int32_t b, float *G, float *ws,
                           int32_t *err, cudaStream_t s) {
    const int64_t count = (int64_t)d * b;
    if (n == 0) return cudaMemsetAsync(G, 0, sizeof(float) * count, s);
    const int32_t bs = tc_slab(b);
    if ((bs != 16 && bs != 32) || b % bs != 0) return cudaErrorInvalidValue;
    int kper = 0;
    const int ns = tc_splits(n, d, kper);
    const dim3 grid((d + TC_M - 1) / TC_M, ns);
    const CUtensorMap *ah = reinterpret_cast<const CUtensorMap *>(g.ah);
    const CUtensorMap *al = reinterpret_cast<const CUtensorMap *>(g.al);
    const CUtensorMap *bh = reinterpret_cast<const CUtensorMap *>(g.bh);
    const CUtensorMap *bl = reinterpret_cast<const CUtensorMap *>(g.bl);
    static bool attr16 = false, attr32 = false;
    cudaError_t e = cudaSuccess;
    if (bs == 16 && !attr16) {
        e = cudaFuncSetAttribute(k_tc_gram<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcGramCfg<16>::SMEM);
        if (e != cudaSuccess) return e;
        attr16 = true;
    }
    if (bs == 32 && !attr32) {
        e = cudaFuncSetAttribute(k_tc_gram<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcGramCfg<32>::SMEM);
        if (e != cudaSuccess) return e;
        attr32 = true;
    }
    // one slab of bs columns at a time (split-K partials, then a fixed-order
    // reduce into columns c0 .. c0 + bs - 1 of G)
    for (int32_t c0 = 0; c0 < b; c0 += bs) {
        if (bs == 16)
            k_tc_gram<16><<<grid, 128, TcGramCfg<16>::SMEM, s>>>(*ah, *al, *bh, *bl, n, d, p0 + c0, bs, kper, ws, err);
        else
            k_tc_gram<32><<<grid, 128, TcGramCfg<32>::SMEM, s>>>(*ah, *al, *bh, *bl, n, d, p0 + c0, bs, kper, ws, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_gram_reduce_cols(ws, ns, d, bs, G, b, c0, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ials
