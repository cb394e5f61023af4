// Shared pieces of the CTA-per-row block step for block sizes B = 64 and 128:
// the staged gathers and residual updates, the shared-memory blocked Cholesky
// in 16-column panels (used by the fold-in kernel), and the FP64 re-solve of
// rows whose FP32 pivot failed: statistics accumulated from scratch in FP64 by
// 8 x 8 tile owners, a blocked Cholesky in panels of 8 in FP64 (the routine
// cta_cholesky, templated on the type), apply and residual update.  The FP32
// and BF16 kernels themselves are in k_sparse_rc.cuh and k_sparse_cta_bf16.cuh.
#pragma once

#include "k_sparse_impl.cuh"

namespace ials {

template <int B>
struct CtaCfg {
    static constexpr int NB = B / 8;
    static constexpr int NTL = NB * (NB + 1) / 2;
    static constexpr int NG = B == 64 ? 7 : (B == 128 ? 2 : 1);
    static constexpr int ACTIVE = NTL * NG;
    static constexpr int THREADS = (ACTIVE + 31) / 32 * 32;
    static constexpr int SB = B + 4;   // row stride of staging buffers and of M
    static constexpr int CH = 32;
    static constexpr int BUF = CH * SB;
    // floats: two staging buffers, e[2][CH], a[2][CH], M (B+1 rows), diag0, invd, x, flag
    static constexpr int SMEM_FLOATS = 2 * BUF + 4 * CH + (B + 1) * SB + 3 * B + 4;
    static constexpr int SMEM_BYTES = SMEM_FLOATS * 4;
};

// Lower-triangle tile index t -> (ti, tj), ti >= tj.
__device__ __forceinline__ void tri_index(int t, int &ti, int &tj) {
    int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i * (i + 1) / 2 > t) --i;
    ti = i;
    tj = t - i * (i + 1) / 2;
}

// Blocked Cholesky of the SPD matrix in rows 0..B-1 of M (lower part used),
// carrying the right-hand side in row B.  On return the lower part of rows
// 0..B-1 holds L, row B holds z = L^{-1} rhs, invd[k] = 1 / L_kk.  A pivot that
// is not above rel * diag0[k] (or not finite) sets *bad.  All threads call it.
template <int B, int SM, typename T>
__device__ void cta_cholesky(T *M, T *invd, const T *diag0, int *bad, T rel) {
    constexpr int NB = B / 8;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int p = 0; p < NB; ++p) {
        const int k0 = 8 * p;
        if (tid < 32) {  // diagonal 8 x 8 block: lane r < 8 owns row k0 + r
            const int lane = tid;
            T r[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) r[j] = lane < 8 ? M[(k0 + lane) * SM + k0 + j] : T(0);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const T akk = __shfl_sync(kFull, r[k], k);
                if (lane == k && (!(akk > rel * diag0[k0 + k]) || !(akk < T(1e300)))) *bad = 1;
                const T l = sqrt(akk > T(0) ? akk : T(1e-30));
                const T inv = T(1) / l;
                const T lck = r[k] * inv;
                if (lane == k) invd[k0 + k] = inv;
                r[k] = lck;
#pragma unroll
                for (int j = k + 1; j < 8; ++j) r[j] -= lck * __shfl_sync(kFull, lck, j);
            }
            if (lane < 8) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (j <= lane) M[(k0 + lane) * SM + k0 + j] = r[j];
            }
        }
        __syncthreads();
        // panel: rows k0+8 .. B (the last one is the right-hand side): x L_D^T = a
        for (int i = k0 + 8 + tid; i <= B; i += nt) {
            T x[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = M[i * SM + k0 + j];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
#pragma unroll
                for (int m = 0; m < j; ++m) x[j] -= x[m] * M[(k0 + j) * SM + k0 + m];
                x[j] *= invd[k0 + j];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) M[i * SM + k0 + j] = x[j];
        }
        __syncthreads();
        // trailing update: rows i in [k0+8, B], columns j in [k0+8, min(i, B-1)], in units
        // of 2 rows x 8 columns: M[i][j] -= sum_m M[i][k0+m] M[j][k0+m]
        const int r0 = k0 + 8;
        const int nrow = B + 1 - r0;            // includes the right-hand side row
        const int nrp = (nrow + 1) / 2;         // row pairs
        const int ncb = (B - r0) / 8;           // column blocks
        const int units = nrp * ncb;
        for (int u = tid; u < units; u += nt) {
            const int rp = u / ncb, cb = u % ncb;
            const int i0 = r0 + 2 * rp, j0 = r0 + 8 * cb;
            if (j0 > i0 + 1 && i0 < B) continue;  // wholly above the diagonal (the rhs row never is)
            T a0[8], a1[8];
            const bool two = i0 + 1 <= B;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                a0[m] = M[i0 * SM + k0 + m];
                a1[m] = two ? M[(i0 + 1) * SM + k0 + m] : T(0);
            }
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const int j = j0 + jj;
                T t0 = 0, t1 = 0;
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const T bm = M[j * SM + k0 + m];
                    t0 += a0[m] * bm;
                    t1 += a1[m] * bm;
                }
                if (j <= i0 || i0 == B) M[i0 * SM + j] -= t0;
                if (two && (j <= i0 + 1 || i0 + 1 == B)) M[(i0 + 1) * SM + j] -= t1;
            }
        }
        __syncthreads();
    }
}

// Backward substitution L^T x = z (z in x on entry), panel by panel from the bottom.
template <int B, int SM, typename T>
__device__ void cta_backsolve(const T *M, const T *invd, T *x) {
    constexpr int NB = B / 8;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int p = NB - 1; p >= 0; --p) {
        const int k0 = 8 * p;
        if (tid == 0) {
            for (int j = 7; j >= 0; --j) {
                T v = x[k0 + j];
                for (int m = j + 1; m < 8; ++m) v -= M[(k0 + m) * SM + k0 + j] * x[k0 + m];
                x[k0 + j] = v * invd[k0 + j];
            }
        }
        __syncthreads();
        for (int j = tid; j < k0; j += nt) {
            T v = x[j];
#pragma unroll
            for (int m = 0; m < 8; ++m) v -= M[(k0 + m) * SM + j] * x[k0 + m];
            x[j] = v;
        }
        __syncthreads();
    }
}

// FP32 blocked Cholesky of rows 0..B-1 of M (lower part used; row stride SM must
// be = 4 mod 32 and a multiple of 4) with the right-hand side carried as row B,
// in panels of 16 columns:
//  1. the 16 x 16 diagonal block is factorised by warp 0 in registers (lane i
//     holds row k0 + i; column values are exchanged with shuffles);
//  2. the rows below it (and row B) are solved against it, x L_11^T = a, one
//     thread per row, the block read as shared-memory broadcasts;
//  3. the trailing lower triangle (and row B) is updated, M -= L_21 L_21^T: a
//     warp takes 8 rows, its lanes columns c, c + 32, ... (16-byte loads of 8
//     consecutive rows per phase, free of bank conflicts), 8 x 4 panel values
//     at a time in registers.
// On return the lower part of rows 0..B-1 holds L, row B holds z = L^{-1} rhs and
// invd[k] = 1 / L_kk.  A pivot that is not above rel * diag0[k] (or not finite)
// sets *bad.  All threads of the block call it (blockDim.x >= 128, whole warps).
template <int B, int SM>
__device__ void cta_chol16(float *M, float *invd, const float *diag0, int *bad, float rel) {
    static_assert(B % 16 == 0 && SM % 32 == 4, "panel layout");
    constexpr int P = 16, NP = B / P;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
        const int k0 = P * p;
        if (warp == 0) {
            float r[P];
            const int row = k0 + (lane & (P - 1));
#pragma unroll
            for (int j = 0; j < P; j += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(M + row * SM + k0 + j);
                r[j] = v.x; r[j + 1] = v.y; r[j + 2] = v.z; r[j + 3] = v.w;
            }
#pragma unroll
            for (int k = 0; k < P; ++k) {
                const float d = __shfl_sync(kFull, r[k], k);
                if (lane == k && (!(d > rel * diag0[k0 + k]) || !(d <= 3.0e38f))) *bad = 1;
                const float inv = rsqrtf(fmaxf(d, 1e-30f));
                const float lk = r[k] * inv;
                if (lane == k) invd[k0 + k] = inv;
                r[k] = lk;
#pragma unroll
                for (int j = k + 1; j < P; ++j) r[j] -= lk * __shfl_sync(kFull, lk, j);
            }
            if (lane < P) {
#pragma unroll
                for (int j = 0; j < P; j += 4)
                    *reinterpret_cast<float4 *>(M + row * SM + k0 + j) = make_float4(r[j], r[j + 1], r[j + 2], r[j + 3]);
            }
        }
        __syncthreads();
        const int r0 = k0 + P;
        for (int i = r0 + tid; i <= B; i += nt) {
            float x[P];
#pragma unroll
            for (int j = 0; j < P; j += 4) {
                const float4 v = *reinterpret_cast<const float4 *>(M + i * SM + k0 + j);
                x[j] = v.x; x[j + 1] = v.y; x[j + 2] = v.z; x[j + 3] = v.w;
            }
#pragma unroll
            for (int j = 0; j < P; ++j) {
#pragma unroll
                for (int m = 0; m < j; ++m) x[j] -= x[m] * M[(k0 + j) * SM + k0 + m];
                x[j] *= invd[k0 + j];
            }
#pragma unroll
            for (int j = 0; j < P; j += 4)
                *reinterpret_cast<float4 *>(M + i * SM + k0 + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
        }
        __syncthreads();
        if (r0 < B) {
            const int nrb = (B + 1 - r0 + 7) / 8;  // 8-row blocks of rows r0..B
#pragma unroll 1
            for (int rb = warp; rb < nrb; rb += nw) {
                const int i0 = r0 + 8 * rb;
                const int jend = min(i0 + 8, B);           // columns r0 .. jend-1 can be touched
                const int nc = (jend - r0 + 31) >> 5;      // 32-column groups (<= 4), warp-uniform
                float out[8][4];
#pragma unroll
                for (int a = 0; a < 8; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) out[a][c] = 0.f;
#pragma unroll
                for (int m = 0; m < P; m += 4) {
                    float4 av[8];
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const int i = min(i0 + a, B);
                        av[a] = *reinterpret_cast<const float4 *>(M + i * SM + k0 + m);
                    }
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (c >= nc) break;
                        const int j = min(r0 + lane + 32 * c, B - 1);
                        const float4 bv = *reinterpret_cast<const float4 *>(M + j * SM + k0 + m);
#pragma unroll
                        for (int a = 0; a < 8; ++a)
                            out[a][c] += av[a].x * bv.x + av[a].y * bv.y + av[a].z * bv.z + av[a].w * bv.w;
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (c >= nc) break;
                    const int j = r0 + lane + 32 * c;
#pragma unroll
                    for (int a = 0; a < 8; ++a) {
                        const int i = i0 + a;
                        if (i <= B && j < B && (j <= i || i == B)) M[i * SM + j] -= out[a][c];
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Forward substitution L z = g for a factor left by cta_chol16 (g in x on entry),
// 16-blocks from the top: warp 0 solves the block with shuffles, then all
// threads remove its contribution from the entries below it.
template <int B, int SM>
__device__ void cta_forward16(const float *M, const float *invd, float *x) {
    constexpr int P = 16, NP = B / P;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int p = 0; p < NP; ++p) {
        const int k0 = P * p;
        if (warp == 0) {
            const int m = lane & (P - 1);
            float z = x[k0 + m];
#pragma unroll
            for (int j = 0; j < P; ++j) {
                const float zj = __shfl_sync(kFull, z * invd[k0 + j], j);
                if (m > j) z -= M[(k0 + m) * SM + k0 + j] * zj;
                else if (m == j) z = zj;
            }
            if (lane < P) x[k0 + m] = z;
        }
        __syncthreads();
        for (int q = k0 + P + tid; q < B; q += nt) {
            float v = x[q];
#pragma unroll
            for (int j = 0; j < P; j += 4) {
                const float4 l = *reinterpret_cast<const float4 *>(M + q * SM + k0 + j);
                v -= l.x * x[k0 + j] + l.y * x[k0 + j + 1] + l.z * x[k0 + j + 2] + l.w * x[k0 + j + 3];
            }
            x[q] = v;
        }
        __syncthreads();
    }
}

// Backward substitution L^T x = z for the factor left by cta_chol16 (z in x on
// entry), 16-blocks from the bottom: warp 0 solves the block with shuffles, then
// all threads remove its contribution from the entries above it.
template <int B, int SM>
__device__ void cta_backsolve16(const float *M, const float *invd, float *x) {
    constexpr int P = 16, NP = B / P;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
#pragma unroll 1
    for (int p = NP - 1; p >= 0; --p) {
        const int k0 = P * p;
        if (warp == 0) {
            const int m = lane & (P - 1);
            float z = x[k0 + m];
#pragma unroll
            for (int j = P - 1; j >= 0; --j) {
                const float xj = __shfl_sync(kFull, z * invd[k0 + j], j);
                if (m < j) z -= M[(k0 + j) * SM + k0 + m] * xj;
                else if (m == j) z = xj;
            }
            if (lane < P) x[k0 + m] = z;
        }
        __syncthreads();
        for (int q = tid; q < k0; q += nt) {
            float v = x[q];
#pragma unroll
            for (int j = 0; j < P; ++j) v -= M[(k0 + j) * SM + q] * x[k0 + j];
            x[q] = v;
        }
        __syncthreads();
    }
}

// Adds alpha0 G_pipi + lambda I to rows 0..B-1 of M (lower part) and R_r to row B;
// records the diagonal in diag0.
template <int B, int SM, typename T, bool WITH_R = true>
__device__ void cta_dense_terms(const StepArgs &a, T *M, T *diag0, int row, T lam) {
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int i = e / B, j = e % B;
        if (j > i) continue;
        T v = M[i * SM + j] + (T)a.alpha0 * (T)a.G[(int64_t)(a.p0 + i) * B + j];
        if (i == j) {
            v += lam;
            diag0[i] = v;
        }
        M[i * SM + j] = v;
    }
    if (WITH_R)
        for (int j = threadIdx.x; j < B; j += blockDim.x) M[B * SM + j] += (T)a.R[(int64_t)row * B + j];
}

// Gather `cnt` slices starting at CSR position s0 into buf (all threads).
template <int B>
__device__ __forceinline__ void cta_gather(const StepArgs &a, int64_t s0, int cnt, float *buf) {
    constexpr int V = B / 4, SB = CtaCfg<B>::SB;
    for (int f = threadIdx.x; f < cnt * V; f += blockDim.x) {
        const int k = f / V, v = f % V;
        const int64_t c = a.idx[s0 + k];
        cp_async16(buf + k * SB + 4 * v, a.F + c * a.d + a.p0 + 4 * v);
    }
}

// Residual update e_s -= <x, f_{c_s,pi}> for the CSR range [s0, s0 + len):
// slices staged 32 at a time, one warp per interaction with lanes splitting b.
template <int B, bool PERM>
__device__ void cta_residual_update(const StepArgs &a, int64_t s0, int len, const float *x,
                                    float *buf) {
    constexpr int CH = CtaCfg<B>::CH, SB = CtaCfg<B>::SB;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c0 = 0; c0 < len; c0 += CH) {
        const int cnt = min(CH, len - c0);
        cta_gather<B>(a, s0 + c0, cnt, buf);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        for (int k = warp; k < cnt; k += nw) {
            float t = 0.f;
#pragma unroll
            for (int j = lane; j < B; j += 32) t += x[j] * buf[k * SB + j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == 0) {
                const int64_t s = s0 + c0 + k;
                const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                a.e[q] -= t;
            }
        }
        __syncthreads();
    }
}

// Residual update after the solve, using what the accumulation left staged: the
// last two chunks of the row are still in the two staging buffers (chunk ch in
// buffer ch & 1), so they are used first; chunks 0 .. nch-3 are gathered again,
// double-buffered.  One warp per interaction, lanes splitting b.
template <int B, bool PERM>
__device__ void cta_residual_update2(const StepArgs &a, int64_t s0, int len, int nch, const float *x,
                                     float *buf0) {
    constexpr int CH = CtaCfg<B>::CH, SB = CtaCfg<B>::SB, BUF = CtaCfg<B>::BUF;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    float xr[B / 32];
#pragma unroll
    for (int m = 0; m < B / 32; ++m) xr[m] = x[lane + 32 * m];
    auto process = [&](int ch, const float *bp) {
        const int cnt = min(CH, len - ch * CH);
        for (int k = warp; k < cnt; k += nw) {
            float t = 0.f;
#pragma unroll
            for (int m = 0; m < B / 32; ++m) t += xr[m] * bp[k * SB + lane + 32 * m];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == 0) {
                const int64_t s = s0 + (int64_t)ch * CH + k;
                const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                a.e[q] -= t;
            }
        }
    };
    for (int ch = nch - 1; ch >= 0 && ch >= nch - 2; --ch) process(ch, buf0 + (ch & 1) * BUF);
    if (nch <= 2) return;
    __syncthreads();  // the staged chunks are consumed before they are overwritten
    cta_gather<B>(a, s0, CH, buf0);
    cp_async_commit();
    for (int ch = 0; ch <= nch - 3; ++ch) {
        cp_async_wait_all();
        __syncthreads();
        if (ch + 1 <= nch - 3) {
            cta_gather<B>(a, s0 + (int64_t)(ch + 1) * CH, CH, buf0 + ((ch + 1) & 1) * BUF);
            cp_async_commit();
        }
        process(ch, buf0 + (ch & 1) * BUF);
    }
}

// FP64 re-solve of queued rows: statistics accumulated from scratch in FP64 by
// the tile owners (one group, reading slices straight from global memory), the
// blocked Cholesky in FP64, apply and residual update.
// Above b = 128 the FP64 system (B + 1)^2 doubles does not fit shared memory;
// it lives in a per-block slice of a.retry_ws instead.
template <int B>
constexpr bool retry_in_global() { return B > 128; }

template <int B, bool PERM, bool HAS_A, bool DIRECT = false>
__global__ void __launch_bounds__(CtaCfg<B>::THREADS) k_retry_cta(const StepArgs a) {
    using C = CtaCfg<B>;
    constexpr int SM = B + 1;
    extern __shared__ float4 smem4[];
    float *buf = reinterpret_cast<float *>(smem4);  // CH x SB staging for the residual update
    double *sm_after = reinterpret_cast<double *>(buf + C::BUF);
    double *M = retry_in_global<B>() ? a.retry_ws + (int64_t)blockIdx.x * (B + 1) * SM : sm_after;
    double *diag0 = retry_in_global<B>() ? sm_after : M + (B + 1) * SM;
    double *invd = diag0 + B;
    double *xd = invd + B;
    int *flag = reinterpret_cast<int *>(xd + B);
    float *xf = reinterpret_cast<float *>(flag + 4);
    const int tid = threadIdx.x;
    int ti = 0, tj = 0;
    tri_index(tid % C::NTL, ti, tj);
    const int count = *(volatile int *)a.retry;
    for (int q = blockIdx.x; q < count; q += gridDim.x) {
        const int row = a.retry[1 + q];
        const int64_t beg = a.ptr[row], end = a.ptr[row + 1];
        if (tid < C::NTL) {
            double acc[8][8], g[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                g[i] = 0.0;
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.0;
            }
            for (int64_t s = beg; s < end; ++s) {
                const int64_t r = PERM ? (int64_t)a.pos[s] : s;
                const float *f = a.F + (int64_t)a.idx[s] * a.d + a.p0;
                const double al = HAS_A ? (double)a.alpha[r] : 1.0;
                const double er = al * (double)(DIRECT ? (a.y ? a.y[r] : 1.f) : a.e[r]);
                double xa[8], xb[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) { xa[i] = f[8 * ti + i]; xb[i] = f[8 * tj + i]; }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    g[i] += er * xa[i];
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] += al * xa[i] * xb[j];
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 8; ++j) M[(8 * ti + i) * SM + 8 * tj + j] = acc[i][j];
                if (tj == 0) M[B * SM + 8 * ti + i] = g[i];
            }
        }
        if (tid == 0) flag[1] = 0;
        __syncthreads();
        const double lam = (double)a.lambda * (1.0 + (double)a.nu * (double)(end - beg));
        cta_dense_terms<B, SM, double, !DIRECT>(a, M, diag0, row, lam);
        __syncthreads();
        cta_cholesky<B, SM, double>(M, invd, diag0, &flag[1], 1e-13);
        bool ok = !flag[1];
        if (ok) {
            for (int j = tid; j < B; j += blockDim.x) xd[j] = M[B * SM + j];
            __syncthreads();
            cta_backsolve<B, SM, double>(M, invd, xd);
            for (int j = 0; j < B; ++j) ok = ok && isfinite(xd[j]);
        }
        if (!ok) {
            if (tid == 0) atomicAdd((unsigned long long *)&a.stats[1], 1ull);
            __syncthreads();
            continue;
        }
        for (int j = tid; j < B; j += blockDim.x) {
            xf[j] = (float)xd[j];
            if (DIRECT) set_value(a.X, a.Xh, a.Xl, (int64_t)row * a.d + a.p0 + j, xf[j]);
            else apply_delta(a.X, a.Xh, a.Xl, (int64_t)row * a.d + a.p0 + j, xf[j]);
        }
        __syncthreads();
        if (!DIRECT) cta_residual_update<B, PERM>(a, beg, (int)(end - beg), xf, buf);
        if (tid == 0) atomicAdd((unsigned long long *)&a.stats[0], 1ull);
    }
}

template <int B>
constexpr int retry_cta_smem() {
    return CtaCfg<B>::BUF * 4 + ((retry_in_global<B>() ? 0 : (B + 1) * (B + 1)) + 3 * B) * 8 + 16 + B * 4;
}
// Blocks of the FP64 re-solve kernel, and its global workspace (doubles) above b = 128.
constexpr int kRetryBlocks = 76;
template <int B>
constexpr int64_t retry_ws_doubles() { return retry_in_global<B>() ? (int64_t)kRetryBlocks * (B + 1) * (B + 1) : 0; }

}  // namespace ials
