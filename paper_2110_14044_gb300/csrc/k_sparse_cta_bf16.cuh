// Sparse block step of Algorithm 3 on BF16 tensor cores for block sizes B = 64
// and 128 (precision IALS_PREC_BF16, one CTA per task).
//
// The statistics of a row are the product [A_r | g_r] = X^T [X | e] of
// k_sparse_bf16.cuh (Eqs. 11-12): staged hi/lo slices, mma.sync.m16n8k16 with
// compensated products hi*hi + hi*lo + lo*hi, the residual riding as column B
// of the staged tile.  At these block sizes the (m16 x n8) tiles on or below
// the diagonal of A_r (MT (MT + 1) of them, MT = B / 16) are spread over MT
// warps: warp w takes half of the tiles of the row pair (w / 2, MT - 1 - w / 2),
// MT + 1 tiles, so every warp does the same number of products.  Each warp's
// tile list is fixed at compile time (the kernel dispatches on the warp index),
// which keeps its fragments and accumulators in registers; a warp loads only
// the 16-column blocks its tiles touch.  For a whole row the accumulators start
// from the dense terms alpha0 G_pipi + lambda_r I and R_r.  The fragments go to
// a shared FP32 matrix, from which the owners of the 8 x 8 tiles of
// k_sparse_rc.cuh take them into registers for its blocked Cholesky and
// substitutions; the residual update uses the staged (hi + lo) slices.
#pragma once

#include "k_sparse_bf16.cuh"
#include "k_sparse_cta.cuh"
#include "k_sparse_rc.cuh"

namespace ials {

template <int B>
struct CtaBfCfg {
    static constexpr int MT = B / 16;       // 16-row tiles of A_r
    static constexpr int WARPS = MT;        // MT / 2 row pairs, two warps each
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int NPT = MT + 1;      // (m16 x n8) tiles per warp
    static constexpr int SBH = B + 8;       // bf16 row stride of a staged tile; column B holds the residual
    static constexpr int CH = 32;           // interactions per chunk
    static constexpr int TILE = CH * SBH;   // bf16 elements of one hi (or lo) tile
    static constexpr int BUF = 2 * TILE;    // one staging buffer: hi tile, then lo tile
    static constexpr int SM = B + 4;        // float row stride of the shared matrix (= 4 mod 32)
    static constexpr int M_FLOATS = (B + 1) * SM;
    static constexpr int SMEM_BYTES = 2 * BUF * 2 + (M_FLOATS + B) * 4 + 16 + 2 * CH * 4;  // + sqrt(alpha) per staged row
    static_assert(M_FLOATS >= 2 * RegChol<B>::PANEL, "the panels reuse M");
    static_assert(THREADS >= RegChol<B>::NTL, "one tile per thread");
};

// Compile-time tile list of warp W: the tiles of rows I1 = W / 2 and I2 = MT - 1 - W / 2
// (row i has tiles n = 0 .. 2 i + 1), listed row I1 first, split in two halves.
template <int B, int W>
struct CtaBfWarp {
    static constexpr int MT = B / 16, NPT = MT + 1, H = W % 2, I1 = W / 2, I2 = MT - 1 - W / 2;
    static constexpr int N1 = 2 * I1 + 2;
    __host__ __device__ static constexpr int ti(int s) { return H * NPT + s < N1 ? I1 : I2; }
    __host__ __device__ static constexpr int tn(int s) { return H * NPT + s < N1 ? H * NPT + s : H * NPT + s - N1; }
    static constexpr int GRAD = H == 0 ? I1 : I2;  // the gradient m-tile this warp forms
    __host__ __device__ static constexpr unsigned blocks() {
        unsigned m = 1u << GRAD;
        for (int s = 0; s < NPT; ++s) m |= (1u << ti(s)) | (1u << (tn(s) >> 1));
        return m;
    }
};

// One k-step (16 staged interactions) of warp W's products.
template <int B, int W>
__device__ __forceinline__ void cta_bf_kstep(float (&acc)[CtaBfCfg<B>::NPT][4], float (&gac)[4],
                                             const __nv_bfloat16 *th, const __nv_bfloat16 *tl, int ks, int lane) {
    using C = CtaBfCfg<B>;
    using WT = CtaBfWarp<B, W>;
    constexpr int MT = C::MT, SBH = C::SBH;
    constexpr unsigned MASK = WT::blocks();
    const int mj = lane >> 3, mr = lane & 7;
    unsigned Rh[MT][4], Rl[MT][4], E[4];
#pragma unroll
    for (int g = 0; g < MT; ++g) {
        if ((MASK >> g) & 1u) {
            const int off = (ks * 16 + (mj >> 1) * 8 + mr) * SBH + g * 16 + (mj & 1) * 8;
            ldsm_x4_t(Rh[g], th + off);
            ldsm_x4_t(Rl[g], tl + off);
        }
    }
    ldsm_x4_t(E, (mj < 2 ? th : tl) + (ks * 16 + (mj & 1) * 8 + mr) * SBH + B);
#pragma unroll
    for (int s = 0; s < C::NPT; ++s) {
        const int i = WT::ti(s), n = WT::tn(s), g2 = n >> 1, h = n & 1;
        mma_bf16(acc[s], Rh[i], Rh[g2][h], Rh[g2][h + 2]);
        mma_bf16(acc[s], Rh[i], Rl[g2][h], Rl[g2][h + 2]);
        mma_bf16(acc[s], Rl[i], Rh[g2][h], Rh[g2][h + 2]);
    }
    mma_bf16(gac, Rh[WT::GRAD], E[0], E[1]);
    mma_bf16(gac, Rh[WT::GRAD], E[2], E[3]);
    mma_bf16(gac, Rl[WT::GRAD], E[0], E[1]);
}

// Warp W's accumulators -> rows/columns of the shared matrix M; gradient -> row B.
template <int B, int W>
__device__ __forceinline__ void cta_bf_store(const float (&acc)[CtaBfCfg<B>::NPT][4], const float (&gac)[4],
                                             float *M, int lane) {
    using C = CtaBfCfg<B>;
    using WT = CtaBfWarp<B, W>;
    constexpr int SM = C::SM;
    const int r = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
    for (int s = 0; s < C::NPT; ++s) {
        const int i = WT::ti(s), n = WT::tn(s);
        *reinterpret_cast<float2 *>(M + (16 * i + r) * SM + 8 * n + c2) = make_float2(acc[s][0], acc[s][1]);
        *reinterpret_cast<float2 *>(M + (16 * i + r + 8) * SM + 8 * n + c2) = make_float2(acc[s][2], acc[s][3]);
    }
    if ((lane & 3) == 0) {
        M[B * SM + 16 * WT::GRAD + r] = gac[0];
        M[B * SM + 16 * WT::GRAD + r + 8] = gac[2];
    }
}

// Whole rows: warp W's accumulators start from alpha0 G_pipi + lambda_r I (its
// tiles) and the gradient accumulator from R_r (column 0 of the E tile).
template <int B, int W>
__device__ __forceinline__ void cta_bf_init(float (&acc)[CtaBfCfg<B>::NPT][4], float (&gac)[4], const StepArgs &a,
                                            int row, float lam, int lane) {
    using C = CtaBfCfg<B>;
    using WT = CtaBfWarp<B, W>;
    const int r = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
    for (int s = 0; s < C::NPT; ++s) {
        const int i = WT::ti(s), n = WT::tn(s);
        const int r0 = 16 * i + r, r1 = r0 + 8, c = 8 * n + c2;
        const float2 g0 = *reinterpret_cast<const float2 *>(a.G + (int64_t)(a.p0 + r0) * B + c);
        const float2 g1 = *reinterpret_cast<const float2 *>(a.G + (int64_t)(a.p0 + r1) * B + c);
        acc[s][0] = a.alpha0 * g0.x + (r0 == c ? lam : 0.f);
        acc[s][1] = a.alpha0 * g0.y + (r0 == c + 1 ? lam : 0.f);
        acc[s][2] = a.alpha0 * g1.x + (r1 == c ? lam : 0.f);
        acc[s][3] = a.alpha0 * g1.y + (r1 == c + 1 ? lam : 0.f);
    }
    if ((lane & 3) == 0) {
        gac[0] = a.R[(int64_t)row * B + 16 * WT::GRAD + r];
        gac[2] = a.R[(int64_t)row * B + 16 * WT::GRAD + r + 8];
    }
}

template <int B>
__device__ __forceinline__ void cta_bf_init_any(int warp, float (&acc)[CtaBfCfg<B>::NPT][4], float (&gac)[4],
                                                const StepArgs &a, int row, float lam, int lane) {
    if constexpr (B == 64) {
        switch (warp) {
            case 0: cta_bf_init<B, 0>(acc, gac, a, row, lam, lane); break;
            case 1: cta_bf_init<B, 1>(acc, gac, a, row, lam, lane); break;
            case 2: cta_bf_init<B, 2>(acc, gac, a, row, lam, lane); break;
            default: cta_bf_init<B, 3>(acc, gac, a, row, lam, lane); break;
        }
    } else {
        switch (warp) {
            case 0: cta_bf_init<B, 0>(acc, gac, a, row, lam, lane); break;
            case 1: cta_bf_init<B, 1>(acc, gac, a, row, lam, lane); break;
            case 2: cta_bf_init<B, 2>(acc, gac, a, row, lam, lane); break;
            case 3: cta_bf_init<B, 3>(acc, gac, a, row, lam, lane); break;
            case 4: cta_bf_init<B, 4>(acc, gac, a, row, lam, lane); break;
            case 5: cta_bf_init<B, 5>(acc, gac, a, row, lam, lane); break;
            case 6: cta_bf_init<B, 6>(acc, gac, a, row, lam, lane); break;
            default: cta_bf_init<B, 7>(acc, gac, a, row, lam, lane); break;
        }
    }
}

template <int B>
__device__ __forceinline__ void cta_bf_kstep_any(int warp, float (&acc)[CtaBfCfg<B>::NPT][4], float (&gac)[4],
                                                 const __nv_bfloat16 *th, const __nv_bfloat16 *tl, int ks,
                                                 int lane) {
    if constexpr (B == 64) {
        switch (warp) {
            case 0: cta_bf_kstep<B, 0>(acc, gac, th, tl, ks, lane); break;
            case 1: cta_bf_kstep<B, 1>(acc, gac, th, tl, ks, lane); break;
            case 2: cta_bf_kstep<B, 2>(acc, gac, th, tl, ks, lane); break;
            default: cta_bf_kstep<B, 3>(acc, gac, th, tl, ks, lane); break;
        }
    } else {
        switch (warp) {
            case 0: cta_bf_kstep<B, 0>(acc, gac, th, tl, ks, lane); break;
            case 1: cta_bf_kstep<B, 1>(acc, gac, th, tl, ks, lane); break;
            case 2: cta_bf_kstep<B, 2>(acc, gac, th, tl, ks, lane); break;
            case 3: cta_bf_kstep<B, 3>(acc, gac, th, tl, ks, lane); break;
            case 4: cta_bf_kstep<B, 4>(acc, gac, th, tl, ks, lane); break;
            case 5: cta_bf_kstep<B, 5>(acc, gac, th, tl, ks, lane); break;
            case 6: cta_bf_kstep<B, 6>(acc, gac, th, tl, ks, lane); break;
            default: cta_bf_kstep<B, 7>(acc, gac, th, tl, ks, lane); break;
        }
    }
}

template <int B>
__device__ __forceinline__ void cta_bf_store_any(int warp, const float (&acc)[CtaBfCfg<B>::NPT][4],
                                                 const float (&gac)[4], float *M, int lane) {
    if constexpr (B == 64) {
        switch (warp) {
            case 0: cta_bf_store<B, 0>(acc, gac, M, lane); break;
            case 1: cta_bf_store<B, 1>(acc, gac, M, lane); break;
            case 2: cta_bf_store<B, 2>(acc, gac, M, lane); break;
            default: cta_bf_store<B, 3>(acc, gac, M, lane); break;
        }
    } else {
        switch (warp) {
            case 0: cta_bf_store<B, 0>(acc, gac, M, lane); break;
            case 1: cta_bf_store<B, 1>(acc, gac, M, lane); break;
            case 2: cta_bf_store<B, 2>(acc, gac, M, lane); break;
            case 3: cta_bf_store<B, 3>(acc, gac, M, lane); break;
            case 4: cta_bf_store<B, 4>(acc, gac, M, lane); break;
            case 5: cta_bf_store<B, 5>(acc, gac, M, lane); break;
            case 6: cta_bf_store<B, 6>(acc, gac, M, lane); break;
            default: cta_bf_store<B, 7>(acc, gac, M, lane); break;
        }
    }
}

// Gather the hi and lo slices of interactions [s0, s0 + cnt) into (th, tl); all threads.
template <int B>
__device__ __forceinline__ void cta_bf_gather(const StepArgs &a, int64_t s0, int cnt, __nv_bfloat16 *th,
                                              __nv_bfloat16 *tl) {
    constexpr int HC = B / 8, SBH = CtaBfCfg<B>::SBH;  // 16-byte chunks per hi slice
    for (int f = threadIdx.x; f < cnt * 2 * HC; f += blockDim.x) {
        const int k = f / (2 * HC), v = f % (2 * HC), half = v / HC, vc = v % HC;
        const int64_t c = a.idx[s0 + k];
        cp_async16((half ? tl : th) + k * SBH + vc * 8, (half ? a.Fl : a.Fh) + c * a.d + a.p0 + vc * 8);
    }
}

template <int B, bool PERM, bool DIRECT, bool HAS_A>
__global__ void __launch_bounds__(CtaBfCfg<B>::THREADS, 2) k_sparse_cta_bf16(const StepArgs a) {
    using C = CtaBfCfg<B>;
    constexpr int SBH = C::SBH, CH = C::CH, SM = C::SM, NPT = C::NPT;
    extern __shared__ float4 smem4[];
    __nv_bfloat16 *bufs = reinterpret_cast<__nv_bfloat16 *>(smem4);  // buffer bi: hi at bufs + bi * BUF, lo + TILE
    float *M = reinterpret_cast<float *>(bufs + 2 * C::BUF);
    float *xv = M + C::M_FLOATS;
    int *flag = reinterpret_cast<int *>(xv + B);  // [0] next task, [1] bad pivot
    float *sal = reinterpret_cast<float *>(flag + 4);  // weighted data: sqrt(alpha) of staged row k in buffer bi
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x, nw = nt >> 5;
    const bool own = tid < RegChol<B>::NTL;
    int ti = 0, tj = 0;
    tri_index(tid % RegChol<B>::NTL, ti, tj);
    for (int i = tid; i < 2 * C::BUF * 2 / 16; i += nt)
        reinterpret_cast<uint4 *>(bufs)[i] = make_uint4(0u, 0u, 0u, 0u);  // padding columns stay zero
    if (tid == 0) flag[0] = atomicAdd(a.counter, 1);  // the next task is fetched while one runs
    for (;;) {
        __syncthreads();
        const int tsk = flag[0];
        if (tsk >= a.n_tasks) break;
        __syncthreads();  // every thread has read flag[0]
        if (tid == 0) flag[0] = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float acc[NPT][4], gac[4];
#pragma unroll
        for (int s = 0; s < NPT; ++s)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[s][q] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) gac[q] = 0.f;
        const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
        if (tk.slot < 0) {
            cta_bf_init_any<B>(warp, acc, gac, a, tk.row, lam, lane);
            if (DIRECT) {  // Eq. 3: the right-hand side is sum alpha y f, no row term
#pragma unroll
                for (int q = 0; q < 4; ++q) gac[q] = 0.f;
            }
        }
        // chunk j into buffer bi: residual column (hi, lo), zero rows up to the next
        // multiple of 16, and the slices
        auto issue = [&](int j, int bi) {
            const int cnt = min(CH, tk.len - j * CH);
            __nv_bfloat16 *th = bufs + bi * C::BUF, *tl = th + C::TILE;
            const int rows16 = (cnt + 15) & ~15;
            for (int r = tid; r < rows16; r += nt) {
                if (r < cnt) {
                    const int64_t s = tk.begin + (int64_t)j * CH + r;
                    const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                    float e = DIRECT ? (a.y ? a.y[q] : 1.f) : a.e[q];
                    if (HAS_A) {  // weighted data: row and residual (label) times sqrt(alpha)
                        const float sa = sqrtf(a.alpha[q]);
                        sal[bi * CH + r] = sa;
                        e *= sa;
                    }
                    const __nv_bfloat16 h = __float2bfloat16_rn(e);
                    th[r * SBH + B] = h;
                    tl[r * SBH + B] = __float2bfloat16_rn(e - __bfloat162float(h));
                } else {
#pragma unroll
                    for (int v = 0; v < SBH / 8; ++v) {
                        reinterpret_cast<uint4 *>(th + r * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                        reinterpret_cast<uint4 *>(tl + r * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                    }
                }
            }
            cta_bf_gather<B>(a, tk.begin + (int64_t)j * CH, cnt, th, tl);
            cp_async_commit();
        };
        if (nch > 0) issue(0, 0);
        for (int ch = 0; ch < nch; ++ch) {
            const int bi = ch & 1;
            cp_async_wait_all();
            __syncthreads();
            if (ch + 1 < nch) issue(ch + 1, bi ^ 1);
            const int cnt = min(CH, tk.len - ch * CH);
            const __nv_bfloat16 *th = bufs + bi * C::BUF, *tl = th + C::TILE;
            if (HAS_A) {  // eight threads per staged row, B / 8 values each
                __nv_bfloat16 *wh = bufs + bi * C::BUF, *wl = wh + C::TILE;
                for (int t = tid; t < cnt * 8; t += nt) {
                    const int rr = t >> 3, part = t & 7;
                    const float sa = sal[bi * CH + rr];
#pragma unroll
                    for (int v = 0; v < B / 64; ++v) {
                        uint4 *ph = reinterpret_cast<uint4 *>(wh + rr * SBH + part * (B / 8)) + v;
                        uint4 *pl = reinterpret_cast<uint4 *>(wl + rr * SBH + part * (B / 8)) + v;
                        uint4 hv = *ph, lv = *pl;
                        __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(&hv);
                        __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(&lv);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float2 hf = __bfloat1622float2(h2[q]), lf = __bfloat1622float2(l2[q]);
                            const float x0 = (hf.x + lf.x) * sa, x1 = (hf.y + lf.y) * sa;
                            const __nv_bfloat162 nh = __floats2bfloat162_rn(x0, x1);
                            const float2 nhf = __bfloat1622float2(nh);
                            h2[q] = nh;
                            l2[q] = __floats2bfloat162_rn(x0 - nhf.x, x1 - nhf.y);
                        }
                        *ph = hv;
                        *pl = lv;
                    }
                }
                __syncthreads();
            }
            const int ksteps = (cnt + 15) >> 4;
            for (int ks = 0; ks < ksteps; ++ks) cta_bf_kstep_any<B>(warp, acc, gac, th, tl, ks, lane);
        }
        cta_bf_store_any<B>(warp, acc, gac, M, lane);
        __syncthreads();
        if (tk.slot >= 0) {  // a chunk of a long row: store the partial statistics
            float *P = a.part + (int64_t)tk.slot * (B * B + B);
            for (int e = tid; e < B * B; e += nt) {
                const int i = e / B, j = e % B;
                P[e] = j <= i ? M[i * SM + j] : 0.f;
            }
            for (int j = tid; j < B; j += nt) P[B * B + j] = M[B * SM + j];
            continue;
        }
        // the solve of k_sparse_rc.cuh: owners take their 8 x 8 tile of the system (dense
        // terms are in already) into registers; M is then free and holds the panels
        float t[8][8], inv[8];
        if (own) {
#pragma unroll
            for (int i = 0; i < 8; ++i) load_seg<8>(M + (8 * ti + i) * SM + 8 * tj, t[i]);
        }
        for (int j = tid; j < B; j += nt) xv[j] = M[B * SM + j];
        if (tid == 0) flag[1] = a.force_fp64 ? 1 : 0;
        __syncthreads();
        rc_factor<B>(t, inv, ti, tj, own, M, xv, &flag[1], 1e-5f);
        if (flag[1]) {  // CTA-uniform: queue the row for the FP64 re-solve
            if (tid == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        rc_backsolve<B>(t, inv, ti, tj, own, xv);
        bool fin = true;
        for (int j = tid; j < B; j += nt) fin = fin && isfinite(xv[j]);
        if (!__syncthreads_and(fin)) {
            if (tid == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        if (DIRECT) {  // the solution is the row itself
            for (int j = tid; j < B; j += nt) set_value(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + j, xv[j]);
            continue;
        }
        for (int j = tid; j < B; j += nt) apply_delta(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + j, xv[j]);
        // residual update e_s -= <delta, f_s> with f_s = hi + lo from the staged tiles:
        // the last two chunks are still staged, the others are gathered again
        float xr[B / 32];
#pragma unroll
        for (int m = 0; m < B / 32; ++m) xr[m] = xv[lane + 32 * m];
        auto process = [&](int ch, const __nv_bfloat16 *th) {
            const __nv_bfloat16 *tl = th + C::TILE;
            const int cnt = min(CH, tk.len - ch * CH);
            for (int k = warp; k < cnt; k += nw) {
                float t = 0.f;
#pragma unroll
                for (int m = 0; m < B / 32; ++m)
                    t += xr[m] * (__bfloat162float(th[k * SBH + lane + 32 * m]) +
                                  __bfloat162float(tl[k * SBH + lane + 32 * m]));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
                if (lane == 0) {
                    const int64_t s = tk.begin + (int64_t)ch * CH + k;
                    const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                    a.e[q] -= t;
                }
            }
        };
        if (HAS_A) {  // the staged chunks were scaled: every chunk is gathered again, unscaled
            for (int ch = 0; ch < nch; ++ch) {
                __syncthreads();
                cta_bf_gather<B>(a, tk.begin + (int64_t)ch * CH, min(CH, tk.len - ch * CH), bufs, bufs + C::TILE);
                cp_async_commit();
                cp_async_wait_all();
                __syncthreads();
                process(ch, bufs);
            }
            continue;
        }
        for (int ch = nch - 1; ch >= 0 && ch >= nch - 2; --ch) process(ch, bufs + (ch & 1) * C::BUF);
        if (nch > 2) {
            __syncthreads();  // the staged chunks are consumed before they are overwritten
            cta_bf_gather<B>(a, tk.begin, CH, bufs, bufs + C::TILE);
            cp_async_commit();
            for (int ch = 0; ch <= nch - 3; ++ch) {
                cp_async_wait_all();
                __syncthreads();
                if (ch + 1 <= nch - 3) {
                    __nv_bfloat16 *nb = bufs + ((ch + 1) & 1) * C::BUF;
                    cta_bf_gather<B>(a, tk.begin + (int64_t)(ch + 1) * CH, CH, nb, nb + C::TILE);
                    cp_async_commit();
                }
                process(ch, bufs + (ch & 1) * C::BUF);
            }
        }
    }
}

// Whole sparse part of a BF16 block-side step at B = 64, 128: the CTA kernel,
// then long rows (slot sums and the register-tile solve), their residual
// update (not for DIRECT), FP64 retry.
template <int B, bool PERM, bool DIRECT, bool HAS_A>
cudaError_t launch_sparse_cta_bf16_all(const StepArgs &a, cudaStream_t s) {
    using C = CtaBfCfg<B>;
    using CF = CtaCfg<B>;
    static bool attr_done = false;
    static int per_sm = 0;
    if (!attr_done) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_sparse_cta_bf16<B, PERM, DIRECT, HAS_A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      C::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_split_solve_rc<B, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      RcCfg<B>::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_retry_cta<B, PERM, HAS_A, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      retry_cta_smem<B>())) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse_cta_bf16<B, PERM, DIRECT, HAS_A>, C::THREADS,
                                                               C::SMEM_BYTES)) != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    if (a.n_tasks > 0) {
        int grid = 152 * per_sm;
        if (grid > a.n_tasks) grid = a.n_tasks;
        prof_mark(a.prof, K_SPARSE, s);
        k_sparse_cta_bf16<B, PERM, DIRECT, HAS_A><<<grid, C::THREADS, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 4 ? a.n_split : 152 * 4;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve_rc<B, DIRECT><<<g2, RcCfg<B>::THREADS, RcCfg<B>::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (!DIRECT) {  // always called: the first call sizes the grid, outside any stream capture
        const cudaError_t e = launch_split_resid_reg_bf16<B, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry_cta<B, PERM, HAS_A, DIRECT><<<kRetryBlocks, CF::THREADS, retry_cta_smem<B>(), s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

template <int B, bool HAS_A>
cudaError_t launch_sparse_cta_bf16_weights(const StepArgs &a, cudaStream_t s) {
    if (a.direct)
        return a.pos ? launch_sparse_cta_bf16_all<B, true, true, HAS_A>(a, s)
                     : launch_sparse_cta_bf16_all<B, false, true, HAS_A>(a, s);
    return a.pos ? launch_sparse_cta_bf16_all<B, true, false, HAS_A>(a, s)
                 : launch_sparse_cta_bf16_all<B, false, false, HAS_A>(a, s);
}

template <int B>
cudaError_t launch_sparse_cta_bf16_dispatch(const StepArgs &a, cudaStream_t s) {
    return a.alpha ? launch_sparse_cta_bf16_weights<B, true>(a, s) : launch_sparse_cta_bf16_weights<B, false>(a, s);
}

}  // namespace ials
