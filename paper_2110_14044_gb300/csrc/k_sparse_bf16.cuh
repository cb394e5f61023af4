// Sparse block step of Algorithm 3 on BF16 tensor cores (precision IALS_PREC_BF16),
// block sizes B = 16 and 32, one warp per task.
//
// The statistics of a row (Eqs. 11-12) are one small GEMM: with X the staged
// slices (one row per interaction, B coordinates) and e the residuals,
//     [A_r | g_r] = X^T [X | e]
// so the residual rides as one extra column of the staged tile and the
// gradient falls out of the same mma.sync.m16n8k16 (BF16 in, FP32 accumulate).
// Every operand is split x = hi + lo (hi = bf16(x), lo = bf16(x - hi)) and each
// product is compensated, hi*hi + hi*lo + lo*hi, which keeps about 16 bits
// (the dropped lo*lo term is below 2^-16 relative).  Only the 16 x 8 output
// tiles on or below the diagonal are formed.  The slices come from hi/lo
// shadow copies of the factors kept in HBM (updated wherever a delta is
// applied) and are gathered with cp.async into two staging buffers.  One
// ldmatrix.x4.trans of a 16 x 16 block serves both as the A fragment of an
// m-tile and as the B fragments of the two matching n-tiles.  The Newton solve
// is the warp Gauss-Jordan elimination with 2 x 2 pivot blocks (FP32), the
// apply that of the FP32 kernels.  The
// residual update e_s -= <delta, f_s> is again a tensor-core product: the
// staged tile times delta (split hi + lo, compensated the same way) as the
// only non-zero column of an m16n8k16 B operand.
// Weighted data: sum_s alpha_s f f^T = X~^T X~ with the rows of X~ = sqrt(alpha_s)
// f_s, and sum_s alpha_s e_s f_s = X~^T (sqrt(alpha) e), so each staged row and its
// residual are scaled by sqrt(alpha_s) (and split into hi / lo again) before the
// products; the residual update uses the slices unscaled, gathered again.
#pragma once

#include "k_sparse_impl.cuh"

namespace ials {

template <int B>
struct BfCfg {
    static constexpr int MT = B / 16;           // 16-row tiles of A_r
    static constexpr int NLOW = MT * (MT + 1);  // (m-tile, 8-column tile) pairs on/below the diagonal
    static constexpr int SBH = B + 8;           // bf16 row stride; column B holds the residual
    static constexpr int CH = 32;
    static constexpr int TILE = CH * SBH;       // bf16 elements of one hi (or lo) tile
    static constexpr int BUF_BYTES = 2 * TILE * 2;
    static constexpr int SA = B + 4;            // float row stride of the shared A_r (in buffer 1)
    static constexpr int WARP_BYTES = 2 * BUF_BYTES + B * 4 + 16 + 2 * CH * 4;  // + sqrt(alpha) per staged row
    static constexpr int WARPS = 8;
    static constexpr int SMEM_BYTES = B * B * 4 + WARPS * WARP_BYTES;
    static_assert(B * SA * 4 <= BUF_BYTES, "A_r must fit a staging buffer");
    static_assert(WARP_BYTES % 16 == 0, "alignment");
};

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// B fragments of delta (K = B coordinates, N = 8) with delta in column 0 and
// zeros elsewhere, split delta = hi + lo.  Column 0 of an m16n8k16 B fragment
// lives in lanes 0-3: register 0 holds k = 2 lane + {0, 1}, register 1 holds
// k = 2 lane + 8 + {0, 1}.
template <int B>
__device__ __forceinline__ void delta_frags(const float *v, int lane, unsigned (&dh)[B / 16][2],
                                            unsigned (&dl)[B / 16][2]) {
#pragma unroll
    for (int kb = 0; kb < B / 16; ++kb) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            unsigned hw = 0u, lw = 0u;
            if (lane < 4) {
                const float2 x = *reinterpret_cast<const float2 *>(v + kb * 16 + 8 * r + 2 * lane);
                const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
                const float2 hf = __bfloat1622float2(h);
                const __nv_bfloat162 l = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
                hw = *reinterpret_cast<const unsigned *>(&h);
                lw = *reinterpret_cast<const unsigned *>(&l);
            }
            dh[kb][r] = hw;
            dl[kb][r] = lw;
        }
    }
}

// Projections <delta, f_k> of the first 16 * nmt staged rows as the GEMV
// [F_hi + F_lo] [delta_hi + delta_lo] on the tensor cores (compensated, lo*lo
// dropped).  Row k's value is returned in lane k (k < 32; nmt <= 2).
template <int B>
__device__ __forceinline__ float project_mma(const __nv_bfloat16 *th, const __nv_bfloat16 *tl, int nmt,
                                             const unsigned (&dh)[B / 16][2],
                                             const unsigned (&dl)[B / 16][2], int lane) {
    constexpr int SBH = BfCfg<B>::SBH;
    const int q = lane >> 3, r8 = lane & 7;
    float out = 0.f;
#pragma unroll
    for (int ms = 0; ms < 2; ++ms) {
        if (ms >= nmt) break;
        float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kb = 0; kb < B / 16; ++kb) {
            const int off = (ms * 16 + (q & 1) * 8 + r8) * SBH + kb * 16 + (q >> 1) * 8;
            unsigned Fh[4], Fl[4];
            ldsm_x4(Fh, th + off);
            ldsm_x4(Fl, tl + off);
            mma_bf16(d, Fh, dh[kb][0], dh[kb][1]);
            mma_bf16(d, Fh, dl[kb][0], dl[kb][1]);
            mma_bf16(d, Fl, dh[kb][0], dh[kb][1]);
        }
        // column 0: lane 4 g holds rows g (d[0]) and g + 8 (d[2])
        const float v0 = __shfl_sync(kFull, d[0], 4 * r8);
        const float v2 = __shfl_sync(kFull, d[2], 4 * r8);
        if ((lane >> 4) == ms) out = (lane & 8) ? v2 : v0;
    }
    return out;
}

// Weighted data: row k (< cnt) of the staged hi / lo tiles becomes the hi / lo
// split of sqrt(alpha_k) (hi + lo); lane k takes row k.
template <int B>
__device__ __forceinline__ void scale_rows(__nv_bfloat16 *th, __nv_bfloat16 *tl, const float *sal, int cnt,
                                           int lane) {
    constexpr int SBH = BfCfg<B>::SBH;
    if (lane >= cnt) return;
    const float sa = sal[lane];
#pragma unroll
    for (int v = 0; v < B / 8; ++v) {
        uint4 hv = reinterpret_cast<uint4 *>(th + lane * SBH)[v];
        uint4 lv = reinterpret_cast<uint4 *>(tl + lane * SBH)[v];
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
        reinterpret_cast<uint4 *>(th + lane * SBH)[v] = hv;
        reinterpret_cast<uint4 *>(tl + lane * SBH)[v] = lv;
    }
}

// Gather the hi and lo slices of `cnt` interactions (column id of interaction k in lane k).
template <int B>
__device__ __forceinline__ void gather_hilo(__nv_bfloat16 *th, __nv_bfloat16 *tl,
                                            const StepArgs &a, int c_lane, int cnt, int lane) {
    constexpr int SBH = BfCfg<B>::SBH;
    constexpr int HC = B / 8;          // 16-byte chunks per hi slice
    constexpr int NCI = 2 * HC;        // per interaction (hi + lo)
    constexpr int PASSES = 32 * NCI / 32;
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
        const int f = p * 32 + lane;
        const int k = f / NCI, v = f % NCI;
        const int ck = __shfl_sync(kFull, c_lane, k);
        if (k < cnt) {
            const int half = v / HC, vc = v % HC;
            const __nv_bfloat16 *src = (half ? a.Fl : a.Fh) + (int64_t)ck * a.d + a.p0 + vc * 8;
            __nv_bfloat16 *dst = (half ? tl : th) + k * SBH + vc * 8;
            cp_async16(dst, src);
        }
    }
}

template <int B, bool PERM, bool HAS_A>
__global__ void __launch_bounds__(256, 2) k_sparse_bf16(const StepArgs a) {
    using C = BfCfg<B>;
    constexpr int SBH = C::SBH, CH = C::CH, MT = C::MT, SA = C::SA;
    extern __shared__ float4 smem4[];
    char *sm = reinterpret_cast<char *>(smem4);
    float *sGpp = reinterpret_cast<float *>(sm);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // alpha0 G_pipi, exactly symmetric, read by columns (as in the FP32 kernels)
    for (int i = threadIdx.x; i < B * B; i += blockDim.x)
        sGpp[i] = a.alpha0 * a.G[(int64_t)(a.p0 + max(i / B, i % B)) * B + min(i / B, i % B)];
    char *wb = sm + B * B * 4 + warp * C::WARP_BYTES;
    // staging buffer bi: hi tile at wb + bi * BUF_BYTES, lo tile right after it
    auto th_of = [&](int bi) { return reinterpret_cast<__nv_bfloat16 *>(wb + bi * C::BUF_BYTES); };
    float *vv = reinterpret_cast<float *>(wb + 2 * C::BUF_BYTES);
    float *sal = vv + B + 4;  // sqrt(alpha) of the rows staged in buffer bi: sal[bi * CH + k]
    for (int i = lane; i < 2 * C::BUF_BYTES / 16; i += 32)
        reinterpret_cast<uint4 *>(wb)[i] = make_uint4(0u, 0u, 0u, 0u);  // padding columns stay zero
    __syncthreads();
    float *As = reinterpret_cast<float *>(wb + C::BUF_BYTES);  // A_r and the factor copy reuse buffer 1
    WarpSmem w;
    w.v = vv;
    w.L = As;
    const int col = lane % B, sub = lane / B;
    int nxt = 0;  // lane 0: the next task index, fetched while the current task runs
    if (lane == 0) nxt = atomicAdd(a.counter, 1);
    for (;;) {
        const int tsk = __shfl_sync(kFull, nxt, 0);
        if (tsk >= a.n_tasks) break;
        if (lane == 0) nxt = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float acc[C::NLOW][4], gac[MT][4];
#pragma unroll
        for (int t = 0; t < C::NLOW; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
#pragma unroll
        for (int t = 0; t < MT; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) gac[t][q] = 0.f;
        int cB = 0;
        int64_t qB = 0;
        float eB = 0.f, aB = 1.f;
        auto load_meta = [&](int j) {
            const int cnt = min(CH, tk.len - j * CH);
            if (lane < cnt) {
                const int64_t s = tk.begin + (int64_t)j * CH + lane;
                cB = a.idx[s];
                qB = PERM ? (int64_t)a.pos[s] : s;
                eB = a.e[qB];
                if (HAS_A) aB = a.alpha[qB];
            }
        };
        auto issue = [&](int j, int bi) {
            const int cnt = min(CH, tk.len - j * CH);
            __nv_bfloat16 *th = th_of(bi), *tl = th + C::TILE;
            if (lane < cnt) {  // residual column (times sqrt(alpha) for weighted data)
                float ew = eB;
                if (HAS_A) {
                    const float sa = sqrtf(aB);
                    sal[bi * CH + lane] = sa;
                    ew *= sa;
                }
                const __nv_bfloat16 h = __float2bfloat16_rn(ew);
                th[lane * SBH + B] = h;
                tl[lane * SBH + B] = __float2bfloat16_rn(ew - __bfloat162float(h));
            } else if (lane < ((cnt + 15) & ~15)) {  // rows past the end of a short chunk: zero
#pragma unroll
                for (int v = 0; v < SBH / 8; ++v) {
                    reinterpret_cast<uint4 *>(th + lane * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                    reinterpret_cast<uint4 *>(tl + lane * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
            gather_hilo<B>(th, tl, a, cB, cnt, lane);
            cp_async_commit();
        };
        // chunk ch is staged in buffer (nch - 1 - ch) & 1, so the last chunk ends in
        // buffer 0, which the solve leaves intact: the residual update starts with it
        if (nch > 0) {
            load_meta(0);
            issue(0, (nch - 1) & 1);
            if (nch > 1) load_meta(1);
        }
        for (int ch = 0; ch < nch; ++ch) {
            const int bi = (nch - 1 - ch) & 1;
            cp_async_wait_all();
            __syncwarp();
            if (ch + 1 < nch) {
                issue(ch + 1, bi ^ 1);
                if (ch + 2 < nch) load_meta(ch + 2);
            }
            const int cnt = min(CH, tk.len - ch * CH);
            const __nv_bfloat16 *th = th_of(bi), *tl = th + C::TILE;
            if (HAS_A) {  // rows of this chunk times sqrt(alpha)
                scale_rows<B>(th_of(bi), th_of(bi) + C::TILE, sal + bi * CH, cnt, lane);
                __syncwarp();
            }
            const int ksteps = (cnt + 15) >> 4;
            const int mj = lane >> 3, mr = lane & 7;
            for (int ks = 0; ks < ksteps; ++ks) {
                unsigned Rh[MT][4], Rl[MT][4], E[4];
#pragma unroll
                for (int gi = 0; gi < MT; ++gi) {
                    const int off = (ks * 16 + (mj >> 1) * 8 + mr) * SBH + gi * 16 + (mj & 1) * 8;
                    ldsm_x4_t(Rh[gi], th + off);
                    ldsm_x4_t(Rl[gi], tl + off);
                }
                {
                    const __nv_bfloat16 *base = mj < 2 ? th : tl;
                    ldsm_x4_t(E, base + (ks * 16 + (mj & 1) * 8 + mr) * SBH + B);
                }
                int t = 0;
#pragma unroll
                for (int i = 0; i < MT; ++i) {
#pragma unroll
                    for (int n = 0; n <= 2 * i + 1; ++n) {
                        const int g2 = n >> 1, h = n & 1;
                        mma_bf16(acc[t], Rh[i], Rh[g2][h], Rh[g2][h + 2]);
                        mma_bf16(acc[t], Rh[i], Rl[g2][h], Rl[g2][h + 2]);
                        mma_bf16(acc[t], Rl[i], Rh[g2][h], Rh[g2][h + 2]);
                        ++t;
                    }
                    mma_bf16(gac[i], Rh[i], E[0], E[1]);
                    mma_bf16(gac[i], Rh[i], E[2], E[3]);
                    mma_bf16(gac[i], Rl[i], E[0], E[1]);
                }
            }
            __syncwarp();
        }
        // fragments -> shared A_r (buffer 1) and gradient (vv)
        {
            int t = 0;
            const int r = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
            for (int i = 0; i < MT; ++i) {
#pragma unroll
                for (int n = 0; n <= 2 * i + 1; ++n) {
                    *reinterpret_cast<float2 *>(As + (16 * i + r) * SA + 8 * n + c2) = make_float2(acc[t][0], acc[t][1]);
                    *reinterpret_cast<float2 *>(As + (16 * i + r + 8) * SA + 8 * n + c2) = make_float2(acc[t][2], acc[t][3]);
                    if (n < 2 * i) {  // strictly below the diagonal blocks: mirror, the solver wants whole rows
                        As[(8 * n + c2) * SA + 16 * i + r] = acc[t][0];
                        As[(8 * n + c2 + 1) * SA + 16 * i + r] = acc[t][1];
                        As[(8 * n + c2) * SA + 16 * i + r + 8] = acc[t][2];
                        As[(8 * n + c2 + 1) * SA + 16 * i + r + 8] = acc[t][3];
                    }
                    ++t;
                }
                if ((lane & 3) == 0) {
                    vv[16 * i + r] = gac[i][0];
                    vv[16 * i + r + 8] = gac[i][2];
                }
            }
        }
        __syncwarp();
        float A[B];
#pragma unroll
        for (int j = 0; j < B; j += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(As + col * SA + j);
            A[j] = v.x; A[j + 1] = v.y; A[j + 2] = v.z; A[j + 3] = v.w;
        }
        float g = vv[col];
        __syncwarp();
        if (tk.slot >= 0) {  // a chunk of a long row: store the partial statistics (row col)
            if (sub == 0) {
                float *P = a.part + (int64_t)tk.slot * (B * B + B);
#pragma unroll
                for (int j = 0; j < B; j += 4)
                    *reinterpret_cast<float4 *>(P + col * B + j) = make_float4(A[j], A[j + 1], A[j + 2], A[j + 3]);
                P[B * B + col] = g;
            }
            continue;
        }
        const int row = tk.row;
        const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
#pragma unroll
        for (int j = 0; j < B; ++j) A[j] += sGpp[j * B + col] + (j == col ? lam : 0.f);
        g += a.R[(int64_t)row * B + col];
        float delta;
        if (!gj_solve2<B>(A, g, col, sub, w, a.force_fp64 != 0, delta)) {
            queue_retry(a, lane, row);
            continue;
        }
        if (sub == 0) apply_delta(a.X, a.Xh, a.Xl, (int64_t)row * a.d + a.p0 + col, delta);
        __syncwarp();
        if (sub == 0) vv[col] = delta;
        __syncwarp();
        unsigned dh[MT][2], dl[MT][2];
        delta_frags<B>(vv, lane, dh, dl);
        if (nch > 0) {
            // the last chunk is projected from buffer 0 while chunks 0 .. nch - 2
            // are re-gathered into alternating buffers
            const int clast = tk.len - (nch - 1) * CH;
            int64_t qlast = 0;
            if (lane < clast) {
                const int64_t s = tk.begin + (int64_t)(nch - 1) * CH + lane;
                qlast = PERM ? (int64_t)a.pos[s] : s;
                if (HAS_A) cB = a.idx[s];
            }
            if (HAS_A) {  // the staged last chunk was scaled: gather it again, unscaled
                gather_hilo<B>(th_of(0), th_of(0) + C::TILE, a, cB, clast, lane);
                cp_async_commit();
                cp_async_wait_all();
                __syncwarp();
            }
            auto meta2 = [&](int j) {  // chunks before the last are full
                const int64_t s = tk.begin + (int64_t)j * CH + lane;
                cB = a.idx[s];
                qB = PERM ? (int64_t)a.pos[s] : s;
            };
            int64_t qc = 0;
            if (nch > 1) {
                meta2(0);
                qc = qB;
                gather_hilo<B>(th_of(1), th_of(1) + C::TILE, a, cB, CH, lane);
                cp_async_commit();
                if (nch > 2) meta2(1);
            }
            {
                const __nv_bfloat16 *th = th_of(0), *tl = th + C::TILE;
                const float pr = project_mma<B>(th, tl, (clast + 15) >> 4, dh, dl, lane);
                if (lane < clast) a.e[qlast] -= pr;
                __syncwarp();
            }
            for (int ch = 0; ch + 1 < nch; ++ch) {  // chunk ch sits in buffer (ch + 1) & 1
                const int bi = (ch + 1) & 1;
                cp_async_wait_all();
                __syncwarp();
                int64_t qn = 0;
                if (ch + 2 < nch) {
                    gather_hilo<B>(th_of(bi ^ 1), th_of(bi ^ 1) + C::TILE, a, cB, CH, lane);
                    cp_async_commit();
                    qn = qB;
                    if (ch + 3 < nch) meta2(ch + 2);
                }
                const __nv_bfloat16 *th = th_of(bi), *tl = th + C::TILE;
                const float pr = project_mma<B>(th, tl, 2, dh, dl, lane);  // a full chunk
                a.e[qc] -= pr;
                __syncwarp();
                qc = qn;
            }
        }
    }
}

template <int B, bool PERM, bool HAS_A>
cudaError_t launch_sparse_bf16_all(const StepArgs &a, cudaStream_t s) {
    using C = BfCfg<B>;
    using T = TileCfg<B>;
    static bool attr_done = false;
    static int per_sm = 0;
    if (!attr_done) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_sparse_bf16<B, PERM, HAS_A>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      C::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_split_solve<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      split_solve_smem<B>())) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse_bf16<B, PERM, HAS_A>,
                                                               C::WARPS * 32, C::SMEM_BYTES)) != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    if (a.n_tasks > 0) {
        int grid = 152 * per_sm;
        const int need = (a.n_tasks + C::WARPS - 1) / C::WARPS;
        if (grid > need) grid = need;
        prof_mark(a.prof, K_SPARSE, s);
        k_sparse_bf16<B, PERM, HAS_A><<<grid, C::WARPS * 32, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 8 ? a.n_split : 152 * 8;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve<B><<<g2, 256, split_solve_smem<B>(), s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    {  // always called: the first call sizes the grid, outside any stream capture
        const cudaError_t e = launch_split_resid_reg_bf16<B, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry<B, PERM, HAS_A><<<38, 128, 0, s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

}  // namespace ials
