// Block step of Algorithm 3 for block sizes B = 64, 128 and 256 with the b x b
// system of a row held in registers, spread over the CTA (one CTA per task).
//
// A_r is cut into 8 x 8 tiles; the NTL = NB (NB + 1) / 2 tiles on or below
// the diagonal (NB = B / 8) are owned by threads 0 .. NTL - 1, thread t owning
// tile (ti, tj), ti >= tj, in 64 registers.  The same tile stays with its
// owner through the whole step:
//  * statistics (Eqs. 11-12): NG interaction groups of NTL threads each
//    accumulate their tile over the staged slices (group g takes staged
//    interactions g, g + NG, ...); the owners of column 0 also accumulate the
//    gradient.  Groups 1 .. NG-1 hand their partials to group 0 through
//    shared memory, summed in group order.  For a whole row the owners start
//    from alpha0 G_pipi + lambda_r I and R_r.
//  * Newton solve (Eq. 9): right-looking blocked Cholesky in 8-column panels,
//    every tile updated by its owner in registers.  Panel p: the owner of the
//    diagonal tile factorises it and forward-substitutes its block of the
//    right-hand side; the owners of the tiles below it solve them against it
//    and remove their block's contribution from the right-hand side; the
//    owners of the trailing tiles subtract the rank-8 product.  Only the
//    panel's factor tiles travel, through a double-buffered shared panel.
//    Backward substitution runs panel by panel from the bottom, each block
//    of the solution broadcast through shared memory and removed from the
//    blocks above it by the owners of the factor's row.
// Two CTA barriers per panel in each direction; no thread waits on a single
// serial thread for more than one 8 x 8 factorisation.
#pragma once

#include "k_sparse_cta.cuh"

namespace ials {

template <int B>
struct RegChol {
    static constexpr int NB = B / 8;                 // 8-wide blocks
    static constexpr int NTL = NB * (NB + 1) / 2;    // tiles on or below the diagonal
    static constexpr int PB = 68;                    // floats per panel block: 8 x 8, column-major, padded
    static constexpr int PANEL = NB * PB;            // floats of one panel buffer
};

// Tiles of the (statistics + dense terms) system, one per owning thread.
// Shared: Lp (two panel buffers), zv (B floats: right-hand side, then z, then
// the solution), bad (set on a failed FP32 pivot).
//
// Factorisation A = L L^T and forward substitution z = L^{-1} g.  On entry an
// owner's a[][] holds the lower part of its tile of A (upper part of diagonal
// tiles: anything) and zv holds g.  On return owners hold their tile of L
// (diagonal owners also inv[k] = 1 / L_kk) and zv holds z.  A pivot that is
// not above rel * (its original diagonal) or is not finite sets *bad.  All
// threads of the CTA call it.
template <int B>
__device__ __forceinline__ void rc_factor(float (&a)[8][8], float (&inv)[8], int ti, int tj, bool own,
                                          float *Lp, float *zv, int *bad, float rel) {
    using C = RegChol<B>;
    float d0[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) d0[k] = a[k][k];
#pragma unroll 1
    for (int p = 0; p < C::NB; ++p) {
        float *P = Lp + (p & 1) * C::PANEL;
        if (own && ti == p && tj == p) {
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float dm = a[m][m];
                if (!(dm > rel * d0[m]) || !(dm <= 3.0e38f)) *bad = 1;
                const float im = rsqrtf(fmaxf(dm, 1e-30f));
                inv[m] = im;
                a[m][m] = dm * im;
#pragma unroll
                for (int k = m + 1; k < 8; ++k) a[k][m] *= im;
#pragma unroll
                for (int k = m + 1; k < 8; ++k)
#pragma unroll
                    for (int j = m + 1; j <= k; ++j) a[k][j] = fmaf(-a[k][m], a[j][m], a[k][j]);
            }
            float z[8];
            load_seg<8>(zv + 8 * p, z);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                z[m] *= inv[m];
#pragma unroll
                for (int k = m + 1; k < 8; ++k) z[k] = fmaf(-a[k][m], z[m], z[k]);
            }
            store_tile<8>(zv + 8 * p, z, false);
            float *blk = P + p * C::PB;
#pragma unroll
            for (int m = 0; m < 8; ++m) {  // column m: 1 / L_mm on the diagonal, L_km below
                float col[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) col[k] = k < m ? 0.f : (k == m ? inv[m] : a[k][m]);
                store_tile<8>(blk + 8 * m, col, false);
            }
        }
        __syncthreads();
        if (own && tj == p && ti > p) {
            const float *Lpp = P + p * C::PB;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                float col[8];
                load_seg<8>(Lpp + 8 * m, col);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float l = a[r][m] * col[m];
                    a[r][m] = l;
#pragma unroll
                    for (int k = m + 1; k < 8; ++k) a[r][k] = fmaf(-l, col[k], a[r][k]);
                }
            }
            float *blk = P + ti * C::PB;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                float col[8];
#pragma unroll
                for (int r = 0; r < 8; ++r) col[r] = a[r][m];
                store_tile<8>(blk + 8 * m, col, false);
            }
            float z[8], g[8];
            load_seg<8>(zv + 8 * p, z);
            load_seg<8>(zv + 8 * ti, g);
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int m = 0; m < 8; ++m) g[r] = fmaf(-a[r][m], z[m], g[r]);
            store_tile<8>(zv + 8 * ti, g, false);
        }
        __syncthreads();
        if (own && tj > p) {
            const float *Li = P + ti * C::PB, *Lj = P + tj * C::PB;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                float li[8], lj[8];
                load_seg<8>(Li + 8 * m, li);
                load_seg<8>(Lj + 8 * m, lj);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    const float nl = -li[r];
#pragma unroll
                    for (int c = 0; c < 8; c += 2) fma2(a[r][c], a[r][c + 1], nl, nl, lj[c], lj[c + 1]);
                }
            }
        }
    }
}

// Backward substitution L^T x = z (z in zv on entry, x on return), panel by
// panel from the bottom.  All threads of the CTA call it.
template <int B>
__device__ __forceinline__ void rc_backsolve(const float (&a)[8][8], const float (&inv)[8], int ti, int tj,
                                             bool own, float *zv) {
    using C = RegChol<B>;
#pragma unroll 1
    for (int p = C::NB - 1; p >= 0; --p) {
        if (own && ti == p && tj == p) {
            float x[8];
            load_seg<8>(zv + 8 * p, x);
#pragma unroll
            for (int m = 7; m >= 0; --m) {
#pragma unroll
                for (int k = m + 1; k < 8; ++k) x[m] = fmaf(-a[k][m], x[k], x[m]);
                x[m] *= inv[m];
            }
            store_tile<8>(zv + 8 * p, x, false);
        }
        __syncthreads();
        if (own && ti == p && tj < p) {
            float x[8], z[8];
            load_seg<8>(zv + 8 * p, x);
            load_seg<8>(zv + 8 * tj, z);
#pragma unroll
            for (int c = 0; c < 8; ++c)
#pragma unroll
                for (int r = 0; r < 8; ++r) z[c] = fmaf(-a[r][c], x[r], z[c]);
            store_tile<8>(zv + 8 * tj, z, false);
        }
        __syncthreads();
    }
}

// Configuration of the FP32 kernel: NG interaction groups during the statistics.
template <int B>
struct RcCfg {
    using R = RegChol<B>;
    static constexpr int NG = B == 64 ? 2 : 1;
    static constexpr int ACTIVE = R::NTL * NG;
    static constexpr int THREADS = (ACTIVE + 31) / 32 * 32;
    // resident CTAs per SM (caps registers at ~136; b = 256: 544 threads, one CTA)
    static constexpr int MINB = B == 64 ? 5 : (B == 128 ? 3 : 1);
    static constexpr int SB = CtaCfg<B>::SB, CH = CtaCfg<B>::CH, BUF = CtaCfg<B>::BUF;
    static constexpr int RED = (NG - 1) * R::NTL * 72;  // group partials (tile + gradient block)
    // floats: staging, e[2][CH], alpha[2][CH], group partials, two panels, zv, flags
    static constexpr int SMEM_FLOATS = 2 * BUF + 4 * CH + RED + 2 * R::PANEL + B + 4;
    static constexpr int SMEM_BYTES = SMEM_FLOATS * 4;
};

// a = alpha0 G_pipi + lambda I on tile (ti, tj); gradient block = R_r (owners of column 0).
template <int B, bool DIRECT>
__device__ __forceinline__ void rc_dense_init(const StepArgs &a, int ti, int tj, int row, float lam,
                                              float (&t)[8][8], float (&g)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float *gr = a.G + (int64_t)(a.p0 + 8 * ti + i) * B + 8 * tj;
        float v[8];
        load_seg<8>(gr, v);
#pragma unroll
        for (int j = 0; j < 8; ++j) t[i][j] = a.alpha0 * v[j];
        if (ti == tj) t[i][i] += lam;
        g[i] = (!DIRECT && tj == 0) ? a.R[(int64_t)row * B + 8 * ti + i] : 0.f;
    }
}

template <int B, bool PERM, bool HAS_A, bool DIRECT>
__global__ void __launch_bounds__(RcCfg<B>::THREADS, RcCfg<B>::MINB) k_sparse_rc(const StepArgs a) {
    using C = RcCfg<B>;
    using R = RegChol<B>;
    constexpr int SB = C::SB, CH = C::CH, NTL = R::NTL, NG = C::NG;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *buf0 = smem;                      // staging buffer bi at buf0 + bi * BUF
    float *she = smem + 2 * C::BUF;          // residuals (weighted) [2][CH]
    float *sha = she + 2 * CH;               // weights [2][CH]
    float *red = sha + 2 * CH;               // group partials
    float *Lp = red + C::RED;
    float *zv = Lp + 2 * R::PANEL;
    int *flag = reinterpret_cast<int *>(zv + B);  // [0] next task, [1] bad pivot
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool active = tid < C::ACTIVE;
    const int grp = active ? tid / NTL : NG;
    const bool own = tid < NTL;              // group 0 keeps the tiles through the solve
    const int kstart = active ? grp : CH;    // idle threads skip the accumulation
    int ti = 0, tj = 0;
    tri_index(tid % NTL, ti, tj);
    if (tid == 0) flag[0] = atomicAdd(a.counter, 1);  // the next task is fetched while one runs
    for (;;) {
        __syncthreads();
        const int tsk = flag[0];
        if (tsk >= a.n_tasks) break;
        __syncthreads();  // every thread has read flag[0]
        if (tid == 0) flag[0] = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float t[8][8], g[8];
        const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
        if (tk.slot < 0 && grp == 0) {
            rc_dense_init<B, DIRECT>(a, ti, tj, tk.row, lam, t, g);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                g[i] = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) t[i][j] = 0.f;
            }
        }
        // residual (label, for DIRECT) and weight of chunk j into buffer bi
        auto meta = [&](int j, int bi) {
            const int cnt = min(CH, tk.len - j * CH);
            if (tid < cnt) {
                const int64_t s = tk.begin + (int64_t)j * CH + tid;
                const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                const float r = DIRECT ? (a.y ? a.y[q] : 1.f) : a.e[q];
                const float al = HAS_A ? a.alpha[q] : 1.f;
                she[bi * CH + tid] = HAS_A ? al * r : r;
                if (HAS_A) sha[bi * CH + tid] = al;
            }
        };
        if (nch > 0) {
            meta(0, 0);
            cta_gather<B>(a, tk.begin, min(CH, tk.len), buf0);
            cp_async_commit();
        }
        for (int ch = 0; ch < nch; ++ch) {
            const int bi = ch & 1;
            cp_async_wait_all();
            __syncthreads();
            if (ch + 1 < nch) {
                meta(ch + 1, bi ^ 1);
                cta_gather<B>(a, tk.begin + (int64_t)(ch + 1) * CH, min(CH, tk.len - (ch + 1) * CH),
                              buf0 + (bi ^ 1) * C::BUF);
                cp_async_commit();
            }
            const int cnt = min(CH, tk.len - ch * CH);
            const float *bp = buf0 + bi * C::BUF;
            for (int k = kstart; k < cnt; k += NG) {
                const float *xk = bp + k * SB;
                float xa[8], xb[8];
                load_seg<8>(xk + 8 * ti, xa);
                load_seg<8>(xk + 8 * tj, xb);
                const float ek = she[bi * CH + k];
#pragma unroll
                for (int i = 0; i < 8; ++i) g[i] = fmaf(ek, xa[i], g[i]);
                if (HAS_A) {
                    const float ak = sha[bi * CH + k];
#pragma unroll
                    for (int i = 0; i < 8; ++i) xa[i] *= ak;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; j += 2) fma2(t[i][j], t[i][j + 1], xa[i], xa[i], xb[j], xb[j + 1]);
            }
        }
        if constexpr (NG > 1) {  // fixed-order sum of the group partials into group 0's registers
            if (active && grp > 0) {
                float *o = red + ((grp - 1) * NTL + tid % NTL) * 72;
#pragma unroll
                for (int i = 0; i < 8; ++i) store_tile<8>(o + 8 * i, t[i], false);
                store_tile<8>(o + 64, g, false);
            }
            __syncthreads();
            if (own) {
#pragma unroll 1
                for (int q = 1; q < NG; ++q) {
                    const float *o = red + ((q - 1) * NTL + tid) * 72;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        float v[8];
                        load_seg<8>(o + 8 * i, v);
#pragma unroll
                        for (int j = 0; j < 8; ++j) t[i][j] += v[j];
                    }
                    float v[8];
                    load_seg<8>(o + 64, v);
#pragma unroll
                    for (int i = 0; i < 8; ++i) g[i] += v[i];
                }
            }
        }
        if (tk.slot >= 0) {  // a chunk of a long row: store the partial statistics
            float *P = a.part + (int64_t)tk.slot * (B * B + B);
            if (own) {
#pragma unroll
                for (int i = 0; i < 8; ++i)  // tiles on or below the diagonal (the only ones read back)
                    store_tile<8>(P + (int64_t)(8 * ti + i) * B + 8 * tj, t[i], false);
                if (tj == 0) store_tile<8>(P + (int64_t)B * B + 8 * ti, g, false);
            }
            continue;
        }
        if (own && tj == 0) store_tile<8>(zv + 8 * ti, g, false);
        if (tid == 0) flag[1] = a.force_fp64 ? 1 : 0;
        __syncthreads();
        float inv[8];
        rc_factor<B>(t, inv, ti, tj, own, Lp, zv, &flag[1], 1e-5f);
        if (flag[1]) {  // CTA-uniform (read after the factorisation's last barrier)
            if (tid == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        rc_backsolve<B>(t, inv, ti, tj, own, zv);
        bool fin = true;
        for (int j = tid; j < B; j += nt) fin = fin && isfinite(zv[j]);
        if (!__syncthreads_and(fin)) {
            if (tid == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        if (DIRECT) {  // Eq. 3: the solution is the row itself
            for (int j = tid; j < B; j += nt) set_value(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + j, zv[j]);
        } else {
            for (int j = tid; j < B; j += nt) apply_delta(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + j, zv[j]);
            cta_residual_update2<B, PERM>(a, tk.begin, tk.len, nch, zv, buf0);
        }
    }
}

// One CTA per split row: its partial slots summed tile by tile in slot order,
// the dense terms added, then the register-tile solve.
template <int B, bool DIRECT>
__global__ void __launch_bounds__(RcCfg<B>::THREADS) k_split_solve_rc(const StepArgs a) {
    using C = RcCfg<B>;
    using R = RegChol<B>;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *Lp = smem + 2 * C::BUF + 4 * C::CH + C::RED;
    float *zv = Lp + 2 * R::PANEL;
    int *flag = reinterpret_cast<int *>(zv + B);
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool own = tid < R::NTL;
    int ti = 0, tj = 0;
    tri_index(tid % R::NTL, ti, tj);
    for (int i = blockIdx.x; i < a.n_split; i += gridDim.x) {
        const SplitRow sr = a.split[i];
        const float lam = a.lambda * (1.0f + a.nu * (float)sr.len);
        float t[8][8], g[8];
        rc_dense_init<B, DIRECT>(a, ti, tj, sr.row, lam, t, g);
        if (own) {
            const float *P0 = a.part + (int64_t)sr.slot0 * (B * B + B);
            for (int sl = 0; sl < sr.nslots; ++sl) {
                const float *P = P0 + (int64_t)sl * (B * B + B);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float v[8];
                    load_seg<8>(P + (int64_t)(8 * ti + r) * B + 8 * tj, v);
#pragma unroll
                    for (int j = 0; j < 8; ++j) t[r][j] += v[j];
                }
                if (tj == 0) {
                    float v[8];
                    load_seg<8>(P + (int64_t)B * B + 8 * ti, v);
#pragma unroll
                    for (int r = 0; r < 8; ++r) g[r] += v[r];
                }
            }
            if (tj == 0) store_tile<8>(zv + 8 * ti, g, false);
        }
        if (tid == 0) flag[1] = a.force_fp64 ? 1 : 0;
        __syncthreads();
        float inv[8];
        rc_factor<B>(t, inv, ti, tj, own, Lp, zv, &flag[1], 1e-5f);
        bool ok = !flag[1];
        if (ok) {
            rc_backsolve<B>(t, inv, ti, tj, own, zv);
            bool fin = true;
            for (int j = tid; j < B; j += nt) fin = fin && isfinite(zv[j]);
            ok = __syncthreads_and(fin);
        }
        if (!ok) {
            if (tid == 0) {
                const int q = atomicAdd(a.retry, 1);
                a.retry[1 + q] = sr.row;
            }
            if (!DIRECT)
                for (int j = tid; j < B; j += nt) a.delta[(int64_t)i * B + j] = 0.f;
        } else {
            for (int j = tid; j < B; j += nt) {
                if (DIRECT) {
                    set_value(a.X, a.Xh, a.Xl, (int64_t)sr.row * a.d + a.p0 + j, zv[j]);
                } else {
                    apply_delta(a.X, a.Xh, a.Xl, (int64_t)sr.row * a.d + a.p0 + j, zv[j]);
                    a.delta[(int64_t)i * B + j] = zv[j];
                }
            }
        }
        __syncthreads();
    }
}

template <int B, bool PERM, bool HAS_A, bool DIRECT>
cudaError_t launch_sparse_rc_all(const StepArgs &a, cudaStream_t s) {
    using C = RcCfg<B>;
    using CF = CtaCfg<B>;
    static bool attr_done = false;
    static int per_sm = 0;
    if (!attr_done) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_sparse_rc<B, PERM, HAS_A, DIRECT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_split_solve_rc<B, DIRECT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      C::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_retry_cta<B, PERM, HAS_A, DIRECT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, retry_cta_smem<B>())) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sparse_rc<B, PERM, HAS_A, DIRECT>,
                                                               C::THREADS, C::SMEM_BYTES)) != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    if (a.n_tasks > 0) {
        int grid = 152 * per_sm;
        if (grid > a.n_tasks) grid = a.n_tasks;
        prof_mark(a.prof, K_SPARSE, s);
        k_sparse_rc<B, PERM, HAS_A, DIRECT><<<grid, C::THREADS, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 4 ? a.n_split : 152 * 4;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve_rc<B, DIRECT><<<g2, C::THREADS, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (!DIRECT) {  // always called: the first call sizes the grid, outside any stream capture
        const cudaError_t e = launch_split_resid_reg<B, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry_cta<B, PERM, HAS_A, DIRECT><<<kRetryBlocks, CF::THREADS, retry_cta_smem<B>(), s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

template <int B>
cudaError_t launch_sparse_rc_dispatch(const StepArgs &a, cudaStream_t s) {
    const bool perm = a.pos != nullptr, wa = a.alpha != nullptr;
    if (a.direct) {
        if (perm) return wa ? launch_sparse_rc_all<B, true, true, true>(a, s) : launch_sparse_rc_all<B, true, false, true>(a, s);
        return wa ? launch_sparse_rc_all<B, false, true, true>(a, s) : launch_sparse_rc_all<B, false, false, true>(a, s);
    }
    if (perm) return wa ? launch_sparse_rc_all<B, true, true, false>(a, s) : launch_sparse_rc_all<B, true, false, false>(a, s);
    return wa ? launch_sparse_rc_all<B, false, true, false>(a, s) : launch_sparse_rc_all<B, false, false, false>(a, s);
}

}  // namespace ials
