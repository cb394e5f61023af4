// iALS (Algorithm 1; Eq. 3) for b = d above 256: every row solved directly,
// w_r = (alpha0 G + lambda_r I + sum_{s in S_r} alpha_s f_s f_s^T)^{-1} sum alpha_s y_s f_s,
// with G the full Gramian of the fixed side.
//
// At these d the row system (d^2 floats, 1 MB at d = 512) does not fit on chip,
// so each CTA (256 threads) keeps it in its own slice of a global workspace,
// which its tiles stream through L2.  One CTA per row (whole rows: the chunks
// of a long row are skipped but the first, which takes the row), in 64 x 64
// tiles of the lower triangle:
//  * statistics: for every lower tile, the row's interactions are staged in
//    chunks of 32 (the tile's row and column slices of f_s, the weights), each
//    thread accumulating a 4 x 4 block over them from alpha0 G + lambda_r I; the
//    diagonal tiles also accumulate the right-hand side sum alpha y f;
//  * right-looking blocked Cholesky: the diagonal tile factorised in shared
//    memory (pivots below 1e-5 of the original diagonal, 1e-13 in FP64, or not
//    finite, fail the row), the tiles below it multiplied by the inverse of its
//    factor, the trailing tiles updated with both panel tiles staged
//    (transposed) in shared memory, 16 products per thread per column;
//  * forward and backward substitution block by block (off-diagonal products
//    split over four thread groups and summed in a fixed order, the diagonal
//    blocks by one warp).
// The same kernel in FP64 is the re-solve of rows whose FP32 pivot failed.
#include "ials_internal.cuh"

namespace ials {
namespace {

constexpr int BT = 64;    // tile size
constexpr int BTH = 256;  // threads per CTA
constexpr int BCH = 32;   // interactions per staged chunk

template <typename T>
struct BigCfg {
    static constexpr int SP = BT + 4;                  // shared row stride
    static constexpr int STATS = 2 * BCH * SP + 2 * BCH;
    static constexpr int CHOL = 3 * BT * SP + BT;      // diagonal tile, its inverse pivots, two panel tiles
    static constexpr int MAIN = STATS > CHOL ? STATS : CHOL;
    static constexpr int ELEMS = MAIN + 4 * BT + BT;   // + partial sums, solved block
    static constexpr int SMEM = ELEMS * (int)sizeof(T) + 16;
};

template <typename T>
__device__ __forceinline__ T big_sqrt(T x);
template <>
__device__ __forceinline__ float big_sqrt<float>(float x) { return sqrtf(x); }
template <>
__device__ __forceinline__ double big_sqrt<double>(double x) { return sqrt(x); }

template <typename T>
__device__ __forceinline__ bool big_finite(T x) { return x == x && x <= (T)3.0e38 && x >= (T)-3.0e38; }

template <typename T>
__device__ __forceinline__ void big_set(const StepArgs &a, int row, const T *xv) {
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) set_value(a.X, a.Xh, a.Xl, (int64_t)row * a.d + j, (float)xv[j]);
}

// One row: statistics, factorisation, substitutions.  Returns false (uniformly)
// if a pivot failed or the solution is not finite.
template <typename T, bool PERM>
__device__ bool big_row(const StepArgs &a, T *A, T *gv, T *xv, T *dg, T *sm, int *bad, int64_t beg, int32_t len,
                        bool force_fail, T rel) {
    using C = BigCfg<T>;
    constexpr int SP = C::SP;
    const int d = a.d, nt = d / BT, tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int warp = tid >> 5, lane = tid & 31;
    const T lam = (T)a.lambda * ((T)1 + (T)a.nu * (T)len);
    T *xa = sm, *xb = sm + BCH * SP, *wa = sm + 2 * BCH * SP, *wy = wa + BCH;
    T *red = sm + C::MAIN, *blk = red + 4 * BT;
    // ---- statistics (Eqs. 3, 11-12 at b = d), tile by tile of the lower triangle
    for (int ti = 0; ti < nt; ++ti) {
        for (int tj = 0; tj <= ti; ++tj) {
            T acc[4][4], gacc = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int r = ti * BT + 4 * tr + i, c = tj * BT + 4 * tc + j;
                    acc[i][j] = (T)a.alpha0 * (T)a.G[(int64_t)r * d + c] + (r == c ? lam : (T)0);
                }
            for (int c0 = 0; c0 < len; c0 += BCH) {
                const int cnt = min(BCH, len - c0);
                __syncthreads();  // the previous chunk is consumed
                for (int f = tid; f < cnt * BT; f += BTH) {
                    const int k = f / BT, v = f % BT;
                    const float *fr = a.F + (int64_t)a.idx[beg + c0 + k] * d;
                    xa[k * SP + v] = (T)fr[ti * BT + v];
                    xb[k * SP + v] = (T)fr[tj * BT + v];
                }
                if (tid < cnt) {
                    const int64_t s = beg + c0 + tid;
                    const int64_t q = PERM ? (int64_t)a.pos[s] : s;
                    const T al = a.alpha ? (T)a.alpha[q] : (T)1;
                    wa[tid] = al;
                    wy[tid] = al * (a.y ? (T)a.y[q] : (T)1);
                }
                __syncthreads();
                for (int k = 0; k < cnt; ++k) {
                    const T al = wa[k];
                    T xr[4], xc[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        xr[i] = al * xa[k * SP + 4 * tr + i];
                        xc[i] = xb[k * SP + 4 * tc + i];
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] += xr[i] * xc[j];
                    if (ti == tj && tid < BT) gacc += wy[k] * xa[k * SP + tid];
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) A[(int64_t)(ti * BT + 4 * tr + i) * d + tj * BT + 4 * tc + j] = acc[i][j];
            if (ti == tj && tid < BT) gv[ti * BT + tid] = gacc;
        }
    }
    __syncthreads();
    for (int r = tid; r < d; r += BTH) dg[r] = A[(int64_t)r * d + r];
    if (tid == 0) *bad = force_fail ? 1 : 0;
    __syncthreads();
    // ---- blocked Cholesky A = L L^T (lower tiles, in place)
    T *D = sm, *inv = D + BT * SP, *La = inv + BT, *Lb = La + BT * SP;
    for (int p = 0; p < nt; ++p) {
        for (int f = tid; f < BT * BT; f += BTH) {
            const int r = f / BT, c = f % BT;
            D[r * SP + c] = A[(int64_t)(p * BT + r) * d + p * BT + c];
        }
        __syncthreads();
        for (int c = 0; c < BT; ++c) {
            // every thread takes the pivot (written by the previous column's update);
            // thread 0 checks it and stores the factor's diagonal after the barrier
            const T dc = D[c * SP + c];
            const T l = big_sqrt(dc > (T)0 ? dc : (T)1), il = (T)1 / l;
            if (tid == 0 && (!(dc > rel * dg[p * BT + c]) || !big_finite(dc))) *bad = 1;
            for (int r = c + 1 + tid; r < BT; r += BTH) D[r * SP + c] *= il;
            __syncthreads();
            if (tid == 0) {
                D[c * SP + c] = l;
                inv[c] = il;
            }
            const int m = BT - 1 - c;
            for (int f = tid; f < m * m; f += BTH) {
                const int r = c + 1 + f / m, s = c + 1 + f % m;
                if (s <= r) D[r * SP + s] -= D[r * SP + c] * D[s * SP + c];
            }
            __syncthreads();
        }
        for (int f = tid; f < BT * BT; f += BTH) {
            const int r = f / BT, c = f % BT;
            if (c <= r) A[(int64_t)(p * BT + r) * d + p * BT + c] = D[r * SP + c];
        }
        // tiles below the diagonal one: L_ip = A_ip L_pp^{-T} = A_ip (L_pp^{-1})^T.  The
        // inverse of L_pp first (thread c: column c, by forward substitution), kept
        // as Lb[c][r] = (L_pp^{-1})[r][c]; then each tile is the product of the staged
        // (transposed) A_ip with it, as in the trailing update
        __syncthreads();
        if (tid < BT) {
            const int c = tid;
            for (int r = 0; r < c; ++r) Lb[c * SP + r] = 0;
            Lb[c * SP + c] = inv[c];
            for (int r = c + 1; r < BT; ++r) {
                T t = 0;
                for (int mm = c; mm < r; ++mm) t += D[r * SP + mm] * Lb[c * SP + mm];
                Lb[c * SP + r] = -t * inv[r];
            }
        }
        __syncthreads();
        for (int i = p + 1; i < nt; ++i) {
            for (int f = tid; f < BT * BT; f += BTH) {  // La[k][r] = A_ip[r][k]
                const int r = f / BT, k = f % BT;
                La[k * SP + r] = A[(int64_t)(i * BT + r) * d + p * BT + k];
            }
            __syncthreads();
            T acc[4][4];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = 0;
            for (int k = 0; k < BT; ++k) {  // (A_ip Linv^T)[r][c] = sum_k A_ip[r][k] Linv[c][k]
                T u[4], v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    u[q] = La[k * SP + 4 * tr + q];
                    v[q] = Lb[k * SP + 4 * tc + q];
                }
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += u[ii] * v[jj];
            }
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) A[(int64_t)(i * BT + 4 * tr + ii) * d + p * BT + 4 * tc + jj] = acc[ii][jj];
            __syncthreads();
        }
        // trailing update A_ij -= L_ip L_jp^T, p < j <= i
        for (int i = p + 1; i < nt; ++i) {
            for (int j = p + 1; j <= i; ++j) {
                for (int f = tid; f < BT * BT; f += BTH) {  // both panel tiles, transposed: La[k][r] = L_ip[r][k]
                    const int r = f / BT, k = f % BT;
                    La[k * SP + r] = A[(int64_t)(i * BT + r) * d + p * BT + k];
                    Lb[k * SP + r] = A[(int64_t)(j * BT + r) * d + p * BT + k];
                }
                __syncthreads();
                T acc[4][4];
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) acc[ii][jj] = 0;
                for (int k = 0; k < BT; ++k) {
                    T u[4], v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        u[q] = La[k * SP + 4 * tr + q];
                        v[q] = Lb[k * SP + 4 * tc + q];
                    }
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) acc[ii][jj] += u[ii] * v[jj];
                }
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj)
                        A[(int64_t)(i * BT + 4 * tr + ii) * d + j * BT + 4 * tc + jj] -= acc[ii][jj];
                __syncthreads();
            }
        }
    }
    if (*bad) return false;  // uniform: set before the last barrier
    // ---- forward substitution L y = g (y overwrites g); the diagonal block staged in D
    const int r64 = tid & (BT - 1), part = tid >> 6;
    for (int p = 0; p < nt; ++p) {
        for (int r = warp; r < BT; r += BTH / 32) {  // rows of block p against y of the blocks before
            const T *lrow = A + (int64_t)(p * BT + r) * d;
            T t = 0;
            for (int c = lane; c < p * BT; c += 32) t += lrow[c] * gv[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
            if (lane == 0) red[r] = t;
        }
        for (int f = tid; f < BT * BT; f += BTH) {
            const int r = f / BT, c = f % BT;
            D[r * SP + c] = A[(int64_t)(p * BT + r) * d + p * BT + c];
        }
        __syncthreads();
        if (warp == 0) {  // L_pp y_p = g_p - (L y)_p, row by row
            for (int r = 0; r < BT; ++r) {
                T t = 0;
                for (int mm = lane; mm < r; mm += 32) t += D[r * SP + mm] * gv[p * BT + mm];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
                if (lane == 0) gv[p * BT + r] = (gv[p * BT + r] - red[r] - t) / D[r * SP + r];
                __syncwarp();
            }
        }
        __syncthreads();
    }
    // ---- backward substitution L^T x = y
    for (int p = nt - 1; p >= 0; --p) {
        T t = 0;
        for (int c = (p + 1) * BT + part; c < d; c += 4) t += A[(int64_t)c * d + p * BT + r64] * xv[c];
        red[part * BT + r64] = t;
        for (int f = tid; f < BT * BT; f += BTH) {
            const int r = f / BT, c = f % BT;
            D[r * SP + c] = A[(int64_t)(p * BT + r) * d + p * BT + c];
        }
        __syncthreads();
        if (tid < BT) blk[tid] = gv[p * BT + tid] - (((red[tid] + red[BT + tid]) + red[2 * BT + tid]) + red[3 * BT + tid]);
        __syncthreads();
        if (warp == 0) {  // L_pp^T x_p = blk, from the last row
            for (int r = BT - 1; r >= 0; --r) {
                T t2 = 0;
                for (int mm = r + 1 + lane; mm < BT; mm += 32) t2 += D[mm * SP + r] * blk[mm];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t2 += __shfl_xor_sync(kFull, t2, o);
                if (lane == 0) blk[r] = (blk[r] - t2) / D[r * SP + r];
                __syncwarp();
            }
        }
        __syncthreads();
        if (tid < BT) xv[p * BT + tid] = blk[tid];
        __syncthreads();
    }
    bool fin = true;
    for (int j = tid; j < d; j += BTH) fin = fin && big_finite(xv[j]);
    return __syncthreads_and(fin);
}

template <typename T, bool PERM, bool RETRY>
__global__ void __launch_bounds__(BTH) k_ials_big(const StepArgs a, T *ws) {
    using C = BigCfg<T>;
    extern __shared__ float4 smem4[];
    T *sm = reinterpret_cast<T *>(smem4);
    int *flag = reinterpret_cast<int *>(sm + C::ELEMS);  // [0] next task, [1] bad pivot
    const int d = a.d, tid = threadIdx.x;
    T *A = ws + (int64_t)blockIdx.x * ((int64_t)d * d + 3 * d);
    T *gv = A + (int64_t)d * d, *xv = gv + d, *dg = xv + d;
    const T rel = RETRY ? (T)1e-13 : (T)1e-5;
    if (RETRY) {
        const int count = *(volatile int *)a.retry;
        for (int q = blockIdx.x; q < count; q += gridDim.x) {
            const int row = a.retry[1 + q];
            const int64_t beg = a.ptr[row];
            const int32_t len = (int32_t)(a.ptr[row + 1] - beg);
            const bool ok = big_row<T, PERM>(a, A, gv, xv, dg, sm, &flag[1], beg, len, false, rel);
            if (ok) big_set(a, row, xv);
            if (tid == 0) atomicAdd((unsigned long long *)&a.stats[ok ? 0 : 1], 1ull);
            __syncthreads();
        }
        return;
    }
    if (tid == 0) flag[0] = atomicAdd(a.counter, 1);
    for (;;) {
        __syncthreads();
        const int tsk = flag[0];
        if (tsk >= a.n_tasks) break;
        __syncthreads();
        if (tid == 0) flag[0] = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        int64_t beg = tk.begin;
        int32_t len = tk.len, row = tk.row;
        if (tk.slot >= 0) {  // a chunk of a long row: its first chunk takes the whole row
            const SplitRow sr = a.split[tk.srow];
            if (tk.slot != sr.slot0) continue;
            beg = sr.begin;
            len = sr.len;
            row = sr.row;
        }
        const bool ok = big_row<T, PERM>(a, A, gv, xv, dg, sm, &flag[1], beg, len, a.force_fp64 != 0, rel);
        if (ok) {
            big_set(a, row, xv);
        } else if (tid == 0) {
            const int i = atomicAdd(a.retry, 1);
            a.retry[1 + i] = row;
        }
    }
}

constexpr int kBigGrid = 2 * 152;    // FP32 blocks (two per SM)
constexpr int kBigRetryGrid = 76;    // FP64 re-solve blocks

template <bool PERM>
cudaError_t launch_big(const StepArgs &a, float *ws, double *ws64, cudaStream_t s) {
    if (a.n_tasks > 0) {
        prof_mark(a.prof, K_SPARSE, s);
        k_ials_big<float, PERM, false><<<kBigGrid, BTH, BigCfg<float>::SMEM, s>>>(a, ws);
        prof_mark(a.prof, -1, s);
    }
    prof_mark(a.prof, K_RETRY, s);
    k_ials_big<double, PERM, true><<<kBigRetryGrid, BTH, BigCfg<double>::SMEM, s>>>(a, ws64);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

}  // namespace

bool ials_big_supported(int32_t d) { return d > 256 && d <= 1024 && d % BT == 0; }

int64_t ials_big_ws_floats(int32_t d) { return (int64_t)kBigGrid * ((int64_t)d * d + 3 * d); }
int64_t ials_big_ws_doubles(int32_t d) { return (int64_t)kBigRetryGrid * ((int64_t)d * d + 3 * d); }

cudaError_t ials_big_prepare() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_ials_big<float, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  BigCfg<float>::SMEM)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ials_big<float, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  BigCfg<float>::SMEM)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_ials_big<double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  BigCfg<double>::SMEM)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_ials_big<double, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                BigCfg<double>::SMEM);
}

cudaError_t launch_ials_big(const StepArgs &a, cudaStream_t s) {
    if (!ials_big_supported(a.d) || a.b != a.d || !a.direct || !a.big_ws || !a.big_ws64) return cudaErrorInvalidValue;
    return a.pos ? launch_big<true>(a, a.big_ws, a.big_ws64, s) : launch_big<false>(a, a.big_ws, a.big_ws64, s);
}

}  // namespace ials
