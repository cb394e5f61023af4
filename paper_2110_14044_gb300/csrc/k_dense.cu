// Dense-side kernels of the iALS++ epoch:
//   * residual cache e = yhat - y over S (Algorithm 3, "Compute yhat"; Eq. 1)
//   * FP64 pieces of the objective L(W,H) (Eq. 2)
//   * split-K partial Gramian G^{pi} = X^T X[:, pi] (Eq. 10) and the full
//     FP64-accumulated Gramian used by the objective (Eq. 4)
//   * row terms alpha0 x_r G^{pi} + lambda_r x_{r,pi} (Algorithm 3, gradient
//     initialisation; first and last terms of Eq. 11)
//   * seeded normal initialisation of the factors
#include "ials_internal.cuh"

#include <math.h>

namespace ials {

namespace {

constexpr int kSMs = 152;  // GB300: 2 dies x 76 SMs

__device__ __forceinline__ float dot4(float4 a, float4 b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}

// ------------------------------------------------------------------ residual
// One warp per user row.  The warp loads the column ids of 32 interactions at
// once (one coalesced load), then sub-groups of SG = 2^SGL lanes take
// interactions sub, sub + 32/SG, ...; lane l of a sub-group owns float4 chunks
// l, l + SG, ... (MAXV of them) of the d-vector.  Each sub-group keeps up to
// four gathers in flight before it reduces.  Each block accumulates
// alpha_s (<w_u, h_i> - y_s)^2 in FP64 and writes one partial sum.
template <int SGL, int MAXV>
__global__ void __launch_bounds__(256) k_residual(const int64_t *__restrict__ u_ptr,
                                                  const int32_t *__restrict__ u_idx,
                                                  const float *__restrict__ W,
                                                  const float *__restrict__ H,
                                                  const float *__restrict__ y,
                                                  const float *__restrict__ alpha,
                                                  int32_t n_users, int32_t d,
                                                  double *__restrict__ part) {
    constexpr int SG = 1 << SGL, NSUB = 32 / SG;  // NSUB sub-groups, SG interactions each per chunk
    constexpr int UMAX = MAXV >= 16 ? 1 : (MAXV >= 8 ? 2 : 4);  // keep U * MAXV float4 in registers <= 16
    constexpr int U = SG < UMAX ? SG : UMAX;
    const int lane = threadIdx.x & 31;
    const int sub = lane >> SGL, sl = lane & (SG - 1);
    const int nv4 = d >> 2;
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
    const float4 *H4 = reinterpret_cast<const float4 *>(H);
    const int warps_total = (gridDim.x * blockDim.x) >> 5;
    double loss = 0.0;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n_users; u += warps_total) {
        float4 wv[MAXV];
#pragma unroll
        for (int m = 0; m < MAXV; ++m) {
            const int v = sl + m * SG;
            wv[m] = v < nv4 ? W4[(int64_t)u * nv4 + v] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int64_t beg = u_ptr[u], end = u_ptr[u + 1];
        for (int64_t s0 = beg; s0 < end; s0 += 32) {
            const int cnt = (int)min((int64_t)32, end - s0);
            const int my_c = lane < cnt ? u_idx[s0 + lane] : 0;
#pragma unroll
            for (int m0 = 0; m0 < SG; m0 += U) {
                float acc[U];
                float4 h[U][MAXV];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int k = sub + NSUB * (m0 + q);
                    const int64_t c = __shfl_sync(kFull, my_c, k);
                    acc[q] = 0.f;
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) {
                        const int v = sl + m * SG;
                        h[q][m] = (k < cnt && v < nv4) ? __ldg(H4 + c * nv4 + v)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) acc[q] += dot4(wv[m], h[q][m]);
#pragma unroll
                    for (int o = SG >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], o);
                }
                if (sl == 0) {
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int k = sub + NSUB * (m0 + q);
                        if (k < cnt) {
                            const int64_t s = s0 + k;
                            const float r = acc[q] - (y ? y[s] : 1.0f);
                            loss += (alpha ? (double)alpha[s] : 1.0) * (double)r * (double)r;
                        }
                    }
                }
            }
        }
    }
    __shared__ double red[256];
    red[threadIdx.x] = loss;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Residual cache e = W H^T - y over S (Alg. 3, "Compute yhat"), persistent and
// work-stealing: warps take the user-side tasks (rows, or pieces of long rows;
// the list is sorted by decreasing length) from an atomic counter, so the long
// rows start first and no warp idles while work remains.  Lane layout as in
// k_residual (sub-groups of SG lanes per interaction, U interactions in flight
// per sub-group); the column ids of the next 32 interactions are loaded before
// the current 32 are processed.  Each e_s is written once by one lane, so the
// result does not depend on the schedule.
template <int SGL, int MAXV>
__global__ void __launch_bounds__(256) k_residual_tasks(const Task *__restrict__ tasks, int32_t n_tasks,
                                                        const int32_t *__restrict__ u_idx,
                                                        const float *__restrict__ W,
                                                        const float *__restrict__ H,
                                                        const float *__restrict__ y, int32_t d,
                                                        float *__restrict__ e, int32_t *counter) {
    constexpr int SG = 1 << SGL, NSUB = 32 / SG;
    constexpr int UMAX = MAXV >= 16 ? 1 : (MAXV >= 8 ? 2 : 4);
    constexpr int U = SG < UMAX ? SG : UMAX;
    const int lane = threadIdx.x & 31;
    const int sub = lane >> SGL, sl = lane & (SG - 1);
    const int nv4 = d >> 2;
    const float4 *W4 = reinterpret_cast<const float4 *>(W);
    const float4 *H4 = reinterpret_cast<const float4 *>(H);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tasks) break;
        const Task tk = tasks[t];
        const int64_t beg = tk.begin, end = tk.begin + tk.len;
        float4 wv[MAXV];
#pragma unroll
        for (int m = 0; m < MAXV; ++m) {
            const int v = sl + m * SG;
            wv[m] = v < nv4 ? W4[(int64_t)tk.row * nv4 + v] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        int my_c = beg + lane < end ? u_idx[beg + lane] : 0;
        for (int64_t s0 = beg; s0 < end; s0 += 32) {
            const int cnt = (int)min((int64_t)32, end - s0);
            const int nxt_c = s0 + 32 + lane < end ? u_idx[s0 + 32 + lane] : 0;
#pragma unroll
            for (int m0 = 0; m0 < SG; m0 += U) {
                float acc[U];
                float4 h[U][MAXV];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int k = sub + NSUB * (m0 + q);
                    const int64_t c = __shfl_sync(kFull, my_c, k);
                    acc[q] = 0.f;
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) {
                        const int v = sl + m * SG;
                        h[q][m] = (k < cnt && v < nv4) ? __ldg(H4 + c * nv4 + v)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) acc[q] += dot4(wv[m], h[q][m]);
#pragma unroll
                    for (int o = SG >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], o);
                }
                if (sl == 0) {
#pragma unroll
                    for (int q = 0; q < U; ++q) {
                        const int k = sub + NSUB * (m0 + q);
                        if (k < cnt) {
                            const int64_t s = s0 + k;
                            e[s] = acc[q] - (y ? y[s] : 1.0f);
                        }
                    }
                }
            }
            my_c = nxt_c;
        }
    }
}

// Fixed-order sum of n doubles by one block; *out = (acc ? *out : 0) + scale * sum.
__global__ void k_sum_parts(const double *__restrict__ part, int32_t n, double scale,
                            double *out, int acc) {
    __shared__ double red[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (acc ? *out : 0.0) + scale * red[0];
}

// sum_r lambda (1 + nu n_r) |x_r|^2, one warp per row, FP64 accumulation.
__global__ void __launch_bounds__(256) k_reg_loss(const int64_t *__restrict__ ptr,
                                                  const float *__restrict__ X, int32_t n_rows,
                                                  int32_t d, double lambda, double nu,
                                                  double *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int warps_total = (gridDim.x * blockDim.x) >> 5;
    double acc = 0.0;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n_rows; r += warps_total) {
        double t = 0.0;
        for (int f = lane; f < d; f += 32) {
            const double x = X[(int64_t)r * d + f];
            t += x * x;
        }
        acc += lambda * (1.0 + nu * (double)(ptr[r + 1] - ptr[r])) * t;
    }
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_frobenius(const double *__restrict__ A, const double *__restrict__ B,
                            int64_t count, double scale, double *out) {
    __shared__ double red[256];
    double t = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) t += A[i] * B[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = blockDim.x >> 1; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out += scale * red[0];
}

// ------------------------------------------------------------------ Gramian
// Split-K tile kernel: block (tm, tn, split) accumulates the TM x TN output
// tile [tm*TM, +TM) x [tn*TN, +TN) of X^T X[:, p0:p0+bs] over the rows
// [split*rows_per, +rows_per) of X.  256 threads, 4 x 4 outputs each; the tile
// shape follows bs ((256,16), (128,32) or (64,64)) so no thread idles at small b.
// F64: accumulate each 16-row slab in FP32 and fold it into FP64 accumulators.
constexpr int GK = 16;

template <int TM, int TN, bool F64>
__global__ void __launch_bounds__(256) k_gram_tile(const float *__restrict__ X, int64_t n,
                                                   int32_t d, int32_t p0, int32_t bs,
                                                   int64_t rows_per, void *__restrict__ ws) {
    static_assert((TM / 4) * (TN / 4) == 256, "tile shape");
    __shared__ __align__(16) float As[GK][TM];
    __shared__ __align__(16) float Bs[GK][TN];
    const int tid = threadIdx.x, tx = tid % (TN / 4), ty = tid / (TN / 4);
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int64_t k_beg = (int64_t)blockIdx.z * rows_per;
    const int64_t k_end = min(n, k_beg + rows_per);
    float acc[4][4];
    double acc64[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; acc64[i][j] = 0.0; }
    for (int64_t k0 = k_beg; k0 < k_end; k0 += GK) {
        for (int i = tid; i < GK * TM; i += 256) {
            const int kk = i / TM, mm = i % TM;
            const int64_t k = k0 + kk;
            As[kk][mm] = (k < k_end && m0 + mm < d) ? X[k * d + m0 + mm] : 0.f;
        }
        for (int i = tid; i < GK * TN; i += 256) {
            const int kk = i / TN, nn = i % TN;
            const int64_t k = k0 + kk;
            Bs[kk][nn] = (k < k_end && n0 + nn < bs) ? X[k * d + p0 + n0 + nn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        if (F64) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) { acc64[i][j] += (double)acc[i][j]; acc[i][j] = 0.f; }
        }
        __syncthreads();
    }
    const int64_t base = (int64_t)blockIdx.z * d * bs;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= d) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + tx * 4 + j;
            if (nn >= bs) continue;
            if (F64) static_cast<double *>(ws)[base + (int64_t)m * bs + nn] = acc64[i][j];
            else static_cast<float *>(ws)[base + (int64_t)m * bs + nn] = acc[i][j];
        }
    }
}

// Large-d split-K Gramian (d % 512 == 0, bs % 32 == 0): 512 (coordinates) x 32
// (block columns) output tile per block, 256 threads with 8 x 8 outputs each
// (packed FP32 pairs), 16-row slabs of X staged by cp.async into two buffers so
// the next slab loads while the current one is multiplied.  Partials as k_gram_tile.
constexpr int GB_TM = 512, GB_TN = 32, GB_KS = 16;
constexpr int GB_SMEM = 2 * GB_KS * (GB_TM + GB_TN) * 4;

__device__ __forceinline__ void cp_async16_dense(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void fma2_dense(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rd, {%0, %1};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rd;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

__global__ void __launch_bounds__(256, 2) k_gram_big(const float *__restrict__ X, int64_t n, int32_t d,
                                                     int32_t p0, int32_t bs, int64_t rows_per,
                                                     float *__restrict__ ws) {
    extern __shared__ float4 gsm4[];
    float *As = reinterpret_cast<float *>(gsm4);          // [2][KS][TM]
    float *Bs = As + 2 * GB_KS * GB_TM;                    // [2][KS][TN]
    const int tid = threadIdx.x, tx = tid & 3, ty = tid >> 2;
    const int m0 = blockIdx.x * GB_TM, n0 = blockIdx.y * GB_TN;
    const int64_t k_beg = (int64_t)blockIdx.z * rows_per;
    const int64_t k_end = min(n, k_beg + rows_per);
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    auto load = [&](int64_t k0, int bi) {
        float *a = As + bi * GB_KS * GB_TM, *b = Bs + bi * GB_KS * GB_TN;
#pragma unroll
        for (int q = 0; q < 8; ++q) {  // 16 rows x 128 float4
            const int f = tid + 256 * q, kk = f >> 7, v = f & 127;
            const int64_t k = k0 + kk;
            if (k < k_end) cp_async16_dense(a + kk * GB_TM + 4 * v, X + k * d + m0 + 4 * v);
            else *reinterpret_cast<float4 *>(a + kk * GB_TM + 4 * v) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (tid < GB_KS * GB_TN / 4) {
            const int kk = tid >> 3, v = tid & 7;
            const int64_t k = k0 + kk;
            if (k < k_end) cp_async16_dense(b + kk * GB_TN + 4 * v, X + k * d + p0 + n0 + 4 * v);
            else *reinterpret_cast<float4 *>(b + kk * GB_TN + 4 * v) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    int bi = 0;
    if (k_beg < k_end) load(k_beg, 0);
    for (int64_t k0 = k_beg; k0 < k_end; k0 += GB_KS) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        if (k0 + GB_KS < k_end) load(k0 + GB_KS, bi ^ 1);
        const float *a = As + bi * GB_KS * GB_TM + ty * 8, *b = Bs + bi * GB_KS * GB_TN + tx * 8;
#pragma unroll
        for (int kk = 0; kk < GB_KS; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(a + kk * GB_TM);
            const float4 a1 = *reinterpret_cast<const float4 *>(a + kk * GB_TM + 4);
            const float4 b0 = *reinterpret_cast<const float4 *>(b + kk * GB_TN);
            const float4 b1 = *reinterpret_cast<const float4 *>(b + kk * GB_TN + 4);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; j += 2) fma2_dense(acc[i][j], acc[i][j + 1], av[i], av[i], bv[j], bv[j + 1]);
        }
        bi ^= 1;
    }
    float *out = ws + (int64_t)blockIdx.z * d * bs;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty * 8 + i;
        float4 *o = reinterpret_cast<float4 *>(out + (int64_t)m * bs + n0 + tx * 8);
        o[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        o[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
}

// Large-d row terms (d % 16 == 0, bs % 32 == 0): 256 rows x 32 block columns per
// block (a 1-D grid, column block fastest), 256 threads with 8 rows x 4 columns each; X rows and G in 16-wide
// k-slabs staged by cp.async into two buffers (rows padded to 20 floats).
constexpr int RB_TM = 256, RB_TN = 32, RB_KS = 16, RB_SA = RB_KS + 4;

__global__ void __launch_bounds__(256, 2) k_rowterm_big(const float *__restrict__ X,
                                                        const int64_t *__restrict__ ptr, int32_t n_rows,
                                                        int32_t d, int32_t p0, int32_t bs,
                                                        const float *__restrict__ G, float alpha0,
                                                        float lambda, float nu, float *__restrict__ R) {
    __shared__ __align__(16) float As[2][RB_TM * RB_SA];
    __shared__ __align__(16) float Bs[2][RB_KS * RB_TN];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    // the column blocks of one row tile are consecutive blocks, so the tile's rows are
    // read from DRAM once and then hit in L2
    const int ncb = bs / RB_TN;
    const int64_t r0 = (int64_t)(blockIdx.x / ncb) * RB_TM;
    const int n0 = (int)(blockIdx.x % ncb) * RB_TN;
    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    auto load = [&](int k0, int bi) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // 256 rows x 4 float4
            const int f = tid + 256 * q, rr = f >> 2, v = f & 3;
            const int64_t r = r0 + rr;
            float *dst = &As[bi][rr * RB_SA + 4 * v];
            if (r < n_rows) cp_async16_dense(dst, X + r * d + k0 + 4 * v);
            else *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (tid < RB_KS * RB_TN / 4) {
            const int kk = tid >> 3, v = tid & 7;
            cp_async16_dense(&Bs[bi][kk * RB_TN + 4 * v], G + (int64_t)(k0 + kk) * bs + n0 + 4 * v);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    int bi = 0;
    load(0, 0);
    for (int k0 = 0; k0 < d; k0 += RB_KS) {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        __syncthreads();
        if (k0 + RB_KS < d) load(k0 + RB_KS, bi ^ 1);
#pragma unroll
        for (int kq = 0; kq < RB_KS; kq += 4) {
            float4 av[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) av[i] = *reinterpret_cast<const float4 *>(&As[bi][(ty * 8 + i) * RB_SA + kq]);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float4 b = *reinterpret_cast<const float4 *>(&Bs[bi][(kq + k) * RB_TN + tx * 4]);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float a = k == 0 ? av[i].x : (k == 1 ? av[i].y : (k == 2 ? av[i].z : av[i].w));
                    fma2_dense(acc[i][0], acc[i][1], a, a, b.x, b.y);
                    fma2_dense(acc[i][2], acc[i][3], a, a, b.z, b.w);
                }
            }
        }
        bi ^= 1;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = r0 + ty * 8 + i;
        if (r >= n_rows) continue;
        const float lam = lambda * (1.0f + nu * (float)(ptr[r + 1] - ptr[r]));
        const float4 x = *reinterpret_cast<const float4 *>(X + r * d + p0 + n0 + tx * 4);
        *reinterpret_cast<float4 *>(R + r * bs + n0 + tx * 4) =
            make_float4(alpha0 * acc[i][0] + lam * x.x, alpha0 * acc[i][1] + lam * x.y,
                        alpha0 * acc[i][2] + lam * x.z, alpha0 * acc[i][3] + lam * x.w);
    }
}

// Fixed-order reduction of the split-K partials.
template <typename T>
__global__ void k_gram_reduce(const T *__restrict__ ws, int32_t nsplit, int64_t count,
                              T *__restrict__ G) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    T t = 0;
    for (int s = 0; s < nsplit; ++s) t += ws[(int64_t)s * count + i];
    G[i] = t;
}

}  // namespace

// Kernel attributes of the dense kernels (dynamic shared memory of the large-d
// Gramian); call once outside any stream capture.
cudaError_t dense_prepare() {
    static cudaError_t done = cudaErrorNotReady;
    if (done != cudaSuccess) done = cudaFuncSetAttribute(k_gram_big, cudaFuncAttributeMaxDynamicSharedMemorySize, GB_SMEM);
    return done;
}

namespace {

struct GramPlan {
    int tm_size, tn_size, tm, tn, nsplit;
    int64_t rows_per;
};

inline void tile_shape(int32_t bs, int &TM, int &TN) {
    if (bs <= 16) { TM = 256; TN = 16; }
    else if (bs <= 32) { TM = 128; TN = 32; }
    else { TM = 64; TN = 64; }
}

// The large-d kernel's shapes (FP32 partial Gramians only).
inline bool gram_big(int32_t d, int32_t bs) { return d % GB_TM == 0 && bs % GB_TN == 0; }

GramPlan gram_plan(int64_t n, int32_t d, int32_t bs, bool allow_big = true) {
    GramPlan p;
    tile_shape(bs, p.tm_size, p.tn_size);
    if (allow_big && gram_big(d, bs)) {
        p.tm_size = GB_TM;
        p.tn_size = GB_TN;
    }
    p.tm = (d + p.tm_size - 1) / p.tm_size;
    p.tn = (bs + p.tn_size - 1) / p.tn_size;
    const int64_t tiles = (int64_t)p.tm * p.tn;
    int64_t ns = (2 * kSMs + tiles - 1) / tiles;
    const int64_t kblocks = (n + GK - 1) / GK;
    if (ns > kblocks) ns = kblocks;
    if (ns < 1) ns = 1;
    const int64_t per_blocks = (kblocks + ns - 1) / ns;
    p.rows_per = per_blocks * GK;
    p.nsplit = (int)((n + p.rows_per - 1) / p.rows_per);
    if (p.nsplit < 1) p.nsplit = 1;
    return p;
}

template <bool F64>
void launch_gram_tiles(const GramPlan &p, const float *X, int64_t n, int32_t d, int32_t p0,
                       int32_t bs, void *ws, cudaStream_t s) {
    const dim3 grid(p.tm, p.tn, p.nsplit);
    if (!F64 && p.tm_size == GB_TM) {
        dense_prepare();  // a no-op after the first call (made at context creation)
        k_gram_big<<<grid, 256, GB_SMEM, s>>>(X, n, d, p0, bs, p.rows_per, static_cast<float *>(ws));
        return;
    }
    if (p.tn_size == 16) k_gram_tile<256, 16, F64><<<grid, 256, 0, s>>>(X, n, d, p0, bs, p.rows_per, ws);
    else if (p.tn_size == 32) k_gram_tile<128, 32, F64><<<grid, 256, 0, s>>>(X, n, d, p0, bs, p.rows_per, ws);
    else k_gram_tile<64, 64, F64><<<grid, 256, 0, s>>>(X, n, d, p0, bs, p.rows_per, ws);
}

// ------------------------------------------------------------------ row terms
// R[r, f] = alpha0 * sum_k X[r, k] G[k, f] + lambda (1 + nu n_r) X[r, p0 + f]
// TM x TN output tile per block (rows x coordinates), K = d in slabs of 16.
template <int TM, int TN>
__global__ void __launch_bounds__(256) k_rowterm(const float *__restrict__ X,
                                                 const int64_t *__restrict__ ptr, int32_t n_rows,
                                                 int32_t d, int32_t p0, int32_t bs,
                                                 const float *__restrict__ G, float alpha0,
                                                 float lambda, float nu, float *__restrict__ R) {
    static_assert((TM / 4) * (TN / 4) == 256, "tile shape");
    __shared__ __align__(16) float As[GK][TM + 4];
    __shared__ __align__(16) float Bs[GK][TN];
    const int tid = threadIdx.x, tx = tid % (TN / 4), ty = tid / (TN / 4);
    const int64_t r0 = (int64_t)blockIdx.x * TM;
    const int n0 = blockIdx.y * TN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < d; k0 += GK) {
        for (int i = tid; i < GK * TM; i += 256) {
            const int rr = i / GK, kk = i % GK;
            const int64_t r = r0 + rr;
            const int k = k0 + kk;
            As[kk][rr] = (r < n_rows && k < d) ? X[r * d + k] : 0.f;
        }
        for (int i = tid; i < GK * TN; i += 256) {
            const int kb = i / TN, nn = i % TN;
            Bs[kb][nn] = (k0 + kb < d && n0 + nn < bs) ? G[(int64_t)(k0 + kb) * bs + n0 + nn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t r = r0 + ty * 4 + i;
        if (r >= n_rows) continue;
        const float lam = lambda * (1.0f + nu * (float)(ptr[r + 1] - ptr[r]));
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int f = n0 + tx * 4 + j;
            if (f >= bs) continue;
            R[r * bs + f] = alpha0 * acc[i][j] + lam * X[r * d + p0 + f];
        }
    }
}

// ------------------------------------------------------------------- init
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void k_init_normal(float *X, int64_t count, double std, uint64_t key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const uint64_t a = splitmix64(key ^ (2 * (uint64_t)i));
    const uint64_t b = splitmix64(key ^ (2 * (uint64_t)i + 1));
    const double u1 = ((double)(a >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(b >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    X[i] = (float)(std * sqrt(-2.0 * log(u1)) * cospi(2.0 * u2));
}

__global__ void k_split_bf16(const float *__restrict__ X, int64_t count, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = X[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

int residual_grid(int32_t n_rows) {
    int g = (n_rows + 7) / 8;
    return g < 4 * kSMs ? (g > 0 ? g : 1) : 4 * kSMs;
}

cudaError_t launch_sq_loss_parts(const int64_t *u_ptr, const int32_t *u_idx, const float *W,
                                 const float *H, const float *y, const float *alpha,
                                 int32_t n_users, int32_t d, double *part, int grid, cudaStream_t s) {
    // sub-group size: about four float4 chunks per lane, at most 32 lanes
    const int nv4 = d / 4;
    int sg_log = 0;
    while ((2 << sg_log) <= 32 && (2 << sg_log) * 4 <= nv4) ++sg_log;
    const int SG = 1 << sg_log;
    const int maxv = (nv4 + SG - 1) / SG;
#define IALS_RES(SGL, MV)                                                                    \
    k_residual<SGL, MV><<<grid, 256, 0, s>>>(u_ptr, u_idx, W, H, y, alpha, n_users, d, part)
    // maxv < 8 whenever sg_log < 5 (the loop above stops at 4 chunks per lane)
    if (sg_log == 0) {
        if (maxv <= 1) IALS_RES(0, 1);
        else if (maxv <= 2) IALS_RES(0, 2);
        else if (maxv <= 4) IALS_RES(0, 4);
        else IALS_RES(0, 8);
    } else if (sg_log == 1) { if (maxv <= 4) IALS_RES(1, 4); else IALS_RES(1, 8); }
    else if (sg_log == 2) { if (maxv <= 4) IALS_RES(2, 4); else IALS_RES(2, 8); }
    else if (sg_log == 3) { if (maxv <= 4) IALS_RES(3, 4); else IALS_RES(3, 8); }
    else if (sg_log == 4) { if (maxv <= 4) IALS_RES(4, 4); else IALS_RES(4, 8); }
    else if (maxv <= 4) IALS_RES(5, 4);
    else if (maxv <= 8) IALS_RES(5, 8);
    else if (maxv <= 16) IALS_RES(5, 16);
    else if (maxv <= 32) IALS_RES(5, 32);
    else return cudaErrorInvalidValue;
#undef IALS_RES
    return cudaGetLastError();
}

template <int SGL, int MV>
cudaError_t launch_residual_tasks_t(const Task *tasks, int32_t n_tasks, const int32_t *u_idx,
                                    const float *W, const float *H, const float *y, int32_t d,
                                    float *e, int32_t *counter, cudaStream_t s) {
    static int per_sm = 0;  // resident blocks per SM (same for every context)
    if (per_sm == 0) {
        int n = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_residual_tasks<SGL, MV>, 256, 0);
        if (err != cudaSuccess) return err;
        per_sm = n > 0 ? n : 1;
    }
    int grid = per_sm * kSMs;
    const int need = (n_tasks + 7) / 8;
    if (grid > need) grid = need > 0 ? need : 1;
    k_residual_tasks<SGL, MV><<<grid, 256, 0, s>>>(tasks, n_tasks, u_idx, W, H, y, d, e, counter);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_residual_tasks(const Task *tasks, int32_t n_tasks, const int32_t *u_idx,
                                  const float *W, const float *H, const float *y, int32_t d, float *e,
                                  int32_t *counter, cudaStream_t s) {
    if (n_tasks == 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(counter, 0, sizeof(int32_t), s);
    if (err != cudaSuccess) return err;
    // same sub-group choice as launch_sq_loss_parts
    const int nv4 = d / 4;
    int sg_log = 0;
    while ((2 << sg_log) <= 32 && (2 << sg_log) * 4 <= nv4) ++sg_log;
    const int SG = 1 << sg_log;
    const int maxv = (nv4 + SG - 1) / SG;
#define IALS_REST(SGL, MV) return launch_residual_tasks_t<SGL, MV>(tasks, n_tasks, u_idx, W, H, y, d, e, counter, s)
    if (sg_log == 0) {
        if (maxv <= 1) IALS_REST(0, 1);
        else if (maxv <= 2) IALS_REST(0, 2);
        else if (maxv <= 4) IALS_REST(0, 4);
        else IALS_REST(0, 8);
    } else if (sg_log == 1) { if (maxv <= 4) IALS_REST(1, 4); else IALS_REST(1, 8); }
    else if (sg_log == 2) { if (maxv <= 4) IALS_REST(2, 4); else IALS_REST(2, 8); }
    else if (sg_log == 3) { if (maxv <= 4) IALS_REST(3, 4); else IALS_REST(3, 8); }
    else if (sg_log == 4) { if (maxv <= 4) IALS_REST(4, 4); else IALS_REST(4, 8); }
    else if (maxv <= 4) IALS_REST(5, 4);
    else if (maxv <= 8) IALS_REST(5, 8);
    else if (maxv <= 16) IALS_REST(5, 16);
    else if (maxv <= 32) IALS_REST(5, 32);
#undef IALS_REST
    return cudaErrorInvalidValue;
}

cudaError_t launch_sq_loss(const int64_t *u_ptr, const int32_t *u_idx, const float *W,
                           const float *H, const float *y, const float *alpha,
                           int32_t n_users, int32_t d, double *part, int32_t n_part,
                           double *out, cudaStream_t s) {
    int grid = residual_grid(n_users);
    if (grid > n_part) grid = n_part;
    cudaError_t err = launch_sq_loss_parts(u_ptr, u_idx, W, H, y, alpha, n_users, d, part, grid, s);
    if (err != cudaSuccess) return err;
    k_sum_parts<<<1, 256, 0, s>>>(part, grid, 1.0, out, 0);
    return cudaGetLastError();
}

cudaError_t launch_reg_loss(const int64_t *ptr, const float *X, int32_t n_rows, int32_t d,
                            double lambda, double nu, double *part, int32_t n_part, double *out,
                            cudaStream_t s) {
    int grid = residual_grid(n_rows);
    if (grid > n_part) grid = n_part;
    k_reg_loss<<<grid, 256, 0, s>>>(ptr, X, n_rows, d, lambda, nu, part);
    k_sum_parts<<<1, 256, 0, s>>>(part, grid, 1.0, out, 1);
    return cudaGetLastError();
}

cudaError_t launch_frobenius(const double *A, const double *B, int32_t n, double alpha0,
                             double *out, cudaStream_t s) {
    k_frobenius<<<1, 256, 0, s>>>(A, B, (int64_t)n * n, alpha0, out);
    return cudaGetLastError();
}

int64_t gram_ws_floats(int64_t n, int32_t d, int32_t bs) {
    GramPlan p = gram_plan(n, d, bs);
    return (int64_t)p.nsplit * d * bs;
}

cudaError_t launch_gram(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs, float *G,
                        float *ws, cudaStream_t s) {
    const int64_t count = (int64_t)d * bs;
    if (n == 0) return cudaMemsetAsync(G, 0, sizeof(float) * count, s);
    GramPlan p = gram_plan(n, d, bs);
    launch_gram_tiles<false>(p, X, n, d, p0, bs, ws, s);
    k_gram_reduce<float><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ws, p.nsplit, count, G);
    return cudaGetLastError();
}

int64_t gram_ws_floats_capped(int64_t n, int32_t d, int32_t bs, int64_t max_floats) {
    GramPlan p = gram_plan(n, d, bs);
    const int64_t per_split = (int64_t)d * bs;
    if (per_split > max_floats) return -1;
    if ((int64_t)p.nsplit * per_split > max_floats) p.nsplit = (int)(max_floats / per_split);
    return (int64_t)p.nsplit * per_split;
}

cudaError_t launch_gram_capped(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                               float *G, float *ws, int64_t max_floats, cudaStream_t s) {
    const int64_t count = (int64_t)d * bs;
    if (count > max_floats) return cudaErrorInvalidValue;
    if (n == 0) return cudaMemsetAsync(G, 0, sizeof(float) * count, s);
    GramPlan p = gram_plan(n, d, bs);
    if ((int64_t)p.nsplit * count > max_floats) {
        // fewer, longer row ranges so that the partials fit the given workspace
        const int64_t ns = max_floats / count;
        const int64_t kblocks = (n + GK - 1) / GK;
        p.rows_per = (kblocks + ns - 1) / ns * GK;
        p.nsplit = (int)((n + p.rows_per - 1) / p.rows_per);
    }
    launch_gram_tiles<false>(p, X, n, d, p0, bs, ws, s);
    k_gram_reduce<float><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ws, p.nsplit, count, G);
    return cudaGetLastError();
}

// Fixed-order sum of nsplit partial rows x cols blocks into columns col0 .. col0+cols-1
// of G (row stride ldg).
__global__ void k_gram_reduce_cols(const float *__restrict__ ws, int32_t nsplit, int32_t rows, int32_t cols,
                                   float *__restrict__ G, int32_t ldg, int32_t col0) {
    const int64_t count = (int64_t)rows * cols;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float t = 0.f;
    for (int s = 0; s < nsplit; ++s) t += ws[(int64_t)s * count + i];
    G[(i / cols) * ldg + col0 + (i % cols)] = t;
}

cudaError_t launch_gram_reduce_cols(const float *ws, int nsplit, int32_t rows, int32_t cols, float *G, int32_t ldg,
                                    int32_t col0, cudaStream_t s) {
    const int64_t count = (int64_t)rows * cols;
    k_gram_reduce_cols<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ws, nsplit, rows, cols, G, ldg, col0);
    return cudaGetLastError();
}

int64_t gram64_ws_doubles(int64_t n, int32_t d) {
    GramPlan p = gram_plan(n, d, d, false);
    return (int64_t)p.nsplit * d * d;
}

cudaError_t launch_gram64(const float *X, int64_t n, int32_t d, double *G64, double *ws,
                          cudaStream_t s) {
    const int64_t count = (int64_t)d * d;
    if (n == 0) return cudaMemsetAsync(G64, 0, sizeof(double) * count, s);
    GramPlan p = gram_plan(n, d, d, false);
    launch_gram_tiles<true>(p, X, n, d, 0, d, ws, s);
    k_gram_reduce<double><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(ws, p.nsplit, count, G64);
    return cudaGetLastError();
}

cudaError_t launch_rowterm(const float *X, const int64_t *ptr, int32_t n_rows, int32_t d,
                           int32_t p0, int32_t bs, const float *G, float alpha0, float lambda,
                           float nu, float *R, cudaStream_t s) {
    if (n_rows == 0) return cudaSuccess;
    if (d % RB_KS == 0 && bs % RB_TN == 0) {
        const unsigned grid = (unsigned)(((int64_t)n_rows + RB_TM - 1) / RB_TM * (bs / RB_TN));
        k_rowterm_big<<<grid, 256, 0, s>>>(X, ptr, n_rows, d, p0, bs, G, alpha0, lambda, nu, R);
        return cudaGetLastError();
    }
    int TM, TN;
    tile_shape(bs, TM, TN);
    dim3 grid((n_rows + TM - 1) / TM, (bs + TN - 1) / TN);
    if (TN == 16) k_rowterm<256, 16><<<grid, 256, 0, s>>>(X, ptr, n_rows, d, p0, bs, G, alpha0, lambda, nu, R);
    else if (TN == 32) k_rowterm<128, 32><<<grid, 256, 0, s>>>(X, ptr, n_rows, d, p0, bs, G, alpha0, lambda, nu, R);
    else k_rowterm<64, 64><<<grid, 256, 0, s>>>(X, ptr, n_rows, d, p0, bs, G, alpha0, lambda, nu, R);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float *X, int64_t count, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                              cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    k_split_bf16<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(X, count, hi, lo);
    return cudaGetLastError();
}

cudaError_t launch_init_normal(float *X, int64_t count, double std, uint64_t seed,
                               uint64_t stream_id, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const uint64_t key = seed * 0x9E3779B97F4A7C15ull + stream_id * 0xD1B54A32D192ED03ull + 1;
    k_init_normal<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(X, count, std, key);
    return cudaGetLastError();
}

}  // namespace ials
