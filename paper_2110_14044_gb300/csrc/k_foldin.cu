// Fold-in of new users against frozen item factors (the evaluation protocol of
// Section 5.1.1 gives held-out users' interactions at evaluation time; the
// procedure used is: w = 0, then `sweeps` passes of the user-side block steps
// of Algorithm 3 with H and G^I = H^T H fixed).
//
// One CTA per request; nothing is shared between requests, so a result does
// not depend on what it is batched with.  Because H is frozen, the block
// Hessian A_pi = sum_s h_{s,pi} h_{s,pi}^T + alpha0 G^I_pipi + lambda_u I is the
// same in every sweep: it is accumulated (8 x 8 thread tiles over its lower
// triangle, slices staged with cp.async) and factorised (blocked shared-memory
// Cholesky) once per block, kept in the request's workspace, and reused.  Each
// sweep then only forms the gradient
//   g = alpha0 (w G^I)_pi + lambda_u w_pi + sum_s e_s h_{s,pi}
// solves L L^T delta = g, applies w_pi -= delta and updates the request's
// residuals e_s -= <delta, h_{s,pi}> (e starts at -y since w = 0).
#include "k_sparse_cta.cuh"

namespace ials {

namespace {

template <int B>
struct FoldCfg {
    static constexpr int NB = B / 8;
    static constexpr int NTL = NB * (NB + 1) / 2;
    static constexpr int NG0 = 256 / NTL;
    static constexpr int NG = NG0 < 8 ? NG0 : 8;
    static constexpr int ACTIVE = NTL * NG;
    static constexpr int SB = B + 4;
    static constexpr int CH = 32;
    static constexpr int BUF = CH * SB;
    // floats: 2 staging buffers, M (B+1 rows), diag0, invd, x, gradient partials (8 x B), flag
    static constexpr int FIXED_FLOATS = 2 * BUF + (B + 1) * SB + 3 * B + 8 * B + 4;
};

// Forward substitution L z = g (g in x on entry), panel by panel.
template <int B, int SM>
__device__ void cta_forwardsolve(const float *M, const float *invd, float *x) {
    constexpr int NB = B / 8;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int p = 0; p < NB; ++p) {
        const int k0 = 8 * p;
        if (tid == 0) {
            for (int j = 0; j < 8; ++j) {
                float v = x[k0 + j];
                for (int m = 0; m < j; ++m) v -= M[(k0 + j) * SM + k0 + m] * x[k0 + m];
                x[k0 + j] = v * invd[k0 + j];
            }
        }
        __syncthreads();
        for (int i = k0 + 8 + tid; i < B; i += nt) {
            float v = x[i];
#pragma unroll
            for (int m = 0; m < 8; ++m) v -= M[i * SM + k0 + m] * x[k0 + m];
            x[i] = v;
        }
        __syncthreads();
    }
}

template <int B>
__global__ void __launch_bounds__(256) k_foldin(FoldArgs a) {
    using C = FoldCfg<B>;
    constexpr int SB = C::SB, CH = C::CH;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *buf0 = smem;
    float *M = buf0 + 2 * C::BUF;
    float *diag0 = M + (B + 1) * SB;
    float *invd = diag0 + B;
    float *xv = invd + B;
    float *gp = xv + B;                 // 8 x B gradient partials
    int *flag = reinterpret_cast<int *>(gp + 8 * B);
    float *wv = reinterpret_cast<float *>(flag + 4);  // d floats
    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = a.d, nb = d / B;
    const bool active = tid < C::ACTIVE;
    const int grp = active ? tid / C::NTL : C::NG;
    const int kstart = active ? grp : CH;
    int ti = 0, tj = 0;
    tri_index(tid % C::NTL, ti, tj);
    for (int r = blockIdx.x; r < a.n_req; r += gridDim.x) {
        const FoldReq rq = a.req[r];
        const int n = rq.n;
        uint8_t *base = a.arena + rq.off;
        const int32_t *items = reinterpret_cast<const int32_t *>(base);
        const float *yv = reinterpret_cast<const float *>(base + rq.y_off);
        float *ev = reinterpret_cast<float *>(base + rq.e_off);
        float *Lg = reinterpret_cast<float *>(base + rq.l_off);  // nb x (B*B + B): L rows, then 1/L_kk
        float *wout = reinterpret_cast<float *>(base + rq.w_off);
        const float lam = a.lambda * (1.0f + a.nu * (float)n);
        for (int s = tid; s < n; s += nt) ev[s] = rq.has_y ? -yv[s] : -1.0f;
        for (int j = tid; j < d; j += nt) wv[j] = 0.f;
        if (tid == 0) flag[1] = 0;
        __syncthreads();
        // ---- per block: Hessian, factor, keep
        for (int k = 0; k < nb; ++k) {
            const int p0 = k * B;
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            const int nch = (n + CH - 1) / CH;
            auto gather = [&](int ch, float *bufp) {
                const int cnt = min(CH, n - ch * CH);
                for (int f = tid; f < cnt * (B / 4); f += nt) {
                    const int kk = f / (B / 4), v = f % (B / 4);
                    const int64_t item = items[ch * CH + kk];
                    cp_async16(bufp + kk * SB + 4 * v, a.H + item * d + p0 + 4 * v);
                }
                cp_async_commit();
            };
            if (nch > 0) gather(0, buf0);
            for (int ch = 0; ch < nch; ++ch) {
                cp_async_wait_all();
                __syncthreads();
                if (ch + 1 < nch) gather(ch + 1, buf0 + ((ch + 1) & 1) * C::BUF);
                const int cnt = min(CH, n - ch * CH);
                const float *bp = buf0 + (ch & 1) * C::BUF;
                for (int kk = kstart; kk < cnt; kk += C::NG) {
                    float xa[8], xb[8];
                    load_seg<8>(bp + kk * SB + 8 * ti, xa);
                    load_seg<8>(bp + kk * SB + 8 * tj, xb);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] += xa[i] * xb[j];
                }
            }
            __syncthreads();
#pragma unroll 1
            for (int ph = 0; ph < C::NG; ++ph) {
                if (grp == ph) {
#pragma unroll
                    for (int i = 0; i < 8; ++i) store_tile<8>(M + (8 * ti + i) * SB + 8 * tj, acc[i], ph > 0);
                }
                __syncthreads();
            }
            if (nch == 0) {  // no interactions: the statistics are zero
                for (int e = tid; e < B * B; e += nt) M[(e / B) * SB + (e % B)] = 0.f;
                __syncthreads();
            }
            for (int e = tid; e < B * B; e += nt) {
                const int i = e / B, j = e % B;
                if (j > i) continue;
                float v = M[i * SB + j] + a.alpha0 * a.G[(int64_t)(p0 + i) * d + p0 + j];
                if (i == j) {
                    v += lam;
                    diag0[i] = v;
                }
                M[i * SB + j] = v;
            }
            for (int j = tid; j < B; j += nt) M[B * SB + j] = 0.f;
            __syncthreads();
            cta_cholesky<B, SB, float>(M, invd, diag0, &flag[1], 1e-5f);
            float *Lk = Lg + (int64_t)k * (B * B + B);
            for (int e = tid; e < B * B; e += nt) Lk[e] = M[(e / B) * SB + (e % B)];
            for (int j = tid; j < B; j += nt) Lk[B * B + j] = invd[j];
            __syncthreads();
        }
        // ---- sweeps of gradient, solve, apply, residual update
        for (int sw = 0; sw < a.sweeps && !flag[1]; ++sw) {
            for (int k = 0; k < nb; ++k) {
                const int p0 = k * B;
                // gradient: thread (g, j) with j < B, g < nt / B sums a strided share
                const int gsz = nt / B < 8 ? nt / B : 8;  // gp holds 8 partial rows
                const int j = tid % B, g = tid / B;
                if (g < gsz) {
                    float t = 0.f;
                    for (int s = g; s < n; s += gsz) t += ev[s] * a.H[(int64_t)items[s] * d + p0 + j];
                    if (g == 0) {
                        float u = 0.f;
                        for (int q = 0; q < d; ++q) u += wv[q] * a.G[(int64_t)q * d + p0 + j];
                        t += a.alpha0 * u + lam * wv[p0 + j];
                    }
                    gp[g * B + j] = t;
                }
                const float *Lk = Lg + (int64_t)k * (B * B + B);
                for (int e = tid; e < B * B; e += nt) M[(e / B) * SB + (e % B)] = Lk[e];
                for (int q = tid; q < B; q += nt) invd[q] = Lk[B * B + q];
                __syncthreads();
                for (int q = tid; q < B; q += nt) {
                    float t = 0.f;
                    for (int gg = 0; gg < gsz; ++gg) t += gp[gg * B + q];
                    xv[q] = t;
                }
                __syncthreads();
                cta_forwardsolve<B, SB>(M, invd, xv);
                cta_backsolve<B, SB, float>(M, invd, xv);
                for (int q = tid; q < B; q += nt) wv[p0 + q] -= xv[q];
                // residuals: one warp per interaction, lanes split the block
                const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
                for (int s = warp; s < n; s += nw) {
                    const float *h = a.H + (int64_t)items[s] * d + p0;
                    float t = 0.f;
                    for (int q = lane; q < B; q += 32) t += xv[q] * h[q];
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
                    if (lane == 0) ev[s] -= t;
                }
                __syncthreads();
            }
        }
        for (int j = tid; j < d; j += nt) wout[j] = wv[j];
        if (tid == 0) a.status[r] = flag[1] ? 4 : 0;
        __syncthreads();
    }
}

template <int B>
int foldin_smem(int d) {
    return (FoldCfg<B>::FIXED_FLOATS + d) * 4 + 16;
}

template <int B>
cudaError_t launch_foldin_b(const FoldArgs &a, int grid, cudaStream_t s) {
    const int sm = foldin_smem<B>(a.d);
    cudaError_t e = cudaFuncSetAttribute(k_foldin<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_foldin<B><<<grid, 256, sm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_foldin(const FoldArgs &a, cudaStream_t s) {
    if (a.n_req <= 0) return cudaSuccess;
    const int grid = a.n_req;
    switch (a.b) {
        case 16: return launch_foldin_b<16>(a, grid, s);
        case 32: return launch_foldin_b<32>(a, grid, s);
        case 64: return launch_foldin_b<64>(a, grid, s);
        case 128: return launch_foldin_b<128>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int64_t foldin_factor_floats(int32_t d, int32_t b) { return (int64_t)(d / b) * (b * b + b); }

}  // namespace ials
