// Fold-in of new users against frozen item factors (the evaluation protocol of
// Section 5.1.1 gives held-out users' interactions at evaluation time; the
// procedure used is: w = 0, then `sweeps` passes of the user-side block steps
// of Algorithm 3 with H and G^I = H^T H fixed).
//
// One CTA per request; nothing is shared between requests, so a result does
// not depend on what it is batched with.  Because H is frozen, the block
// Hessian A_pi = sum_s h_{s,pi} h_{s,pi}^T + alpha0 G^I_pipi + lambda_u I is the
// same in every sweep: it is accumulated (8 x 8 thread tiles over its lower
// triangle, slices staged with cp.async) and factorised (Cholesky in 16-column
// panels) once per block, kept in the request's workspace, and reused.  Each
// sweep then only forms the gradient (from staged slices; u = w G^I is kept
// up to date after every apply)
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
    static constexpr int SB = B % 32 == 0 ? B + 4 : B + 20;  // = 4 mod 32 (layout of cta_chol16)
    static constexpr int CH = B <= 64 ? 128 : 64;  // interactions staged per chunk
    static constexpr int BUF = CH * SB;
    // floats: 2 staging buffers, staged residuals (2 x CH), M (B+1 rows), diag0, invd, x,
    // gradient partials (8 x B), flag; then w and u = w G^I (d floats each)
    static constexpr int FIXED_FLOATS = 2 * BUF + 2 * CH + (B + 1) * SB + 3 * B + 8 * B + 4;
};

template <int B>
__global__ void __launch_bounds__(256) k_foldin(FoldArgs a) {
    using C = FoldCfg<B>;
    constexpr int SB = C::SB, CH = C::CH;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    float *buf0 = smem;
    float *she = buf0 + 2 * C::BUF;     // residuals of the staged chunks [2][CH]
    float *M = she + 2 * CH;
    float *diag0 = M + (B + 1) * SB;
    float *invd = diag0 + B;
    float *xv = invd + B;
    float *gp = xv + B;                 // 8 x B gradient partials
    int *flag = reinterpret_cast<int *>(gp + 8 * B);
    float *wv = reinterpret_cast<float *>(flag + 4);  // w (d floats)
    float *uv = wv + a.d;                              // u = w G^I (d floats)
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
        for (int j = tid; j < d; j += nt) wv[j] = uv[j] = 0.f;
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
            cta_chol16<B, SB>(M, invd, diag0, &flag[1], 1e-5f);
            float *Lk = Lg + (int64_t)k * (B * B + B);
            for (int e = tid; e < B * B; e += nt) Lk[e] = M[(e / B) * SB + (e % B)];
            for (int j = tid; j < B; j += nt) Lk[B * B + j] = invd[j];
            __syncthreads();
        }
        // ---- sweeps of gradient, solve, apply, residual update.  The request's
        // slices of block k are staged chunk by chunk (cp.async, two buffers) for
        // the gradient pass and again for the residual pass; u = w G^I is kept up
        // to date after every apply, so the alpha0 (w G^I)_pi term is a lookup.
        const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
        const int gsz = nt / B < 8 ? nt / B : 8;  // gradient groups (gp holds 8 partial rows)
        const int gj = tid % B, gg = tid / B;
        const int nch = (n + CH - 1) / CH;
        auto stage = [&](int ch, int p0, int bi, bool with_e) {
            const int cnt = min(CH, n - ch * CH);
            float *bufp = buf0 + bi * C::BUF;
            for (int f = tid; f < cnt * (B / 4); f += nt) {
                const int kk = f / (B / 4), v = f % (B / 4);
                const int64_t item = items[ch * CH + kk];
                cp_async16(bufp + kk * SB + 4 * v, a.H + item * d + p0 + 4 * v);
            }
            if (with_e && tid < cnt) she[bi * CH + tid] = ev[ch * CH + tid];
            cp_async_commit();
        };
        for (int sw = 0; sw < a.sweeps && !flag[1]; ++sw) {
            for (int k = 0; k < nb; ++k) {
                const int p0 = k * B;
                float t = 0.f;
                if (nch > 0) stage(0, p0, 0, true);
                for (int ch = 0; ch < nch; ++ch) {
                    const int bi = ch & 1;
                    cp_async_wait_all();
                    __syncthreads();
                    if (ch + 1 < nch) stage(ch + 1, p0, bi ^ 1, true);
                    const int cnt = min(CH, n - ch * CH);
                    const float *bp = buf0 + bi * C::BUF;
                    if (gg < gsz)
                        for (int kk = gg; kk < cnt; kk += gsz) t += she[bi * CH + kk] * bp[kk * SB + gj];
                }
                if (gg < gsz) gp[gg * B + gj] = t;
                const float *Lk = Lg + (int64_t)k * (B * B + B);
                for (int e = tid; e < B * B; e += nt) M[(e / B) * SB + (e % B)] = Lk[e];
                for (int q = tid; q < B; q += nt) invd[q] = Lk[B * B + q];
                __syncthreads();
                for (int q = tid; q < B; q += nt) {
                    float v = a.alpha0 * uv[p0 + q] + lam * wv[p0 + q];
                    for (int g2 = 0; g2 < gsz; ++g2) v += gp[g2 * B + q];
                    xv[q] = v;
                }
                __syncthreads();
                cta_forward16<B, SB>(M, invd, xv);
                cta_backsolve16<B, SB>(M, invd, xv);
                // apply, then u -= delta^T G^I[pi, :] (coalesced over the columns of G^I)
                for (int q = tid; q < B; q += nt) wv[p0 + q] -= xv[q];
                for (int q = tid; q < d; q += nt) {
                    float v = 0.f;
#pragma unroll 8
                    for (int m = 0; m < B; ++m) v += xv[m] * a.G[(int64_t)(p0 + m) * d + q];
                    uv[q] -= v;
                }
                // residuals e_s -= <delta, h_{s,pi}>: one warp per staged interaction
                if (nch > 0) stage(0, p0, 0, false);
                for (int ch = 0; ch < nch; ++ch) {
                    const int bi = ch & 1;
                    cp_async_wait_all();
                    __syncthreads();
                    if (ch + 1 < nch) stage(ch + 1, p0, bi ^ 1, false);
                    const int cnt = min(CH, n - ch * CH);
                    const float *bp = buf0 + bi * C::BUF;
                    for (int kk = warp; kk < cnt; kk += nw) {
                        float v = 0.f;
                        for (int q = lane; q < B; q += 32) v += xv[q] * bp[kk * SB + q];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
                        if (lane == 0) ev[ch * CH + kk] -= v;
                    }
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
    return (FoldCfg<B>::FIXED_FLOATS + 2 * d) * 4 + 16;
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
