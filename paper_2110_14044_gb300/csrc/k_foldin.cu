// Fold-in of new users against frozen item factors (the evaluation protocol of
// Section 5.1.1 gives held-out users' interactions at evaluation time; the
// procedure used is: w = 0, then `sweeps` passes of the user-side block steps
// of Algorithm 3 with H and G^I = H^T H fixed).
//
// Because H is frozen, the block Hessian
//   A_pi = sum_s h_{s,pi} h_{s,pi}^T + alpha0 G^I_pipi + lambda_u I
// is the same in every sweep: it is accumulated (8 x 8 thread tiles over its
// lower triangle, slices staged with cp.async) and factorised (Cholesky in
// 16-column panels) once per block, kept in the request's workspace, and
// reused.  Each sweep then only forms the gradient
//   g = alpha0 (w G^I)_pi + lambda_u w_pi + sum_s e_s h_{s,pi}
// solves L L^T delta = g, applies w_pi -= delta, keeps u = w G^I current and
// updates the request's residuals e_s -= <delta, h_{s,pi}> (e starts at -y
// since w = 0).
//
// Short requests run on one CTA each.  A request longer than kFoldLong runs on
// a cluster of kFoldCluster CTAs: each CTA takes a contiguous share of the
// interactions, the Hessian and gradient partials are summed by CTA 0 in rank
// order through distributed shared memory, and CTA 0 solves and sends delta
// back to every CTA (cluster barriers between the phases).  Which kernel a
// request takes depends on its length alone, and nothing is shared between
// requests, so a result does not depend on what it is batched with.  Each
// request writes its embedding and a completion flag straight to mapped host
// memory when it finishes, so the server can publish it at once.
#include "k_sparse_cta.cuh"

#include <cooperative_groups.h>

namespace ials {

namespace {

namespace cg = cooperative_groups;

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

// Shared-memory pieces of one fold-in CTA.
template <int B>
struct FoldSmem {
    float *buf0, *she, *M, *diag0, *invd, *xv, *gp, *wv, *uv;
    int *flag;
    __device__ __forceinline__ FoldSmem(float *smem, int d) {
        using C = FoldCfg<B>;
        buf0 = smem;
        she = buf0 + 2 * C::BUF;  // residuals of the staged chunks [2][CH]
        M = she + 2 * C::CH;
        diag0 = M + (B + 1) * C::SB;
        invd = diag0 + B;
        xv = invd + B;
        gp = xv + B;  // 8 x B gradient partials
        flag = reinterpret_cast<int *>(gp + 8 * B);
        wv = reinterpret_cast<float *>(flag + 4);  // w (d floats)
        uv = wv + d;                                // u = w G^I (d floats)
    }
};

// Slices (block starting at p0) of interactions [lo + ch * CH, ...) into buffer bi;
// with_e also stages their residuals.
template <int B>
__device__ __forceinline__ void fold_stage(const FoldArgs &a, const FoldSmem<B> &S, const int32_t *items,
                                           const float *ev, int lo, int hi, int ch, int p0, int bi,
                                           bool with_e) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int s0 = lo + ch * C::CH, cnt = min(C::CH, hi - s0);
    float *bufp = S.buf0 + bi * C::BUF;
    for (int f = tid; f < cnt * (B / 4); f += nt) {
        const int kk = f / (B / 4), v = f % (B / 4);
        const int64_t item = items[s0 + kk];
        cp_async16(bufp + kk * C::SB + 4 * v, a.H + item * a.d + p0 + 4 * v);
    }
    if (with_e && tid < cnt) S.she[bi * C::CH + tid] = ev[s0 + tid];
    cp_async_commit();
}

// Statistics sum_s h_{s,pi} h_{s,pi}^T of interactions [lo, hi), summed in
// group order into the lower triangle of S.M.
template <int B>
__device__ __forceinline__ void fold_hessian(const FoldArgs &a, const FoldSmem<B> &S, const int32_t *items,
                                             int lo, int hi, int p0, int ti, int tj, int grp, int kstart) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int n = hi - lo, nch = (n + C::CH - 1) / C::CH;
    if (nch > 0) fold_stage<B>(a, S, items, nullptr, lo, hi, 0, p0, 0, false);
    for (int ch = 0; ch < nch; ++ch) {
        cp_async_wait_all();
        __syncthreads();
        if (ch + 1 < nch) fold_stage<B>(a, S, items, nullptr, lo, hi, ch + 1, p0, (ch + 1) & 1, false);
        const int cnt = min(C::CH, n - ch * C::CH);
        const float *bp = S.buf0 + (ch & 1) * C::BUF;
        for (int kk = kstart; kk < cnt; kk += C::NG) {
            float xa[8], xb[8];
            load_seg<8>(bp + kk * C::SB + 8 * ti, xa);
            load_seg<8>(bp + kk * C::SB + 8 * tj, xb);
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
            for (int i = 0; i < 8; ++i) store_tile<8>(S.M + (8 * ti + i) * C::SB + 8 * tj, acc[i], ph > 0);
        }
        __syncthreads();
    }
    if (nch == 0) {  // no interactions: the statistics are zero
        for (int e = tid; e < B * B; e += nt) S.M[(e / B) * C::SB + (e % B)] = 0.f;
        __syncthreads();
    }
}

// Dense terms, Cholesky of S.M and the factor (rows of L, then 1 / L_kk) to Lk.
template <int B>
__device__ __forceinline__ void fold_factor(const FoldArgs &a, const FoldSmem<B> &S, int p0, float lam, float *Lk) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < B * B; e += nt) {
        const int i = e / B, j = e % B;
        if (j > i) continue;
        float v = S.M[i * C::SB + j] + a.alpha0 * a.G[(int64_t)(p0 + i) * a.d + p0 + j];
        if (i == j) {
            v += lam;
            S.diag0[i] = v;
        }
        S.M[i * C::SB + j] = v;
    }
    for (int j = tid; j < B; j += nt) S.M[B * C::SB + j] = 0.f;
    __syncthreads();
    cta_chol16<B, C::SB>(S.M, S.invd, S.diag0, &S.flag[1], 1e-5f);
    for (int e = tid; e < B * B; e += nt) Lk[e] = S.M[(e / B) * C::SB + (e % B)];
    for (int j = tid; j < B; j += nt) Lk[B * B + j] = S.invd[j];
    __syncthreads();
}

// Partial gradient sum_s e_s h_{s,pi} over interactions [lo, hi) into S.xv (B floats).
template <int B>
__device__ __forceinline__ void fold_gradient(const FoldArgs &a, const FoldSmem<B> &S, const int32_t *items,
                                              const float *ev, int lo, int hi, int p0) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int gsz = nt / B < 8 ? nt / B : 8;  // gradient groups (gp holds 8 partial rows)
    const int gj = tid % B, gg = tid / B;
    const int n = hi - lo, nch = (n + C::CH - 1) / C::CH;
    float t = 0.f;
    if (nch > 0) fold_stage<B>(a, S, items, ev, lo, hi, 0, p0, 0, true);
    for (int ch = 0; ch < nch; ++ch) {
        const int bi = ch & 1;
        cp_async_wait_all();
        __syncthreads();
        if (ch + 1 < nch) fold_stage<B>(a, S, items, ev, lo, hi, ch + 1, p0, bi ^ 1, true);
        const int cnt = min(C::CH, n - ch * C::CH);
        const float *bp = S.buf0 + bi * C::BUF;
        if (gg < gsz)
            for (int kk = gg; kk < cnt; kk += gsz) t += S.she[bi * C::CH + kk] * bp[kk * C::SB + gj];
    }
    if (gg < gsz) S.gp[gg * B + gj] = t;
    __syncthreads();
    for (int q = tid; q < B; q += nt) {
        float v = 0.f;
        for (int g2 = 0; g2 < gsz; ++g2) v += S.gp[g2 * B + q];
        S.xv[q] = v;
    }
    __syncthreads();
}

// g = alpha0 u_pi + lambda w_pi + partial (in S.xv), the solve with the kept factor
// Lk, apply w_pi -= delta and u -= delta^T G^I[pi, :].  Leaves delta in S.xv.
template <int B>
__device__ __forceinline__ void fold_solve(const FoldArgs &a, const FoldSmem<B> &S, int p0, float lam,
                                           const float *Lk) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x, d = a.d;
    for (int e = tid; e < B * B; e += nt) S.M[(e / B) * C::SB + (e % B)] = Lk[e];
    for (int q = tid; q < B; q += nt) {
        S.invd[q] = Lk[B * B + q];
        S.xv[q] += a.alpha0 * S.uv[p0 + q] + lam * S.wv[p0 + q];
    }
    __syncthreads();
    cta_forward16<B, C::SB>(S.M, S.invd, S.xv);
    cta_backsolve16<B, C::SB>(S.M, S.invd, S.xv);
    for (int q = tid; q < B; q += nt) S.wv[p0 + q] -= S.xv[q];
    for (int q = tid; q < d; q += nt) {  // coalesced over the columns of G^I
        float v = 0.f;
#pragma unroll 8
        for (int m = 0; m < B; ++m) v += S.xv[m] * a.G[(int64_t)(p0 + m) * d + q];
        S.uv[q] -= v;
    }
    __syncthreads();
}

// Residuals e_s -= <delta, h_{s,pi}> of interactions [lo, hi) (delta in dl):
// one warp per staged interaction.
template <int B>
__device__ __forceinline__ void fold_residual(const FoldArgs &a, const FoldSmem<B> &S, const int32_t *items,
                                              float *ev, int lo, int hi, int p0, const float *dl) {
    using C = FoldCfg<B>;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int n = hi - lo, nch = (n + C::CH - 1) / C::CH;
    if (nch > 0) fold_stage<B>(a, S, items, nullptr, lo, hi, 0, p0, 0, false);
    for (int ch = 0; ch < nch; ++ch) {
        const int bi = ch & 1;
        cp_async_wait_all();
        __syncthreads();
        if (ch + 1 < nch) fold_stage<B>(a, S, items, nullptr, lo, hi, ch + 1, p0, bi ^ 1, false);
        const int cnt = min(C::CH, n - ch * C::CH);
        const float *bp = S.buf0 + bi * C::BUF;
        for (int kk = warp; kk < cnt; kk += nw) {
            float v = 0.f;
            for (int q = lane; q < B; q += 32) v += dl[q] * bp[kk * C::SB + q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0) ev[lo + ch * C::CH + kk] -= v;
        }
    }
    __syncthreads();
}

// The finished request r: embedding and status to mapped host memory, then its flag.
__device__ __forceinline__ void fold_publish(const FoldArgs &a, int r, const float *wv, int status) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < a.d; j += nt) a.w_host[(int64_t)r * a.d + j] = wv[j];
    __syncthreads();
    if (tid == 0) {
        a.status[r] = status;
        __threadfence_system();
        *reinterpret_cast<volatile int32_t *>(a.done_host + r) = 1 + status;
    }
}

// One CTA per short request (the requests a.list[0 .. n_list)).
template <int B>
__global__ void __launch_bounds__(256) k_foldin(FoldArgs a) {
    using C = FoldCfg<B>;
    extern __shared__ float4 smem4[];
    const FoldSmem<B> S(reinterpret_cast<float *>(smem4), a.d);
    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = a.d, nb = d / B;
    const bool active = tid < C::ACTIVE;
    const int grp = active ? tid / C::NTL : C::NG;
    const int kstart = active ? grp : C::CH;
    int ti = 0, tj = 0;
    tri_index(tid % C::NTL, ti, tj);
    for (int li = blockIdx.x; li < a.n_list; li += gridDim.x) {
        const int r = a.list[li];
        const FoldReq rq = a.req[r];
        const int n = rq.n;
        uint8_t *base = a.arena + rq.off;
        const int32_t *items = reinterpret_cast<const int32_t *>(base);
        const float *yv = reinterpret_cast<const float *>(base + rq.y_off);
        float *ev = reinterpret_cast<float *>(base + rq.e_off);
        float *Lg = reinterpret_cast<float *>(base + rq.l_off);  // nb x (B*B + B): L rows, then 1/L_kk
        const float lam = a.lambda * (1.0f + a.nu * (float)n);
        for (int s = tid; s < n; s += nt) ev[s] = rq.has_y ? -yv[s] : -1.0f;
        for (int j = tid; j < d; j += nt) S.wv[j] = S.uv[j] = 0.f;
        if (tid == 0) S.flag[1] = 0;
        __syncthreads();
        for (int k = 0; k < nb; ++k) {
            fold_hessian<B>(a, S, items, 0, n, k * B, ti, tj, grp, kstart);
            fold_factor<B>(a, S, k * B, lam, Lg + (int64_t)k * (B * B + B));
        }
        for (int sw = 0; sw < a.sweeps && !S.flag[1]; ++sw) {
            for (int k = 0; k < nb; ++k) {
                fold_gradient<B>(a, S, items, ev, 0, n, k * B);
                fold_solve<B>(a, S, k * B, lam, Lg + (int64_t)k * (B * B + B));
                fold_residual<B>(a, S, items, ev, 0, n, k * B, S.xv);
            }
        }
        fold_publish(a, r, S.wv, S.flag[1] ? 4 : 0);
        __syncthreads();
    }
}

// One cluster of kFoldCluster CTAs per long request (a.list[cluster index]).
// CTA `rank` owns the interactions [rank n / K, (rank + 1) n / K).  Partial
// Hessians and gradients are summed by CTA 0 in rank order (distributed shared
// memory); CTA 0 factorises, solves, keeps w and u, and writes delta (and the
// failure flag) into every CTA's shared memory before the next barrier.
template <int B>
__global__ void __cluster_dims__(kFoldCluster, 1, 1) __launch_bounds__(256) k_foldin_cl(FoldArgs a) {
    using C = FoldCfg<B>;
    constexpr int K = kFoldCluster;
    extern __shared__ float4 smem4[];
    const FoldSmem<B> S(reinterpret_cast<float *>(smem4), a.d);
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int tid = threadIdx.x, nt = blockDim.x;
    const int d = a.d, nb = d / B;
    const bool active = tid < C::ACTIVE;
    const int grp = active ? tid / C::NTL : C::NG;
    const int kstart = active ? grp : C::CH;
    int ti = 0, tj = 0;
    tri_index(tid % C::NTL, ti, tj);
    const int r = a.list[blockIdx.x / K];
    const FoldReq rq = a.req[r];
    const int n = rq.n;
    const int lo = (int)((int64_t)n * rank / K), hi = (int)((int64_t)n * (rank + 1) / K);
    uint8_t *base = a.arena + rq.off;
    const int32_t *items = reinterpret_cast<const int32_t *>(base);
    const float *yv = reinterpret_cast<const float *>(base + rq.y_off);
    float *ev = reinterpret_cast<float *>(base + rq.e_off);
    float *Lg = reinterpret_cast<float *>(base + rq.l_off);
    const float lam = a.lambda * (1.0f + a.nu * (float)n);
    for (int s = lo + tid; s < hi; s += nt) ev[s] = rq.has_y ? -yv[s] : -1.0f;
    for (int j = tid; j < d; j += nt) S.wv[j] = S.uv[j] = 0.f;
    if (tid == 0) S.flag[1] = 0;
    __syncthreads();
    for (int k = 0; k < nb; ++k) {
        fold_hessian<B>(a, S, items, lo, hi, k * B, ti, tj, grp, kstart);
        cl.sync();  // every share's partial Hessian is in its CTA's M
        if (rank == 0) {
            for (int e = tid; e < B * B; e += nt) {
                const int i = e / B, j = e % B;
                if (j > i) continue;
                float v = S.M[i * C::SB + j];
                for (int q = 1; q < K; ++q) v += cl.map_shared_rank(S.M, q)[i * C::SB + j];
                S.M[i * C::SB + j] = v;
            }
        }
        cl.sync();  // the partials have been read; the other CTAs may overwrite their M
        if (rank == 0) fold_factor<B>(a, S, k * B, lam, Lg + (int64_t)k * (B * B + B));
    }
    if (rank == 0 && tid == 0)  // the factor's verdict to every CTA
        for (int q = 1; q < K; ++q) cl.map_shared_rank(S.flag, q)[1] = S.flag[1];
    cl.sync();
    for (int sw = 0; sw < a.sweeps && !S.flag[1]; ++sw) {
        for (int k = 0; k < nb; ++k) {
            fold_gradient<B>(a, S, items, ev, lo, hi, k * B);
            cl.sync();  // every share's partial gradient is in its CTA's xv
            if (rank == 0) {
                for (int q0 = tid; q0 < B; q0 += nt) {
                    float v = S.xv[q0];
                    for (int q = 1; q < K; ++q) v += cl.map_shared_rank(S.xv, q)[q0];
                    S.gp[q0] = v;
                }
                __syncthreads();
                for (int q0 = tid; q0 < B; q0 += nt) S.xv[q0] = S.gp[q0];
                __syncthreads();
                fold_solve<B>(a, S, k * B, lam, Lg + (int64_t)k * (B * B + B));
                for (int q0 = tid; q0 < B; q0 += nt)  // delta to every CTA
                    for (int q = 1; q < K; ++q) cl.map_shared_rank(S.xv, q)[q0] = S.xv[q0];
            }
            cl.sync();  // delta is in every CTA's xv
            fold_residual<B>(a, S, items, ev, lo, hi, k * B, S.xv);
        }
    }
    if (rank == 0) fold_publish(a, r, S.wv, S.flag[1] ? 4 : 0);
}

template <int B>
int foldin_smem(int d) {
    return (FoldCfg<B>::FIXED_FLOATS + 2 * d) * 4 + 16;
}

template <int B>
cudaError_t launch_foldin_b(const FoldArgs &a, bool cluster, cudaStream_t s) {
    const int sm = foldin_smem<B>(a.d);
    if (cluster) {
        cudaError_t e = cudaFuncSetAttribute(k_foldin_cl<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_foldin_cl<B><<<a.n_list * kFoldCluster, 256, sm, s>>>(a);
    } else {
        cudaError_t e = cudaFuncSetAttribute(k_foldin<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        if (e != cudaSuccess) return e;
        k_foldin<B><<<a.n_list, 256, sm, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_foldin(const FoldArgs &a, bool cluster, cudaStream_t s) {
    if (a.n_list <= 0) return cudaSuccess;
    switch (a.b) {
        case 16: return launch_foldin_b<16>(a, cluster, s);
        case 32: return launch_foldin_b<32>(a, cluster, s);
        case 64: return launch_foldin_b<64>(a, cluster, s);
        case 128: return launch_foldin_b<128>(a, cluster, s);
        default: return cudaErrorInvalidValue;
    }
}

int64_t foldin_factor_floats(int32_t d, int32_t b) { return (int64_t)(d / b) * (b * b + b); }

}  // namespace ials
