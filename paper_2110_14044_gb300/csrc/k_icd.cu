// iCD (Algorithm 2; Eqs. 5-7): the b = 1 end point of the block step, as its
// own pass per coordinate instead of the general path's per-block Gramian,
// row-term, statistics and solve kernels.
//
// For coordinate f, a pass over the rows of one side (users, then items) needs
// the column g = G^F[:, f] = sum_j f_j f_{j,f} of the fixed side's Gramian and
// computes, per row r (Eq. 6),
//   num = alpha0 <x_r, g> + lambda_r x_{r,f} + sum_{s in S_r} alpha_s e_s f_{c_s,f}
//   den = alpha0 g_f + lambda_r + sum_{s in S_r} alpha_s f_{c_s,f}^2
//   delta = num / den,  x_{r,f} -= delta,  e_s -= delta f_{c_s,f}   (Eqs. 5, 7)
// The Gramian column the next pass needs (the updated side's column f for the
// item pass; H's column f + 1 for the next user pass) is a sum over the rows
// this pass updates, so each pass forms it on the way: every warp adds
// x'_{r,fn} x'_r for its rows, the blocks' partials are summed in a fixed
// order by the last block to finish.  Rows are assigned to warps statically
// (task t to warp t mod #warps over the length-sorted task list), so the sums
// do not depend on timing.  Long rows are cut into chunks (as in the general
// path): the row kernel stores each chunk's two partial sums; a split kernel
// sums them in chunk order, solves and applies; a residual kernel updates the
// residuals of the long rows' pieces.
//
// Residuals: each side keeps its own copy of the residual cache in its own CSR
// order (users: user-major, items: item-major), so every pass reads and writes
// its residuals contiguously instead of through the position map.  A pass
// changes one coordinate per row, so its effect on the other side's copy is
// one scalar per row: the item pass at f lowers e(u,i) by delta_i w_{u,f}, and
// the next user pass applies that on the fly as it reads its copy,
// e(u,i) - delta_i^{prev} w_{u,f} (and the item pass applies the user pass's
// delta_u h_{i,f} likewise).  Each copy is thus exact whenever its side reads
// it; the user-major cache is rebuilt before anything else reads it.
//
// Layout: the pass reads f_{c,f} from a transposed copy of the fixed side
// (d x n, column f contiguous), which the epoch forms once and every pass keeps
// current by writing x_{r,f} into the updated side's transposed copy as well.
// The coordinate column of H (80 KB at 20,000 items) then stays in L1, and a
// gathered 32-byte sector carries eight useful values instead of one.
#include "ials_internal.cuh"

#include <algorithm>

namespace ials {

namespace {

// warps per block of the row and split kernels: one block per SM; fewer warps
// when d is large (each warp keeps a d-float partial column in shared memory)
__host__ __device__ constexpr int icd_warps(int d) { return d <= 1024 ? 32 : 8; }
constexpr int kIcdMaxWarps = 32;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// <x_r, g> with g in shared memory; x_r row-major (d % 4 == 0).  Warp-uniform result.
__device__ __forceinline__ float row_dot(const float *__restrict__ x, const float *g, int d, int lane) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    const float4 *g4 = reinterpret_cast<const float4 *>(g);
    float acc = 0.f;
    for (int v = lane; v < (d >> 2); v += 32) {
        const float4 a = x4[v], b = g4[v];
        acc = fmaf(a.x, b.x, acc);
        acc = fmaf(a.y, b.y, acc);
        acc = fmaf(a.z, b.z, acc);
        acc = fmaf(a.w, b.w, acc);
    }
    return warp_sum(acc);
}

// part[k] += coef * x'_k for the updated row (x'_f = xf_new), lanes over float4 chunks.
__device__ __forceinline__ void add_row(float *part, const float *__restrict__ x, int d, int f, float xf_new,
                                        float coef, int lane) {
    const float4 *x4 = reinterpret_cast<const float4 *>(x);
    float4 *p4 = reinterpret_cast<float4 *>(part);
    for (int v = lane; v < (d >> 2); v += 32) {
        float4 a = x4[v];
        if ((f >> 2) == v) {
            const int q = f & 3;
            if (q == 0) a.x = xf_new;
            else if (q == 1) a.y = xf_new;
            else if (q == 2) a.z = xf_new;
            else a.w = xf_new;
        }
        float4 p = p4[v];
        p.x = fmaf(coef, a.x, p.x);
        p.y = fmaf(coef, a.y, p.y);
        p.z = fmaf(coef, a.z, p.z);
        p.w = fmaf(coef, a.w, p.w);
        p4[v] = p;
    }
}

// The last block to finish sums the npart partial columns (fixed order) into
// g_out and resets the counter.  Called by every thread of every block after
// its partial is written.
__device__ __forceinline__ void last_block_reduce(const IcdArgs &a, int npart) {
    __shared__ int last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(a.done, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // every thread sums a contiguous range of partials for one entry (so the
    // loads are independent and in flight together); the ranges' sums are then
    // added in range order, which fixes the summation order
    extern __shared__ float4 smem4[];
    float *red = reinterpret_cast<float *>(smem4);  // reuses the kernel's shared memory
    const int d = a.s.d, nt = blockDim.x;
    const int per_k = nt >= d ? nt / d : 1;           // threads per entry
    const int span = (npart + per_k - 1) / per_k;
    __syncthreads();
    for (int k0 = 0; k0 < d; k0 += nt / per_k) {
        const int k = k0 + threadIdx.x / per_k, h = threadIdx.x % per_k;
        float t = 0.f;
        if (k < d && threadIdx.x < per_k * (nt / per_k)) {
            const int p0 = h * span, p1 = min(npart, p0 + span);
            for (int p = p0; p < p1; ++p) t += __ldcg(a.gpart + (int64_t)p * d + k);
        }
        red[threadIdx.x] = t;
        __syncthreads();
        if (h == 0 && k < d && threadIdx.x < per_k * (nt / per_k)) {
            float u = 0.f;
            for (int q = 0; q < per_k; ++q) u += red[threadIdx.x + q];
            a.g_out[k] = u;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *a.done = 0;
}

// Per task: the coordinate-f statistics of a row (or of a chunk of a long row,
// stored to its slot), then for whole rows the update, the residual update and
// the Gramian contribution.  Shared: g (d), one partial column per warp (d each).
// Interactions are visited 64 at a time (two per lane) so that the dependent
// loads of two gathers are in flight together.
template <bool HAS_A, bool DPREV>
__global__ void __launch_bounds__(32 * kIcdMaxWarps) k_icd_rows(const IcdArgs a) {
    extern __shared__ float4 smem4[];
    float *g = reinterpret_cast<float *>(smem4);
    const int d = a.s.d, f = a.f, fn = a.fn, nw = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wpart = g + d + warp * d;
    for (int k = threadIdx.x; k < d; k += blockDim.x) g[k] = a.g_in[k];
    for (int k = lane; k < d; k += 32) wpart[k] = 0.f;
    __syncthreads();
    const StepArgs &s = a.s;
    const float *__restrict__ Ff = a.FT + (int64_t)f * a.n_fixed;  // column f of the fixed side
    float *__restrict__ eo = a.eo;
    const float gf = g[f];
    const int nwarps = gridDim.x * nw;
    for (int t = blockIdx.x * nw + warp; t < s.n_tasks; t += nwarps) {
        const Task tk = s.tasks[t];
        float *x = s.X + (int64_t)tk.row * d;
        const float xp = DPREV ? x[a.fprev] : 0.f;  // this row's coordinate the previous pass's deltas multiply
        float num = 0.f, den = 0.f;
        constexpr int KEEP = 2;  // 64-interaction rounds kept in registers for the residual update
        float ek[KEEP][2], fk[KEEP][2];
        for (int j = 0; j * 64 < tk.len; ++j) {
            float fc[2] = {0.f, 0.f}, ev[2] = {0.f, 0.f}, al[2] = {1.f, 1.f}, dp[2] = {0.f, 0.f};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = j * 64 + h * 32 + lane;
                if (i < tk.len) {
                    const int64_t p = tk.begin + i;
                    const int c = s.idx[p];
                    fc[h] = Ff[c];
                    ev[h] = eo[p];
                    if (DPREV) dp[h] = a.dprev[c];
                    if (HAS_A) al[h] = a.alpha_o[p];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (DPREV) ev[h] = fmaf(-dp[h], xp, ev[h]);
                num = fmaf(al[h] * ev[h], fc[h], num);
                den = fmaf(al[h] * fc[h], fc[h], den);
            }
#pragma unroll
            for (int u = 0; u < KEEP; ++u)
                if (u == j) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) { ek[u][h] = ev[h]; fk[u][h] = fc[h]; }
                }
        }
        num = warp_sum(num);
        den = warp_sum(den);
        if (tk.slot >= 0) {  // a chunk of a long row
            if (lane == 0) {
                s.part[2 * tk.slot] = num;
                s.part[2 * tk.slot + 1] = den;
            }
            continue;
        }
        const float lam = s.lambda * (1.0f + s.nu * (float)tk.len);
        const float dot = row_dot(x, g, d, lane);
        const float xf = x[f];
        num += s.alpha0 * dot + lam * xf;
        den += s.alpha0 * gf + lam;
        float delta = 0.f;
        if (den > 0.f && isfinite(num)) {
            delta = num / den;
        } else if (lane == 0) {
            atomicAdd((unsigned long long *)&s.stats[1], 1ull);
        }
        const float xf_new = xf - delta;
        if (fn >= 0) {
            const float coef = fn == f ? xf_new : x[fn];
            add_row(wpart, x, d, f, xf_new, coef, lane);
        }
        __syncwarp();
        if (lane == 0) {
            x[f] = xf_new;
            a.XT[(int64_t)f * s.n_rows + tk.row] = xf_new;
            a.dself[tk.row] = delta;
        }
        for (int j = 0; j * 64 < tk.len; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = j * 64 + h * 32 + lane;
                if (i >= tk.len) continue;
                const int64_t p = tk.begin + i;
                float ev, fc;
                if (j < KEEP) {
                    ev = 0.f;
                    fc = 0.f;
#pragma unroll
                    for (int u = 0; u < KEEP; ++u)
                        if (u == j) { ev = ek[u][h]; fc = fk[u][h]; }
                } else {
                    const int c = s.idx[p];
                    fc = Ff[c];
                    ev = eo[p];
                    if (DPREV) ev = fmaf(-a.dprev[c], xp, ev);
                }
                eo[p] = fmaf(-delta, fc, ev);
            }
        }
    }
    if (fn < 0) return;
    __syncthreads();
    // warp partials in warp order -> this block's partial column
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += g[d + w * d + k];
        a.gpart[(int64_t)blockIdx.x * d + k] = t;
    }
    if (s.n_split == 0) last_block_reduce(a, gridDim.x);
}

// Long rows: one warp per row sums the chunks' partial sums in chunk order,
// forms the dense terms and the update, applies it and records delta; each
// block sums its rows' Gramian contributions in row order into one partial
// column (after the row kernel's), and the last block reduces all partials.
__global__ void __launch_bounds__(32 * kIcdMaxWarps) k_icd_split(const IcdArgs a) {
    extern __shared__ float4 smem4[];
    float *g = reinterpret_cast<float *>(smem4);
    const int d = a.s.d, f = a.f, fn = a.fn, kIcdWarps = blockDim.x >> 5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wpart = g + d + warp * d;
    for (int k = threadIdx.x; k < d; k += blockDim.x) g[k] = a.g_in[k];
    for (int k = lane; k < d; k += 32) wpart[k] = 0.f;
    __syncthreads();
    const StepArgs &s = a.s;
    const int nwarps = gridDim.x * kIcdWarps;
    for (int i = blockIdx.x * kIcdWarps + warp; i < s.n_split; i += nwarps) {
        const SplitRow sr = s.split[i];
        float num = 0.f, den = 0.f;
        for (int k = 0; k < sr.nslots; ++k) {
            num += s.part[2 * (sr.slot0 + k)];
            den += s.part[2 * (sr.slot0 + k) + 1];
        }
        float *x = s.X + (int64_t)sr.row * d;
        const float lam = s.lambda * (1.0f + s.nu * (float)sr.len);
        const float dot = row_dot(x, g, d, lane);
        const float xf = x[f];
        num += s.alpha0 * dot + lam * xf;
        den += s.alpha0 * g[f] + lam;
        float delta = 0.f;
        if (den > 0.f && isfinite(num)) {
            delta = num / den;
        } else if (lane == 0) {
            atomicAdd((unsigned long long *)&s.stats[1], 1ull);
        }
        const float xf_new = xf - delta;
        if (fn >= 0) add_row(wpart, x, d, f, xf_new, fn == f ? xf_new : x[fn], lane);
        __syncwarp();
        if (lane == 0) {
            if (a.dprev) a.xold[i] = x[a.fprev];  // before the update (fprev may be f)
            x[f] = xf_new;
            a.XT[(int64_t)f * s.n_rows + sr.row] = xf_new;
            s.delta[i] = delta;
            a.dself[sr.row] = delta;
        }
    }
    if (fn < 0) return;
    __syncthreads();
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        float t = 0.f;
        for (int w = 0; w < kIcdWarps; ++w) t += g[d + w * d + k];
        a.gpart[(int64_t)(a.grid + blockIdx.x) * d + k] = t;
    }
    last_block_reduce(a, a.grid + gridDim.x);
}

// Residual update of the long rows, one warp per piece of at most 128 interactions.
template <bool DPREV>
__global__ void __launch_bounds__(256) k_icd_split_resid(const IcdArgs a) {
    const StepArgs &s = a.s;
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const float *__restrict__ Ff = a.FT + (int64_t)a.f * a.n_fixed;
    float *__restrict__ eo = a.eo;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < s.n_stasks; t += nwarps) {
        const Task tk = s.stasks[t];
        const float delta = s.delta[tk.srow];
        const float xp = DPREV ? a.xold[tk.srow] : 0.f;
        // a piece holds at most 128 interactions: four per lane, all loads issued first
        float fc[4], ev[4], dp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            if (i < tk.len) {
                const int64_t p = tk.begin + i;
                const int c = s.idx[p];
                fc[u] = Ff[c];
                ev[u] = eo[p];
                dp[u] = DPREV ? a.dprev[c] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = lane + 32 * u;
            if (i < tk.len) {
                const float e = DPREV ? fmaf(-dp[u], xp, ev[u]) : ev[u];
                eo[tk.begin + i] = fmaf(-delta, fc[u], e);
            }
        }
    }
}

// Own-order residual copy of the item side: e_i[t] = e[pos[t]] (gather) and back (scatter).
__global__ void k_perm_gather(const float *__restrict__ src, const int32_t *__restrict__ pos, int64_t n,
                              float *__restrict__ dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[t] = src[pos[t]];
}
__global__ void k_perm_scatter(const float *__restrict__ src, const int32_t *__restrict__ pos, int64_t n,
                               float *__restrict__ dst) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        dst[pos[t]] = src[t];
}

// g and the warps' partial columns: d (1 + warps) floats, at most 4096 x 9
constexpr int kIcdMaxSmem = (int)(sizeof(float) * 4096 * (1 + 8));
static_assert(1024 * (1 + 32) <= 4096 * (1 + 8), "shared-memory bound of the largest d per warp count");

template <bool HAS_A, bool DPREV>
cudaError_t launch_icd_t(const IcdArgs &a0, cudaStream_t st) {
    IcdArgs a = a0;
    const int kIcdWarps = icd_warps(a.s.d);
    // g and the warps' partial columns; at least one float per thread for the final reduction
    const size_t smem = sizeof(float) * std::max<size_t>((size_t)a.s.d * (1 + kIcdWarps), 32 * kIcdWarps);
    prof_mark(a.s.prof, K_SPARSE, st);
    k_icd_rows<HAS_A, DPREV><<<a.grid, 32 * kIcdWarps, smem, st>>>(a);
    prof_mark(a.s.prof, -1, st);
    if (a.s.n_split > 0) {
        prof_mark(a.s.prof, K_SPLIT_SOLVE, st);
        k_icd_split<<<icd_split_grid(a.s.n_split, a.s.d), 32 * kIcdWarps, smem, st>>>(a);
        prof_mark(a.s.prof, K_SPLIT_RESID, st);
        const int g3 = (int)std::min<int64_t>((a.s.n_stasks + 7) / 8, 152 * 8);
        k_icd_split_resid<DPREV><<<g3 > 0 ? g3 : 1, 256, 0, st>>>(a);
        prof_mark(a.s.prof, -1, st);
    }
    return cudaGetLastError();
}

}  // namespace

int32_t icd_row_grid(int32_t n_tasks, int32_t d) {
    // one block per SM, never more blocks than warp-sized task groups need
    int32_t g = 152;
    const int32_t need = (n_tasks + icd_warps(d) - 1) / icd_warps(d);
    if (g > need) g = need;
    return g > 0 ? g : 1;
}

int32_t icd_split_grid(int32_t n_split, int32_t d) {
    int32_t g = (n_split + icd_warps(d) - 1) / icd_warps(d);
    if (g > 38) g = 38;
    return g > 0 ? g : 1;
}

// X (n x d, row-major) -> XT (d x n), 32 x 32 tiles through shared memory.
__global__ void k_transpose(const float *__restrict__ X, int64_t n, int32_t d, float *__restrict__ XT) {
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int64_t r = r0 + i;
        const int c = c0 + threadIdx.x;
        if (r < n && c < d) tile[i][threadIdx.x] = X[r * d + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i;
        const int64_t r = r0 + threadIdx.x;
        if (r < n && c < d) XT[(int64_t)c * n + r] = tile[threadIdx.x][i];
    }
}

cudaError_t launch_transpose(const float *X, int64_t n, int32_t d, float *XT, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((d + 31) / 32));
    k_transpose<<<grid, dim3(32, 8), 0, s>>>(X, n, d, XT);
    return cudaGetLastError();
}

cudaError_t icd_prepare() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaSuccess) return done;
    cudaError_t e = cudaSuccess;
    const auto set = [&](const void *k) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kIcdMaxSmem);
    };
    set((const void *)k_icd_rows<false, false>);
    set((const void *)k_icd_rows<false, true>);
    set((const void *)k_icd_rows<true, false>);
    set((const void *)k_icd_rows<true, true>);
    set((const void *)k_icd_split);
    done = e;
    return e;
}

cudaError_t launch_icd(const IcdArgs &a, cudaStream_t s) {
    const bool dp = a.dprev != nullptr, wa = a.alpha_o != nullptr;
    if (dp) return wa ? launch_icd_t<true, true>(a, s) : launch_icd_t<false, true>(a, s);
    return wa ? launch_icd_t<true, false>(a, s) : launch_icd_t<false, false>(a, s);
}

cudaError_t launch_perm_gather(const float *src, const int32_t *pos, int64_t n, float *dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_perm_gather<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(src, pos, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_perm_scatter(const float *src, const int32_t *pos, int64_t n, float *dst, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_perm_scatter<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(src, pos, n, dst);
    return cudaGetLastError();
}

}  // namespace ials
