// Sparse block step of Algorithm 3 for block sizes B <= 32 (one warp per task).
//
// For a row r of the side being updated (fixed side F, block pi = [p0, p0+B)):
//   g_r  = R_r + sum_{s in S_r} alpha_s e_s f_{c_s, pi}                 (Eq. 11)
//   A_r  = sum_{s in S_r} alpha_s f_{c_s,pi} f_{c_s,pi}^T
//          + alpha0 G_pipi + lambda_r I                                 (Eq. 12)
//   delta = A_r^{-1} g_r ;  x_{r,pi} -= delta ;  e_s -= <delta, f_{c_s,pi}>  (Eq. 9, Eq. 7 generalised)
// where R_r = alpha0 x_r G^{pi} + lambda_r x_{r,pi} comes from the row-term kernel
// and e = yhat - y is the residual cache in user-major order (items reach it
// through the CSR-position map `pos`).
//
// Warp layout: lane l owns column col = l % B of A_r (and entry col of g_r);
// the 32 / B sub-groups of B lanes accumulate interleaved interactions and
// are summed by a fixed xor butterfly at the end, so results do not depend on
// scheduling.  Interactions are staged 32 at a time: their fixed-side slices
// f_{c,pi} are gathered with 16-byte loads into a padded shared-memory tile
// (row stride B + 4 floats) and then read back as broadcasts.
//
// Long rows are cut into several tasks that write partial (A, g) to a slot;
// k_split_solve sums the slots of a row in slot order and solves it, and
// k_split_resid applies its residual update.  A row whose FP32 solve meets a
// non-positive (or collapsed) pivot is queued; k_retry re-solves it in FP64
// from scratch.
#pragma once

#include "ials_internal.cuh"
#include "k_split_resid_scan.cuh"

namespace ials {

template <int B>
struct SparseCfg {
    static constexpr int G = 32 / B;               // sub-groups per warp
    static constexpr int SB = B < 4 ? 4 : B + 4;   // shared row stride (floats)
    static constexpr int CH = 32;                  // interactions staged per chunk
    static constexpr int VPAD = (B + 3) / 4 * 4;
    static constexpr int CB = B % 4 == 0 ? B + 4 : B + 1;  // solver column buffer (B entries + g_k)
    static constexpr int LREG = 4 * CB;                     // two steps x two column buffers
    static constexpr int WARP_FLOATS_RAW = CH * SB + 3 * CH + VPAD + LREG;
    static constexpr int WARP_FLOATS = (WARP_FLOATS_RAW + 3) / 4 * 4;
    static constexpr int GPP_FLOATS = (B * B + 3) / 4 * 4;
    static constexpr int WARPS = 8;
    static constexpr int SMEM_BYTES = (GPP_FLOATS + WARPS * WARP_FLOATS) * 4;
};

struct WarpSmem {
    float *h;    // CH x SB fixed-side slices
    float *e;    // CH (alpha * e when weighted)
    float *a;    // CH alpha
    int *c;      // CH column ids
    float *v;    // VPAD vector buffer (delta)
    float *L;    // solver column buffers (2 x CB floats, 16-byte aligned)
};

template <int B>
__device__ __forceinline__ WarpSmem warp_smem(float *base, int warp) {
    using C = SparseCfg<B>;
    WarpSmem w;
    float *p = base + C::GPP_FLOATS + warp * C::WARP_FLOATS;
    w.h = p;
    w.e = w.h + C::CH * C::SB;
    w.a = w.e + C::CH;
    w.c = reinterpret_cast<int *>(w.a + C::CH);
    w.v = reinterpret_cast<float *>(w.c + C::CH);
    w.L = w.v + C::VPAD;
    return w;
}

// Stage `cnt` (<= 32) interactions starting at CSR position `begin`: column
// ids, residual (weighted) and the gathered slices.  Lane k keeps the residual
// index of interaction k in q.  LOAD_E = false skips residual / weight loads.
template <int B, bool PERM, bool HAS_A, bool LOAD_E>
__device__ __forceinline__ void stage_chunk(const StepArgs &a, int64_t begin, int cnt, int lane,
                                            const WarpSmem &w, int64_t &q) {
    using C = SparseCfg<B>;
    __syncwarp();
    if (lane < cnt) {
        const int64_t s = begin + lane;
        w.c[lane] = a.idx[s];
        q = PERM ? (int64_t)a.pos[s] : s;
        if (LOAD_E) {
            const float r = a.e[q];
            if (HAS_A) {
                const float al = a.alpha[q];
                w.e[lane] = al * r;
                w.a[lane] = al;
            } else {
                w.e[lane] = r;
            }
        }
    }
    __syncwarp();
    if constexpr (B >= 4) {
        constexpr int VPR = B / 4;        // float4 per slice
        constexpr int RPP = 32 / VPR;     // slices per pass
        constexpr int NP = C::CH / RPP;   // passes
        const int v = lane % VPR, rr = lane / VPR;
        float4 t[NP];
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int k = p * RPP + rr;
            if (k < cnt) {
                const float4 *src = reinterpret_cast<const float4 *>(
                    a.F + (int64_t)w.c[k] * a.d + a.p0);
                t[p] = __ldg(src + v);
            }
        }
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            const int k = p * RPP + rr;
            if (k < cnt) reinterpret_cast<float4 *>(w.h + k * C::SB)[v] = t[p];
        }
    } else {
        if (lane < cnt) {
            const float *src = a.F + (int64_t)w.c[lane] * a.d + a.p0;
#pragma unroll
            for (int j = 0; j < B; ++j) w.h[lane * C::SB + j] = __ldg(src + j);
        }
    }
    __syncwarp();
}

// Packed FP32 pairs (fma / mul .rn.f32x2, sm_100 and later): two independent
// FP32 operations, each rounded exactly as its scalar form, issued as one
// instruction.  fma2: d = a * b + d; mul2: d = d * a.
__device__ __forceinline__ void fma2(float &d0, float &d1, float a0, float a1, float b0, float b1) {
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rd, {%0, %1};\n\t"
        "fma.rn.f32x2 rd, ra, rb, rd;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void mul2(float &d0, float &d1, float a0, float a1) {
    asm("{\n\t.reg .b64 ra, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rd, {%0, %1};\n\t"
        "mul.rn.f32x2 rd, rd, ra;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a0), "f"(a1));
}

// Approximate reciprocal (rcp.approx: at most 1 ulp from 1/x).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Newton solve A delta = g of one row in one warp: Gauss-Jordan elimination
// without pivoting, which is sound for a symmetric positive definite A (its
// pivots are the diagonal of D in A = L D L^T, i.e. the successive Schur
// complements).  Lane l holds the whole row col = l % B of A (both triangles)
// in A[] and entry col of g.  Step k: each lane publishes its column-k entry in
// a double-buffered shared column (lane k also publishes g_k); every lane but
// k then eliminates column k from its row and from g,
//   s = A[col][k] / d_k,  A[col][j] -= s A[k][j] (j > k),  g_col -= s g_k,
// where A[k][j] = A[j][k] is read from the published column (the trailing
// block stays symmetric).  After B steps the system is diagonal and
// delta_col = g_col / d_col.  Compared with Cholesky plus two substitutions
// this has the same trailing-update work per lane (every lane runs every j
// anyway) and a shorter dependent chain per step (store, warp barrier,
// broadcast load, reciprocal), and no substitution passes.  Lane k checks its
// own pivot (positive, finite, not below 1e-5 of its original diagonal, i.e.
// no more than ~17 bits lost); one vote at the end decides for the warp.
// Returns false (warp-uniform) on a bad pivot or a non-finite solution; on
// success `delta` holds entry col of the solution.
// Gauss-Jordan as above with 2 x 2 pivot blocks (B even): step m eliminates the
// columns k = 2m and k + 1 at once.  Lanes publish both column entries (lanes k
// and k + 1 also g_k, g_{k+1}); the pivot block P = [[a, b], [b, c]] is SPD (a
// principal Schur complement), and every other lane eliminates with
//   [s1, s2] = [A[col][k], A[col][k+1]] P^{-1},
//   A[col][j] -= s1 A[k][j] + s2 A[k+1][j] (j > k + 1),  g_col -= s1 g_k + s2 g_{k+1}.
// At the end the system is block diagonal; each pivot pair solves its 2 x 2
// block (the partner's g by a shuffle).  The pivots checked are those of
// A = L D L^T: d_k = a and d_{k+1} = c - b^2 / a.  Half as many dependent steps
// as the scalar version for the same multiply-adds.
template <int B>
__device__ __forceinline__ bool gj_solve2(float (&A)[B], float g, int col, int sub, const WarpSmem &w,
                                          bool force_fail, float &delta) {
    static_assert(B % 4 == 0, "pairs of columns, 16-byte loads");
    constexpr int CB = SparseCfg<B>::CB;
    float diag0 = 0.f;
#pragma unroll
    for (int j = 0; j < B; ++j)
        if (j == col) diag0 = A[j];
    bool bad = force_fail;
    float pa = 1.f, pb = 0.f, pc = 1.f;  // this lane's pivot block
#pragma unroll
    for (int k = 0; k < B; k += 2) {
        float *v1 = w.L + ((k >> 1) & 1) * 2 * CB, *v2 = v1 + CB;
        if (sub == 0) {
            v1[col] = A[k];
            v2[col] = A[k + 1];
            if (col == k) v1[B] = g;
            if (col == k + 1) v2[B] = g;
        }
        __syncwarp();
        const float a = v1[k], b = v1[k + 1], c = v2[k + 1];
        const float g1 = v1[B], g2 = v2[B];
        const float rdet = rcp_approx(a * c - b * b);
        const bool piv = col == k || col == k + 1;
        const float x = A[k], y = A[k + 1];
        const float s1 = piv ? 0.f : (x * c - y * b) * rdet;
        const float s2 = piv ? 0.f : (y * a - x * b) * rdet;
        if (col == k) bad = bad || !(a > 1e-5f * diag0) || !(a <= 3.0e38f);
        if (col == k + 1) {
            const float d1 = c - b * b * rcp_approx(a);
            bad = bad || !(d1 > 1e-5f * diag0) || !(d1 <= 3.0e38f);
        }
        if (piv) {
            pa = a;
            pb = b;
            pc = c;
        }
#pragma unroll
        for (int j0 = (k + 2) & ~3; j0 < B; j0 += 4) {
            // k is even, so the entries j > k + 1 start at a pair boundary
            const float4 q1 = *reinterpret_cast<const float4 *>(v1 + j0);
            const float4 q2 = *reinterpret_cast<const float4 *>(v2 + j0);
            if (j0 > k + 1) {
                fma2(A[j0], A[j0 + 1], -s1, -s1, q1.x, q1.y);
                fma2(A[j0], A[j0 + 1], -s2, -s2, q2.x, q2.y);
            }
            fma2(A[j0 + 2], A[j0 + 3], -s1, -s1, q1.z, q1.w);
            fma2(A[j0 + 2], A[j0 + 3], -s2, -s2, q2.z, q2.w);
        }
        g -= s1 * g1 + s2 * g2;
    }
    if (__any_sync(kFull, bad)) return false;
    // 2 x 2 block solve: lane col pairs with col ^ 1 (same sub-group lanes)
    const float gp = __shfl_xor_sync(kFull, g, 1);
    const float rd = rcp_approx(pa * pc - pb * pb);
    delta = (col & 1) ? (pa * g - pb * gp) * rd : (pc * g - pb * gp) * rd;
    return __all_sync(kFull, isfinite(delta));
}

template <int B>
__device__ __forceinline__ bool chol_solve(float (&A)[B], float g, int col, int sub,
                                           const WarpSmem &w, bool force_fail, float &delta) {
    constexpr int CB = SparseCfg<B>::CB;  // column buffer: B entries, then g_k
    float diag0 = 0.f;
#pragma unroll
    for (int j = 0; j < B; ++j)
        if (j == col) diag0 = A[j];
    bool bad = force_fail;
    float dmine = 1.f;
    float *cb = w.L;
#pragma unroll
    for (int k = 0; k < B; ++k) {
        float *v = cb + (k & 1) * CB;
        if (sub == 0) {
            v[col] = A[k];
            if (col == k) v[B] = g;
        }
        __syncwarp();
        const float dk = v[k];
        const float gk = v[B];
        const float s = col == k ? 0.f : A[k] * rcp_approx(dk);
        if (col == k) {
            bad = bad || !(dk > 1e-5f * diag0) || !(dk <= 3.0e38f);
            dmine = dk;
        }
        if constexpr (B % 4 == 0) {  // 16-byte broadcasts of column k (v is 16-byte aligned)
#pragma unroll
            for (int j0 = (k + 1) & ~3; j0 < B; j0 += 4) {
                const float4 q = *reinterpret_cast<const float4 *>(v + j0);
                if (j0 > k) A[j0] -= s * q.x;
                if (j0 + 1 > k) A[j0 + 1] -= s * q.y;
                if (j0 + 2 > k) A[j0 + 2] -= s * q.z;
                A[j0 + 3] -= s * q.w;
            }
        } else {
#pragma unroll
            for (int j = k + 1; j < B; ++j) A[j] -= s * v[j];
        }
        g -= s * gk;
    }
    if (__any_sync(kFull, bad)) return false;
    delta = g / dmine;
    return __all_sync(kFull, isfinite(delta));
}

template <int B>
__device__ __forceinline__ float dot_slice(const float *v, const float *h) {
    float t = 0.f;
    if constexpr (B >= 4) {
#pragma unroll
        for (int j = 0; j < B; j += 4) {
            const float4 a = *reinterpret_cast<const float4 *>(v + j);
            const float4 b = *reinterpret_cast<const float4 *>(h + j);
            t += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < B; ++j) t += v[j] * h[j];
    }
    return t;
}

__device__ __forceinline__ void queue_retry(const StepArgs &a, int lane, int row) {
    if (lane == 0) {
        const int i = atomicAdd(a.retry, 1);
        a.retry[1 + i] = row;
    }
}

// ------------------------------------------------------------- main kernel
template <int B, bool PERM, bool HAS_A>
__global__ void __launch_bounds__(256, 2) k_sparse(const StepArgs a) {
    using C = SparseCfg<B>;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sGpp = smem;
    // alpha0 G_pipi, exactly symmetric (taken from its lower triangle: the solver
    // treats the trailing block as symmetric); lane col reads column col, which
    // is free of bank conflicts
    for (int i = threadIdx.x; i < B * B; i += blockDim.x)
        sGpp[i] = a.alpha0 * a.G[(int64_t)(a.p0 + max(i / B, i % B)) * B + min(i / B, i % B)];
    __syncthreads();
    const WarpSmem w = warp_smem<B>(smem, warp);
    const int col = lane % B, sub = lane / B;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.n_tasks) break;
        const Task tk = a.tasks[t];
        float acc[B];
#pragma unroll
        for (int j = 0; j < B; ++j) acc[j] = 0.f;
        float g = 0.f;
        int64_t q = 0;
        for (int c0 = 0; c0 < tk.len; c0 += C::CH) {
            const int cnt = min(C::CH, tk.len - c0);
            stage_chunk<B, PERM, HAS_A, true>(a, tk.begin + c0, cnt, lane, w, q);
            for (int k = sub; k < cnt; k += C::G) {
                const float *hk = w.h + k * C::SB;
                const float hc = hk[col];
                g += w.e[k] * hc;
                const float hw = HAS_A ? hc * w.a[k] : hc;
                if constexpr (B >= 4) {
#pragma unroll
                    for (int j = 0; j < B; j += 4) {
                        const float4 v = *reinterpret_cast<const float4 *>(hk + j);
                        acc[j] += v.x * hw;
                        acc[j + 1] += v.y * hw;
                        acc[j + 2] += v.z * hw;
                        acc[j + 3] += v.w * hw;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < B; ++j) acc[j] += hk[j] * hw;
                }
            }
        }
#pragma unroll
        for (int m = B; m < 32; m <<= 1) {
#pragma unroll
            for (int j = 0; j < B; ++j) acc[j] += __shfl_xor_sync(kFull, acc[j], m);
            g += __shfl_xor_sync(kFull, g, m);
        }
        if (tk.slot >= 0) {  // a chunk of a long row: store the partial statistics
            if (sub == 0) {
                float *P = a.part + (int64_t)tk.slot * (B * B + B);
#pragma unroll
                for (int j = 0; j < B; ++j) P[j * B + col] = acc[j];
                P[B * B + col] = g;
            }
            continue;
        }
        const int row = tk.row;
        const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
#pragma unroll
        for (int j = 0; j < B; ++j) acc[j] += sGpp[j * B + col] + (j == col ? lam : 0.f);
        g += a.R[(int64_t)row * B + col];
        float delta;
        if (!chol_solve<B>(acc, g, col, sub, w, a.force_fp64 != 0, delta)) {
            queue_retry(a, lane, row);
            continue;
        }
        if (sub == 0) apply_delta(a.X, a.Xh, a.Xl, (int64_t)row * a.d + a.p0 + col, delta);
        __syncwarp();
        if (sub == 0) w.v[col] = delta;
        __syncwarp();
        if (tk.len <= C::CH) {  // the slices are still staged
            if (lane < tk.len) a.e[q] -= dot_slice<B>(w.v, w.h + lane * C::SB);
        } else {
            for (int c0 = 0; c0 < tk.len; c0 += C::CH) {
                const int cnt = min(C::CH, tk.len - c0);
                stage_chunk<B, PERM, HAS_A, false>(a, tk.begin + c0, cnt, lane, w, q);
                if (lane < cnt) a.e[q] -= dot_slice<B>(w.v, w.h + lane * C::SB);
            }
        }
    }
}

// ------------------------------------------------- tiled kernel, B = 8, 16, 32
// Same step as k_sparse, with the b x b statistics accumulated in registers by
// lane tiles.  A_r is cut into a 4 x 4 grid of T x T tiles (T = B / 4); only
// the 10 tiles on or below the diagonal are formed.  Lane l < 30 belongs to
// interaction group grp = l / 10 (the three groups take interactions k = grp,
// grp + 3, ...) and owns tile t = l % 10, so every staged interaction costs a
// lane T*T FMAs with 2 T / 4 shared loads.  The three group partials are summed
// in a fixed order into a shared copy of A_r, whose rows then feed the same
// warp solver as k_sparse.  Slices are gathered with cp.async into two
// staging buffers, so the next 32 interactions load while the current ones are
// multiplied.
template <int B>
struct TileCfg {
    static constexpr int T = B / 4;
    static constexpr int NT = 10, NG = 3, ACTIVE = NT * NG;
    static constexpr int SB = B + 4;
    static constexpr int CH = 32;
    static constexpr int BUF = CH * SB;
    static constexpr int VEC = (B + 3) / 4 * 4;
    static constexpr int WARP_FLOATS = 2 * BUF + 4 * CH + 2 * VEC;
    static constexpr int WARPS = 8;
    static constexpr int SMEM_BYTES = (B * B + WARPS * WARP_FLOATS) * 4;
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Issue the gathers of `cnt` slices (column id of slice k held by lane k) into buf.
template <int B>
__device__ __forceinline__ void gather_async(float *buf, const float *__restrict__ F, int d, int p0,
                                             int c_lane, int cnt, int lane) {
    constexpr int SB = TileCfg<B>::SB;
    constexpr int VPR = B / 4, RPP = 32 / VPR, NP = 32 / RPP;
    const int v = lane % VPR, rr = lane / VPR;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int k = p * RPP + rr;
        const int ck = __shfl_sync(kFull, c_lane, k);
        if (k < cnt) cp_async16(buf + k * SB + 4 * v, F + (int64_t)ck * d + p0 + 4 * v);
    }
}

template <int T>
__device__ __forceinline__ void load_seg(const float *p, float (&x)[T]) {
    if constexpr (T % 4 == 0) {
#pragma unroll
        for (int i = 0; i < T; i += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(p + i);
            x[i] = v.x; x[i + 1] = v.y; x[i + 2] = v.z; x[i + 3] = v.w;
        }
    } else {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        x[0] = v.x; x[1] = v.y;
    }
}

template <int T>
__device__ __forceinline__ void store_tile(float *p, const float (&x)[T], bool add) {
    if constexpr (T % 4 == 0) {
#pragma unroll
        for (int i = 0; i < T; i += 4) {
            float4 v = make_float4(x[i], x[i + 1], x[i + 2], x[i + 3]);
            if (add) {
                const float4 o = *reinterpret_cast<const float4 *>(p + i);
                v.x += o.x; v.y += o.y; v.z += o.z; v.w += o.w;
            }
            *reinterpret_cast<float4 *>(p + i) = v;
        }
    } else {
        float2 v = make_float2(x[0], x[1]);
        if (add) {
            const float2 o = *reinterpret_cast<const float2 *>(p);
            v.x += o.x; v.y += o.y;
        }
        *reinterpret_cast<float2 *>(p) = v;
    }
}

template <int B, bool PERM, bool HAS_A>
__global__ void __launch_bounds__(256, 2) k_sparse_tiled(const StepArgs a) {
    using C = TileCfg<B>;
    constexpr int T = C::T, SB = C::SB, CH = C::CH;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *sGpp = smem;
    // alpha0 G_pipi, exactly symmetric (taken from its lower triangle: the solver
    // treats the trailing block as symmetric); lane col reads column col, which
    // is free of bank conflicts
    for (int i = threadIdx.x; i < B * B; i += blockDim.x)
        sGpp[i] = a.alpha0 * a.G[(int64_t)(a.p0 + max(i / B, i % B)) * B + min(i / B, i % B)];
    float *wbase = smem + B * B + warp * C::WARP_FLOATS;
    // buffer bi (0 or 1): slices at wbase + bi * BUF, residuals at she + bi * CH,
    // weights at sha + bi * CH
    float *const she = wbase + 2 * C::BUF;
    float *const sha = she + 2 * CH;
    float *gs = wbase + 2 * C::BUF + 4 * CH;   // gradient (B)
    float *vv = gs + C::VEC;                   // delta (B)
    __syncthreads();
    WarpSmem w;
    w.v = vv;
    w.L = wbase + C::BUF;  // the solver's column buffers reuse the second staging buffer
    const int col = lane % B, sub = lane / B;
    const bool active = lane < C::ACTIVE;
    const int grp = active ? lane / C::NT : C::NG, t = lane % C::NT;
    const int ti = t >= 6 ? 3 : (t >= 3 ? 2 : (t >= 1 ? 1 : 0));
    const int tj = t - ti * (ti + 1) / 2;
    int nxt = 0;  // lane 0: the next task index, fetched while the current task runs
    if (lane == 0) nxt = atomicAdd(a.counter, 1);
    for (;;) {
        const int tsk = __shfl_sync(kFull, nxt, 0);
        if (tsk >= a.n_tasks) break;
        if (lane == 0) nxt = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float acc[T][T], gacc[T];
#pragma unroll
        for (int i = 0; i < T; ++i) {
            gacc[i] = 0.f;
#pragma unroll
            for (int j = 0; j < T; ++j) acc[i][j] = 0.f;
        }
        // chunk meta in registers: column id, residual index, residual, weight
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
            gather_async<B>(wbase + bi * C::BUF, a.F, a.d, a.p0, cB, cnt, lane);
            she[bi * CH + lane] = HAS_A ? aB * eB : eB;
            if (HAS_A) sha[bi * CH + lane] = aB;
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
            const float *bp = wbase + bi * C::BUF;
            const float *be = she + bi * CH;
            const float *ba = sha + bi * CH;
            for (int k = grp; k < cnt; k += C::NG) {
                const float *xk = bp + k * SB;
                float xa[T], xb[T];
                load_seg<T>(xk + T * ti, xa);
                load_seg<T>(xk + T * tj, xb);
                const float ek = be[k];
#pragma unroll
                for (int i = 0; i < T; i += 2) fma2(gacc[i], gacc[i + 1], ek, ek, xa[i], xa[i + 1]);
                if (HAS_A) {
                    const float ak = ba[k];
#pragma unroll
                    for (int i = 0; i < T; i += 2) mul2(xa[i], xa[i + 1], ak, ak);
                }
                // pairs (i, j), (i + 1, j + 1) and (i, j + 1), (i + 1, j): both
                // operands are adjacent pairs of the staged slices
#pragma unroll
                for (int i = 0; i < T; i += 2)
#pragma unroll
                    for (int j = 0; j < T; j += 2) {
                        fma2(acc[i][j], acc[i + 1][j + 1], xa[i], xa[i + 1], xb[j], xb[j + 1]);
                        fma2(acc[i][j + 1], acc[i + 1][j], xa[i], xa[i + 1], xb[j + 1], xb[j]);
                    }
            }
            __syncwarp();
        }
        // fixed-order sum of the three group partials into the shared A_r (buffer 1)
        float *As = wbase + C::BUF;
#pragma unroll
        for (int ph = 0; ph < C::NG; ++ph) {
            if (grp == ph) {
#pragma unroll
                for (int i = 0; i < T; ++i) store_tile<T>(As + (T * ti + i) * SB + T * tj, acc[i], ph > 0);
                if (tj == 0) {
#pragma unroll
                    for (int i = 0; i < T; ++i) gs[T * ti + i] = (ph > 0 ? gs[T * ti + i] : 0.f) + gacc[i];
                }
            }
            __syncwarp();
        }
        // row col of A_r, both triangles: only tiles on or below the diagonal
        // were formed, so entries right of the diagonal come from column col
        float A[B];
#pragma unroll
        for (int j = 0; j < B; j += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(As + col * SB + j);
            A[j] = v.x; A[j + 1] = v.y; A[j + 2] = v.z; A[j + 3] = v.w;
        }
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const float u = As[j * SB + col];
            if (j > col) A[j] = u;
        }
        float g = gs[col];
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
        if (nch > 0) {
            // the last chunk is projected from buffer 0 while chunks 0 .. nch - 2
            // (full chunks) are re-gathered into alternating buffers
            const int clast = tk.len - (nch - 1) * CH;
            int64_t qlast = 0;
            if (lane < clast) {
                const int64_t s = tk.begin + (int64_t)(nch - 1) * CH + lane;
                qlast = PERM ? (int64_t)a.pos[s] : s;
            }
            auto meta2 = [&](int j) {
                const int64_t s = tk.begin + (int64_t)j * CH + lane;
                cB = a.idx[s];
                qB = PERM ? (int64_t)a.pos[s] : s;
            };
            int64_t qc = 0;
            if (nch > 1) {
                meta2(0);
                qc = qB;
                gather_async<B>(wbase + C::BUF, a.F, a.d, a.p0, cB, CH, lane);
                cp_async_commit();
                if (nch > 2) meta2(1);
            }
            if (lane < clast) a.e[qlast] -= dot_slice<B>(vv, wbase + lane * SB);
            __syncwarp();
            for (int ch = 0; ch + 1 < nch; ++ch) {  // chunk ch sits in buffer (ch + 1) & 1
                const int bi = (ch + 1) & 1;
                cp_async_wait_all();
                __syncwarp();
                int64_t qn = 0;
                if (ch + 2 < nch) {
                    gather_async<B>(wbase + (bi ^ 1) * C::BUF, a.F, a.d, a.p0, cB, CH, lane);
                    cp_async_commit();
                    qn = qB;
                    if (ch + 3 < nch) meta2(ch + 2);
                }
                a.e[qc] -= dot_slice<B>(vv, wbase + bi * C::BUF + lane * SB);
                __syncwarp();
                qc = qn;
            }
        }
    }
}

// One block per split row: 256 threads sum the partial slots of the row in
// slot order (thread t owns elements t, t + 256, ...; its elements' sums run side
// by side so that the loads of several slots are in flight at once), then warp 0
// adds the dense terms, solves (the warp Gauss-Jordan elimination of the unsplit
// rows; Cholesky below b = 4) and applies.
template <int B>
__global__ void __launch_bounds__(256, 2) k_split_solve(const StepArgs a) {
    constexpr int NE = B * B + B;
    constexpr int PER = (NE + 255) / 256;
    extern __shared__ float4 smem4[];
    float *red = reinterpret_cast<float *>(smem4);
    WarpSmem w;
    w.v = red + (NE + 3) / 4 * 4;
    w.L = w.v + (B + 3) / 4 * 4;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = lane % B, sub = lane / B;
    for (int i = blockIdx.x; i < a.n_split; i += gridDim.x) {
        const SplitRow sr = a.split[i];
        const float *P0 = a.part + (int64_t)sr.slot0 * NE;
        float t[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) t[k] = 0.f;
#pragma unroll 4
        for (int sl = 0; sl < sr.nslots; ++sl) {
            const float *P = P0 + (int64_t)sl * NE;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                const int e = threadIdx.x + 256 * k;
                if (e < NE) t[k] += P[e];
            }
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + 256 * k;
            if (e < NE) red[e] = t[k];
        }
        __syncthreads();
        if (warp == 0) {
            float acc[B];
#pragma unroll
            for (int j = 0; j < B; ++j) acc[j] = red[col * B + j];
            float g = red[B * B + col];
            const float lam = a.lambda * (1.0f + a.nu * (float)sr.len);
#pragma unroll
            for (int j = 0; j < B; ++j)
                acc[j] += a.alpha0 * a.G[(int64_t)(a.p0 + max(j, col)) * B + min(j, col)] + (j == col ? lam : 0.f);
            g += a.R[(int64_t)sr.row * B + col];
            float delta = 0.f;
            bool ok;
            if constexpr (B % 4 == 0) ok = gj_solve2<B>(acc, g, col, sub, w, a.force_fp64 != 0, delta);
            else ok = chol_solve<B>(acc, g, col, sub, w, a.force_fp64 != 0, delta);
            if (!ok) {
                queue_retry(a, lane, sr.row);
                delta = 0.f;  // k_split_resid leaves the row's residuals alone
            } else if (sub == 0) {
                apply_delta(a.X, a.Xh, a.Xl, (int64_t)sr.row * a.d + a.p0 + col, delta);
            }
            if (sub == 0) a.delta[(int64_t)i * B + col] = delta;
        }
        __syncthreads();
    }
}

template <int B>
constexpr int split_solve_smem() {
    return ((B * B + B + 3) / 4 * 4 + (B + 3) / 4 * 4 + SparseCfg<B>::LREG) * 4;
}

// One warp per chunk of a split row: e_s -= <delta_row, f_{c_s,pi}>.
template <int B, bool PERM>
__global__ void __launch_bounds__(256) k_split_resid(const StepArgs a, const Task *__restrict__ stasks,
                                                     int32_t n_stasks) {
    using C = SparseCfg<B>;
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const WarpSmem w = warp_smem<B>(smem, warp);
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < n_stasks; t += nw) {
        const Task tk = stasks[t];
        __syncwarp();
        if (lane < B) w.v[lane] = a.delta[(int64_t)tk.srow * B + lane];
        int64_t q = 0;
        for (int c0 = 0; c0 < tk.len; c0 += C::CH) {
            const int cnt = min(C::CH, tk.len - c0);
            stage_chunk<B, PERM, false, false>(a, tk.begin + c0, cnt, lane, w, q);
            if (lane < cnt) a.e[q] -= dot_slice<B>(w.v, w.h + lane * C::SB);
        }
    }
}

// Residual update of split rows with register gathers (B a multiple of 4):
// e_s -= <delta_row, f_{c_s,pi}> over the pieces (<= 128 interactions) of the
// split rows.  Persistent: warps take pieces from an atomic counter (zeroed by
// the launcher; the list is sorted by decreasing length).  SG lanes share an
// interaction (MAXV float4 each), U interactions per sub-group are loaded
// before any is reduced, and the column ids and residual positions of the
// next 32 interactions are loaded before the current ones are used.  Pieces
// are disjoint and each e_s is updated by one lane, so the result does not
// depend on the schedule.
template <int B>
struct ResRegCfg {
    static constexpr int NV4 = B / 4;
    static constexpr int sgl() {
        int g = 0;
        while ((2 << g) <= 32 && (2 << g) * 4 <= NV4) ++g;
        return g;
    }
    static constexpr int SGL = sgl(), SG = 1 << SGL, NSUB = 32 / SG;
    static constexpr int MAXV = (NV4 + SG - 1) / SG;
    static constexpr int UMAX = MAXV >= 16 ? 1 : (MAXV >= 8 ? 2 : 4);
    static constexpr int U = SG < UMAX ? SG : UMAX;
};

template <int B, bool PERM>
__global__ void __launch_bounds__(256) k_split_resid_reg(const StepArgs a) {
    using C = ResRegCfg<B>;
    constexpr int SGL = C::SGL, SG = C::SG, NSUB = C::NSUB, MAXV = C::MAXV, U = C::U, NV4 = C::NV4;
    const int lane = threadIdx.x & 31;
    const int sub = lane >> SGL, sl = lane & (SG - 1);
    const float4 *F4 = reinterpret_cast<const float4 *>(a.F);
    const float4 *D4 = reinterpret_cast<const float4 *>(a.delta);
    const int64_t d4 = a.d >> 2, p4 = a.p0 >> 2;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.n_stasks) break;
        const Task tk = a.stasks[t];
        float4 dv[MAXV];
#pragma unroll
        for (int m = 0; m < MAXV; ++m) {
            const int v = sl + m * SG;
            dv[m] = v < NV4 ? D4[(int64_t)tk.srow * NV4 + v] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int64_t beg = tk.begin, end = tk.begin + tk.len;
        int my_c = 0, my_q = 0;
        if (beg + lane < end) {
            my_c = a.idx[beg + lane];
            my_q = PERM ? a.pos[beg + lane] : (int)(beg + lane);
        }
        for (int64_t s0 = beg; s0 < end; s0 += 32) {
            const int cnt = (int)min((int64_t)32, end - s0);
            int nx_c = 0, nx_q = 0;
            if (s0 + 32 + lane < end) {
                nx_c = a.idx[s0 + 32 + lane];
                nx_q = PERM ? a.pos[s0 + 32 + lane] : (int)(s0 + 32 + lane);
            }
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
                        h[q][m] = (k < cnt && v < NV4) ? __ldg(F4 + c * d4 + p4 + v)
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
#pragma unroll
                    for (int m = 0; m < MAXV; ++m)
                        acc[q] += dv[m].x * h[q][m].x + dv[m].y * h[q][m].y + dv[m].z * h[q][m].z +
                                  dv[m].w * h[q][m].w;
#pragma unroll
                    for (int o = SG >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], o);
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int k = sub + NSUB * (m0 + q);
                    const int qk = __shfl_sync(kFull, my_q, k);
                    if (sl == 0 && k < cnt) a.e[qk] -= acc[q];
                }
            }
            my_c = nx_c;
            my_q = nx_q;
        }
    }
}

// The same residual update for the BF16 path, gathering the fixed side's hi and
// lo shadows (the arrays the BF16 sparse kernel reads) instead of the FP32
// factors, so the item pass keeps one copy of the fixed side hot in L2;
// f = hi + lo is formed in FP32, as in the BF16 kernel's own residual update.
// SG lanes share an interaction, one 16-byte chunk (8 coordinates) of hi and of
// lo each, with U interactions per sub-group loaded before any is reduced.
template <int B>
struct ResRegBfCfg {
    static constexpr int NV8 = B / 8;                    // 16-byte chunks per slice
    static constexpr int SG = NV8 < 8 ? NV8 : 8;         // lanes per interaction
    static constexpr int SGL = SG == 1 ? 0 : SG == 2 ? 1 : SG == 4 ? 2 : 3;
    static constexpr int NSUB = 32 / SG, MAXV = NV8 / SG;
    static constexpr int U = SG < 4 ? SG : 4;
};

template <int B, bool PERM>
__global__ void __launch_bounds__(256) k_split_resid_reg_bf16(const StepArgs a) {
    using C = ResRegBfCfg<B>;
    constexpr int SGL = C::SGL, SG = C::SG, NSUB = C::NSUB, MAXV = C::MAXV, U = C::U, NV8 = C::NV8;
    const int lane = threadIdx.x & 31;
    const int sub = lane >> SGL, sl = lane & (SG - 1);
    const uint4 *Fh = reinterpret_cast<const uint4 *>(a.Fh);
    const uint4 *Fl = reinterpret_cast<const uint4 *>(a.Fl);
    const int64_t d8 = a.d >> 3, p8 = a.p0 >> 3;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= a.n_stasks) break;
        const Task tk = a.stasks[t];
        float dv[MAXV][8];
#pragma unroll
        for (int m = 0; m < MAXV; ++m)
#pragma unroll
            for (int q = 0; q < 8; ++q) dv[m][q] = a.delta[(int64_t)tk.srow * B + 8 * (sl + m * SG) + q];
        const int64_t beg = tk.begin, end = tk.begin + tk.len;
        int my_c = 0, my_q = 0;
        if (beg + lane < end) {
            my_c = a.idx[beg + lane];
            my_q = PERM ? a.pos[beg + lane] : (int)(beg + lane);
        }
        for (int64_t s0 = beg; s0 < end; s0 += 32) {
            const int cnt = (int)min((int64_t)32, end - s0);
            int nx_c = 0, nx_q = 0;
            if (s0 + 32 + lane < end) {
                nx_c = a.idx[s0 + 32 + lane];
                nx_q = PERM ? a.pos[s0 + 32 + lane] : (int)(s0 + 32 + lane);
            }
#pragma unroll
            for (int m0 = 0; m0 < SG; m0 += U) {
                float acc[U];
                uint4 hv[U][MAXV], lv[U][MAXV];
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int k = sub + NSUB * (m0 + q);
                    const int64_t c = __shfl_sync(kFull, my_c, k);
                    acc[q] = 0.f;
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) {
                        const int v = sl + m * SG;
                        const bool ok = k < cnt && v < NV8;
                        hv[q][m] = ok ? __ldg(Fh + c * d8 + p8 + v) : make_uint4(0u, 0u, 0u, 0u);
                        lv[q][m] = ok ? __ldg(Fl + c * d8 + p8 + v) : make_uint4(0u, 0u, 0u, 0u);
                    }
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
#pragma unroll
                    for (int m = 0; m < MAXV; ++m) {
                        const unsigned hw[4] = {hv[q][m].x, hv[q][m].y, hv[q][m].z, hv[q][m].w};
                        const unsigned lw[4] = {lv[q][m].x, lv[q][m].y, lv[q][m].z, lv[q][m].w};
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float2 fh = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hw[r]));
                            const float2 fl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lw[r]));
                            acc[q] += dv[m][2 * r] * (fh.x + fl.x) + dv[m][2 * r + 1] * (fh.y + fl.y);
                        }
                    }
#pragma unroll
                    for (int o = SG >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(kFull, acc[q], o);
                }
#pragma unroll
                for (int q = 0; q < U; ++q) {
                    const int k = sub + NSUB * (m0 + q);
                    const int qk = __shfl_sync(kFull, my_q, k);
                    if (sl == 0 && k < cnt) a.e[qk] -= acc[q];
                }
            }
            my_c = nx_c;
            my_q = nx_q;
        }
    }
}

template <int B, bool PERM>
cudaError_t launch_split_resid_reg_bf16(const StepArgs &a, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int n = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_split_resid_reg_bf16<B, PERM>, 256, 0);
        if (err != cudaSuccess) return err;
        per_sm = n > 0 ? n : 1;
    }
    if constexpr (PERM && B % 8 == 0) {  // item side: the user-major scan where it applies
        cudaError_t err = split_scan_prepare<B, true>(nullptr);
        if (err != cudaSuccess) return err;
        if (split_scan_applies<B>(a)) return launch_split_resid_scan<B, true>(a, s);
    }
    if (a.n_stasks <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(int32_t), s);
    if (err != cudaSuccess) return err;
    int grid = 152 * per_sm;
    const int need = (a.n_stasks + 7) / 8;
    if (grid > need) grid = need;
    prof_mark(a.prof, K_SPLIT_RESID, s);
    k_split_resid_reg_bf16<B, PERM><<<grid, 256, 0, s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

template <int B, bool PERM>
cudaError_t launch_split_resid_reg(const StepArgs &a, cudaStream_t s) {
    static int per_sm = 0;
    if (per_sm == 0) {
        int n = 0;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_split_resid_reg<B, PERM>, 256, 0);
        if (err != cudaSuccess) return err;
        per_sm = n > 0 ? n : 1;
    }
    if constexpr (PERM && B % 8 == 0) {  // item side: the user-major scan where it applies
        cudaError_t err = split_scan_prepare<B, false>(nullptr);
        if (err != cudaSuccess) return err;
        if (split_scan_applies<B>(a)) return launch_split_resid_scan<B, false>(a, s);
    }
    if (a.n_stasks <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(a.counter, 0, sizeof(int32_t), s);
    if (err != cudaSuccess) return err;
    int grid = 152 * per_sm;
    const int need = (a.n_stasks + 7) / 8;
    if (grid > need) grid = need;
    prof_mark(a.prof, K_SPLIT_RESID, s);
    k_split_resid_reg<B, PERM><<<grid, 256, 0, s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

// FP64 re-solve of queued rows: statistics accumulated from scratch in FP64
// (the FP32 row term R_r is reused), Cholesky in FP64.  A row that still has
// a pivot that is not positive, or below 1e-13 of its original diagonal (the
// matrix is singular to FP64 working accuracy), is counted as not positive
// definite and left unchanged.
template <int B, bool PERM, bool HAS_A>
__global__ void __launch_bounds__(128) k_retry(const StepArgs a) {
    __shared__ double sv[4][32];
    __shared__ double sL[4][B * (B + 1)];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int col = lane % B, sub = lane / B;
    constexpr int G = 32 / B;
    const int count = *(volatile int *)a.retry;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nw) {
        const int row = a.retry[1 + i];
        const int64_t beg = a.ptr[row], end = a.ptr[row + 1];
        double A[B];
#pragma unroll
        for (int j = 0; j < B; ++j) A[j] = 0.0;
        double g = 0.0;
        for (int64_t s = beg + sub; s < end; s += G) {
            const int64_t q = PERM ? (int64_t)a.pos[s] : s;
            const float *h = a.F + (int64_t)a.idx[s] * a.d + a.p0;
            const double al = HAS_A ? (double)a.alpha[q] : 1.0;
            const double hc = h[col];
            g += al * (double)a.e[q] * hc;
#pragma unroll
            for (int j = 0; j < B; ++j) A[j] += al * (double)h[j] * hc;
        }
#pragma unroll
        for (int m = B; m < 32; m <<= 1) {
#pragma unroll
            for (int j = 0; j < B; ++j) A[j] += __shfl_xor_sync(kFull, A[j], m);
            g += __shfl_xor_sync(kFull, g, m);
        }
        const double lam = (double)a.lambda * (1.0 + (double)a.nu * (double)(end - beg));
#pragma unroll
        for (int j = 0; j < B; ++j)
            A[j] += (double)a.alpha0 * (double)a.G[(int64_t)(a.p0 + max(j, col)) * B + min(j, col)] +
                    (j == col ? lam : 0.0);
        g += (double)a.R[(int64_t)row * B + col];
        // right-looking Cholesky, lane col holds row col
        double diag0 = 0.0;
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (j == col) diag0 = A[j];
        bool ok = true;
        double inv_diag = 0.0;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const double akk = __shfl_sync(kFull, A[k], k);
            const double d0 = __shfl_sync(kFull, diag0, k);
            ok = ok && (akk > 1e-13 * d0) && (akk < 1e300);
            const double lkk = sqrt(akk > 0.0 ? akk : 1e-300);
            const double lck = A[k] / lkk;
            if (col == k) inv_diag = 1.0 / lkk;
            A[k] = lck;
            __syncwarp();
            if (sub == 0) sv[warp][col] = lck;
            __syncwarp();
#pragma unroll
            for (int j = k + 1; j < B; ++j) A[j] -= lck * sv[warp][j];
        }
        if (!ok) {
            if (lane == 0) atomicAdd((unsigned long long *)&a.stats[1], 1ull);
            continue;
        }
        double z = g;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            const double zk = __shfl_sync(kFull, z * inv_diag, k);
            if (col > k) z -= A[k] * zk;
            else if (col == k) z = zk;
        }
        __syncwarp();
        if (sub == 0) {
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (j <= col) sL[warp][col * (B + 1) + j] = A[j];
        }
        __syncwarp();
        double x = z;
#pragma unroll
        for (int k = B - 1; k >= 0; --k) {
            const double xk = __shfl_sync(kFull, x * inv_diag, k);
            if (col < k) x -= sL[warp][k * (B + 1) + col] * xk;
            else if (col == k) x = xk;
        }
        const float delta = (float)x;
        if (sub == 0) apply_delta(a.X, a.Xh, a.Xl, (int64_t)row * a.d + a.p0 + col, delta);
        __syncwarp();
        if (sub == 0) sv[warp][col] = (double)delta;
        __syncwarp();
        for (int64_t s = beg + lane; s < end; s += 32) {
            const int64_t q = PERM ? (int64_t)a.pos[s] : s;
            const float *h = a.F + (int64_t)a.idx[s] * a.d + a.p0;
            float t = 0.f;
#pragma unroll
            for (int j = 0; j < B; ++j) t += (float)sv[warp][j] * h[j];
            a.e[q] -= t;
        }
        if (lane == 0) atomicAdd((unsigned long long *)&a.stats[0], 1ull);
    }
}

template <int B, bool PERM, bool HAS_A>
constexpr auto main_kernel() {
    if constexpr (B >= 8) return k_sparse_tiled<B, PERM, HAS_A>;
    else return k_sparse<B, PERM, HAS_A>;
}

template <int B, bool PERM, bool HAS_A>
cudaError_t launch_step_b(const StepArgs &a, cudaStream_t s) {
    using C = SparseCfg<B>;
    constexpr bool TILED = B >= 8;
    auto kmain = main_kernel<B, PERM, HAS_A>();
    constexpr int MAIN_SMEM = TILED ? TileCfg<(B >= 8 ? B : 8)>::SMEM_BYTES : C::SMEM_BYTES;
    static bool attr_done = false;
    static int per_sm = 0;
    if (!attr_done) {
        cudaError_t e1 = cudaFuncSetAttribute(kmain, cudaFuncAttributeMaxDynamicSharedMemorySize, MAIN_SMEM);
        cudaError_t e2 = cudaFuncSetAttribute(k_split_solve<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              split_solve_smem<B>());
        cudaError_t e3 = cudaSuccess;
        if constexpr (B % 4 != 0)
            e3 = cudaFuncSetAttribute(k_split_resid<B, PERM>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
        if (e1 != cudaSuccess) return e1;
        if (e2 != cudaSuccess) return e2;
        if (e3 != cudaSuccess) return e3;
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, kmain, C::WARPS * 32, MAIN_SMEM);
        if (err != cudaSuccess) return err;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    int grid = 152 * per_sm;
    const int need = (a.n_tasks + C::WARPS - 1) / C::WARPS;
    if (grid > need) grid = need > 0 ? need : 1;
    if (a.n_tasks > 0) {
        prof_mark(a.prof, K_SPARSE, s);
        kmain<<<grid, C::WARPS * 32, MAIN_SMEM, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 8 ? a.n_split : 152 * 8;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve<B><<<g2, 256, split_solve_smem<B>(), s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    return cudaGetLastError();
}

template <int B, bool PERM, bool HAS_A>
cudaError_t launch_split_resid_b(const StepArgs &a, cudaStream_t s) {
    using C = SparseCfg<B>;
    if constexpr (B % 4 == 0) {
        cudaError_t e = launch_split_resid_reg<B, PERM>(a, s);
        if (e != cudaSuccess) return e;
    } else if (a.n_stasks > 0) {
        int g3 = (a.n_stasks + C::WARPS - 1) / C::WARPS;
        if (g3 > 152 * 8) g3 = 152 * 8;
        prof_mark(a.prof, K_SPLIT_RESID, s);
        k_split_resid<B, PERM><<<g3, C::WARPS * 32, C::SMEM_BYTES, s>>>(a, a.stasks, a.n_stasks);
        prof_mark(a.prof, -1, s);
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry<B, PERM, HAS_A><<<38, 128, 0, s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

// Whole sparse part of a block-side step for block size B.
template <int B, bool PERM, bool HAS_A>
cudaError_t launch_sparse_all(const StepArgs &a, cudaStream_t s) {
    cudaError_t e = launch_step_b<B, PERM, HAS_A>(a, s);
    if (e != cudaSuccess) return e;
    return launch_split_resid_b<B, PERM, HAS_A>(a, s);
}

template <int B>
cudaError_t launch_sparse_dispatch(const StepArgs &a, cudaStream_t s) {
    const bool perm = a.pos != nullptr, wa = a.alpha != nullptr;
    if (perm) return wa ? launch_sparse_all<B, true, true>(a, s) : launch_sparse_all<B, true, false>(a, s);
    return wa ? launch_sparse_all<B, false, true>(a, s) : launch_sparse_all<B, false, false>(a, s);
}

}  // namespace ials
