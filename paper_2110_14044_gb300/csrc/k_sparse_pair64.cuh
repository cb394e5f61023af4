// Block step of Algorithm 3 at block size b = 64, FP32, one row per pair of
// warps.
//
// A CTA holds four independent pairs.  A pair takes one task at a time from the
// longest-first work queue and carries it end to end with only its own named
// barrier (no CTA-wide synchronisation), so that one pair's gathers, products,
// solve and residual update overlap the other pairs' phases.
//
// Statistics (Eqs. 11-12).  The lower triangle of the 64 x 64 system in 8 x 8
// tiles is 28 off-diagonal tiles and 8 diagonal ones.  Each of the pair's 64
// threads owns one 4 x 8 half tile: the 56 halves of the off-diagonal tiles,
// and for each diagonal tile R its lower half (rows 8R + 4 .. 8R + 7, all 8
// columns).  The eight diagonal threads (the last eight lanes of the second
// warp) also accumulate the upper-left 4 x 4 block of their tile and the eight
// gradient entries of rows 8R .. 8R + 7, from operands they already hold.  So
// every staged interaction is read by all 64 threads once, each doing 16 paired
// FMAs (28 on the diagonal lanes), with no partial sums to combine.
//
// Solve (Eq. 9).  The tiles are written, mirrored into both triangles, to the
// (then idle) staging buffers in the solve layout: two rows per thread, the
// columns interleaved between the two threads of a row pair.  The pair runs a
// Gauss-Jordan elimination with 2 x 2 pivots in registers, one pair barrier per
// step; each pivot-row value read from shared memory updates two rows, which
// halves the shared-memory traffic of a one-row-per-thread elimination.  Apply,
// then the residual update (Eq. 7) over the row's chunks, gathered again.
//
// Gathers: chunks of 32 interactions through a double-buffered cp.async
// pipeline (column ids and positions two chunks ahead, slices and residuals
// one chunk ahead).  About 20 KB of shared memory per pair and at most 128
// registers per thread keep two CTAs (16 warps) on an SM.  Chunks of long rows
// store their partial statistics (lower tiles and gradient) to their slot for
// the split-row solve, as the other kernels do.
#pragma once

#include "k_sparse_cta_bf16.cuh"
#include "k_sparse_rc.cuh"

namespace ials {

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Barrier of the two warps (64 threads) of pair `pr` (ids 1 .. 4; id 0 is
// __syncthreads).
__device__ __forceinline__ void pair_sync(int pr) {
    asm volatile("bar.sync %0, 64;\n" ::"r"(pr + 1) : "memory");
}

struct Pair64 {
    static constexpr int B = 64, PAIRS = 4, THREADS = 64 * PAIRS;
    static constexpr int CH = 32, SB = B + 4, STAGE = CH * SB;
    static constexpr int P = 1, NS = P + 1, NI = 2 * P + 1;
    static constexpr int GJB = 2 * 2 * 72 + 8;          // published pivot columns (two steps), rhs, votes
    // floats per pair: stages (the system in their place), residuals, weights, ids,
    // positions, Gauss-Jordan exchange, right-hand side / solution, flags
    static constexpr int FLOATS = NS * STAGE + 2 * NS * CH + 2 * NI * CH + GJB + B + 4;
    static constexpr int SMEM_BYTES = PAIRS * FLOATS * 4;
    static_assert(FLOATS % 4 == 0, "pair regions stay 16-byte aligned");
    static_assert(B * B <= NS * STAGE, "the system fits in the staging buffers");
};

// BF16 statistics: a stage holds the hi and lo tiles of a chunk (bf16, rows of
// 72 with the residual in column 64).
struct Pair64Bf {
    static constexpr int B = 64, PAIRS = 4, THREADS = 64 * PAIRS;
    static constexpr int CH = 32, SBH = CtaBfCfg<64>::SBH, TILE = CH * SBH, STAGE = TILE;  // floats = 2 TILE bf16
    static constexpr int P = 1, NS = P + 1, NI = 2 * P + 1;
    static constexpr int GJB = Pair64::GJB;
    static constexpr int FLOATS = NS * STAGE + 2 * NS * CH + 2 * NI * CH + GJB + B + 4;
    static constexpr int SMEM_BYTES = PAIRS * FLOATS * 4;
    static_assert(FLOATS % 4 == 0, "pair regions stay 16-byte aligned");
    static_assert(B * B <= NS * STAGE, "the system fits in the staging buffers");
};

template <class C>
struct PairSmem {
    float *stage, *she, *sha, *gjb, *dl;  // gjb: Gauss-Jordan exchange; dl: right-hand side, then solution
    int *ci, *cq, *flag;                  // flag[0]: next task
    __device__ __forceinline__ explicit PairSmem(float *base) {
        stage = base;
        she = stage + C::NS * C::STAGE;
        sha = she + C::NS * C::CH;
        ci = reinterpret_cast<int *>(sha + C::NS * C::CH);
        cq = ci + C::NI * C::CH;
        gjb = reinterpret_cast<float *>(cq + C::NI * C::CH);
        dl = gjb + C::GJB;
        flag = reinterpret_cast<int *>(dl + C::B);
    }
};
using Pair64Smem = PairSmem<Pair64>;

// The 4 x 8 half tile of pair thread u: rows 8 ti + 4 h .. + 3, columns 8 tj .. + 7.
// u < 56: off-diagonal tile u / 2 (ti > tj, in row-major lower order), half u % 2;
// u >= 56: diagonal tile u - 56, lower half.
__device__ __forceinline__ void p64_unit(int u, int &ti, int &tj, int &h) {
    if (u >= 56) {
        ti = tj = u - 56;
        h = 1;
        return;
    }
    const int t = u >> 1;
    int i = 1;
    while ((i + 1) * i / 2 <= t) ++i;  // tiles with ti < i: i (i - 1) / 2
    ti = i;
    tj = t - i * (i - 1) / 2;
    h = u & 1;
}

__device__ __forceinline__ float4 p64_ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void p64_st4(float *p, float x, float y, float z, float w) {
    *reinterpret_cast<float4 *>(p) = make_float4(x, y, z, w);
}

// Software pipeline of one pair over `total` chunks.  stage0(i, ib): cp.async of
// chunk i's column ids / positions into id stage ib; stage1(i, sb, ib): the
// gathers of chunk i (reading its ids from id stage ib) into slice stage sb;
// body(j, sb, ib): the work on chunk j.  Every iteration commits one cp.async
// group, so waiting for all but the last P - 1 groups leaves chunk j's slices
// (and chunk j + P's ids) complete; the pair's barrier then publishes them.
template <typename S0, typename S1, typename Body>
__device__ __forceinline__ void p64_pipeline(int pr, int total, S0 stage0, S1 stage1, Body body) {
    constexpr int P = Pair64::P, NS = Pair64::NS, NI = Pair64::NI;
    for (int i = 0; i < 2 * P && i < total; ++i) stage0(i, i % NI);
    cp_async_commit();
    cp_async_wait_all();
    pair_sync(pr);
    for (int i = 0; i < P; ++i) {
        if (i < total) stage1(i, i % NS, i % NI);
        cp_async_commit();
    }
#pragma unroll 1
    for (int j = 0; j < total; ++j) {
        cp_async_wait_group<P - 1>();
        pair_sync(pr);
        const int n1 = j + P, n0 = j + 2 * P;
        if (n1 < total) stage1(n1, n1 % NS, n1 % NI);
        if (n0 < total) stage0(n0, n0 % NI);
        cp_async_commit();
        body(j, j % NS, j % NI);
    }
    cp_async_wait_all();
    pair_sync(pr);
}

// The row system for the solve, two rows per thread: thread 2 q + c of the pair
// holds rows 2 q and 2 q + 1 at the columns j = 2 m + c (m = 0 .. 31).  In shared
// memory (64 floats a row, over the staging buffers) entry (r, j) sits in the
// half j % 2 of row r, at position j / 2, its 4-float group XOR-ed with
// 2 ((r / 2) % 4) + j % 2, so that the eight threads of a quarter warp loading
// their rows hit eight different 4-bank groups.
__device__ __forceinline__ int p64_at(int r, int half, int group) {
    return r * 64 + half * 32 + 4 * (group ^ ((((r >> 1) & 3) << 1) | half));
}

// Gauss-Jordan elimination with 2 x 2 pivots of the SPD system held as above
// (A[t][m] = entry (2 q + t, 2 m + c), g[t] its right-hand side).  Step m
// eliminates columns k = 2 m, k + 1 with the pivot block [[a, b], [b, c]]: every
// thread publishes its two rows' entries in the column it holds of the pair
// (k + c), which by the symmetry of the trailing block are also the pivot rows'
// entries in the trailing columns; then every row r outside the pivot pair takes
// [s1, s2] = [A_rk, A_r,k+1] P^{-1} (its other column from the neighbouring
// thread) and updates A_rj -= s1 A_kj + s2 A_k+1,j for its columns j > k + 1, each
// published value serving both of the thread's rows.  One pair barrier per step
// (double-buffered exchange).  Pivots are checked against the original diagonal
// (not below 1e-5 of it, finite).  Returns 0 (uniformly) when every pivot passed
// and the solution is finite; x[t] is then solution entry 2 q + t.
__device__ __forceinline__ int p64_gj(float (&A)[2][32], float (&g)[2], float dorig, float *gjb, int pr, int pt,
                                      bool force_fail, float (&x)[2]) {
    const int rq = pt >> 1, ch = pt & 1, hw = pt >> 5;
    float *pub = gjb;                      // [2 steps][2 columns][2 (row % 2)][36: row / 2, padding]
    float *gb = gjb + 288;                 // [2 steps][2]
    int *vote = reinterpret_cast<int *>(gjb + 292);
    bool bad = force_fail;
    float pa = 1.f, pb = 0.f, pc = 1.f;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        float *b = pub + (m & 1) * 144;
        b[ch * 72 + rq] = A[0][m];         // entry (2 q, k + c)
        b[ch * 72 + 36 + rq] = A[1][m];    // entry (2 q + 1, k + c)
        if (rq == m && ch == 0) {
            gb[(m & 1) * 2] = g[0];
            gb[(m & 1) * 2 + 1] = g[1];
        }
        pair_sync(pr);
        const float a = b[m], bb = b[36 + m], c = b[72 + 36 + m];
        const float gk = gb[(m & 1) * 2], gk1 = gb[(m & 1) * 2 + 1];
        const float rdet = rcp_approx(a * c - bb * bb);
        const bool piv = rq == m;
        if (piv) {
            if (ch == 0) bad = bad || !(a > 1e-5f * dorig) || !(a <= 3.0e38f);
            else {
                const float d1 = c - bb * bb * rcp_approx(a);
                bad = bad || !(d1 > 1e-5f * dorig) || !(d1 <= 3.0e38f);
            }
            pa = a;
            pb = bb;
            pc = c;
        }
        float s1[2], s2[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const float other = __shfl_xor_sync(kFull, A[t][m], 1);
            const float xk = ch == 0 ? A[t][m] : other, yk = ch == 0 ? other : A[t][m];
            s1[t] = piv ? 0.f : (xk * c - yk * bb) * rdet;
            s2[t] = piv ? 0.f : (yk * a - xk * bb) * rdet;
        }
        const float *v1 = b + ch * 36, *v2 = b + 72 + ch * 36;  // entries (k, 2 m' + c), (k + 1, 2 m' + c)
#pragma unroll
        for (int q4 = (m + 1) >> 2; q4 < 8; ++q4) {
            const float4 p1 = p64_ld4(v1 + 4 * q4), p2 = p64_ld4(v2 + 4 * q4);
            const float u1[4] = {p1.x, p1.y, p1.z, p1.w}, u2[4] = {p2.x, p2.y, p2.z, p2.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int mm = 4 * q4 + e;
                if (mm > m) {
                    fma2(A[0][mm], A[1][mm], -s1[0], -s1[1], u1[e], u1[e]);
                    fma2(A[0][mm], A[1][mm], -s2[0], -s2[1], u2[e], u2[e]);
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) g[t] -= s1[t] * gk + s2[t] * gk1;
    }
    const float rd = rcp_approx(pa * pc - pb * pb);
    x[0] = (pc * g[0] - pb * g[1]) * rd;
    x[1] = (pa * g[1] - pb * g[0]) * rd;
    const bool fail = __any_sync(kFull, bad || !isfinite(x[0]) || !isfinite(x[1]));
    if ((pt & 31) == 0) vote[hw] = fail ? 1 : 0;
    pair_sync(pr);
    return vote[0] | vote[1];
}

template <bool PERM, bool HAS_A>
__global__ void __launch_bounds__(Pair64::THREADS, 2) k_sparse_pair64(const StepArgs a) {
    using C = Pair64;
    constexpr int B = 64, CH = C::CH, SB = C::SB;
    extern __shared__ float4 smem4[];
    const int pr = threadIdx.x >> 6, pt = threadIdx.x & 63;
    const Pair64Smem S(reinterpret_cast<float *>(smem4) + pr * C::FLOATS);
    int ti, tj, hh;
    p64_unit(pt, ti, tj, hh);
    const int ro = 8 * ti + 4 * hh, co = 8 * tj;
    const bool dg = pt >= 56;
    if (pt == 0) S.flag[0] = atomicAdd(a.counter, 1);
    for (;;) {
        pair_sync(pr);
        const int tsk = S.flag[0];
        if (tsk >= a.n_tasks) break;
        pair_sync(pr);  // the pair has read flag[0]
        if (pt == 0) S.flag[0] = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float acc[4][8], up[4][4], g[8];
        if (tk.slot < 0) {  // dense terms alpha0 G_pipi + lambda_r I and the row term
            const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
            const float *Gb = a.G + (int64_t)(a.p0 + ro) * B + co;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float v[8];
                load_seg<8>(Gb + i * B, v);
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = a.alpha0 * v[j] + (ro + i == co + j ? lam : 0.f);
            }
            if (dg) {
                const float *Gd = a.G + (int64_t)(a.p0 + co) * B + co;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float v[4];
                    load_seg<4>(Gd + i * B, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) up[i][j] = a.alpha0 * v[j] + (i == j ? lam : 0.f);
                }
                load_seg<8>(a.R + (int64_t)tk.row * B + co, g);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            if (dg) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) up[i][j] = 0.f;
#pragma unroll
                for (int j = 0; j < 8; ++j) g[j] = 0.f;
            }
        }
        auto cnt_of = [&](int c) { return min(CH, tk.len - c * CH); };
        auto stage0 = [&](int i, int ib) {  // column ids (and residual positions) of chunk i
            const int cnt = cnt_of(i);
            const int64_t s0 = tk.begin + (int64_t)i * CH;
            if (pt < cnt) cp_async4(S.ci + ib * CH + pt, a.idx + s0 + pt);
            if (PERM && pt >= 32 && pt - 32 < cnt) cp_async4(S.cq + ib * CH + pt - 32, a.pos + s0 + pt - 32);
        };
        auto stage1 = [&](int i, int sb, int ib) {  // slices, residuals and weights of chunk i
            const int cnt = cnt_of(i);
            const int *ids = S.ci + ib * CH;
            float *buf = S.stage + sb * C::STAGE;
            for (int f = pt; f < cnt * (B / 4); f += 64) {
                const int k = f >> 4, v = f & 15;
                cp_async16(buf + k * SB + 4 * v, a.F + (int64_t)ids[k] * a.d + a.p0 + 4 * v);
            }
            if (pt < cnt) {
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + pt] : tk.begin + (int64_t)i * CH + pt;
                cp_async4(S.she + sb * CH + pt, a.e + q);
                if (HAS_A) cp_async4(S.sha + sb * CH + pt, a.alpha + q);
            }
        };
        auto body = [&](int j, int sb, int) {
            const int cnt = cnt_of(j);
            const float *xs = S.stage + sb * C::STAGE;
            const float *es = S.she + sb * CH, *as = S.sha + sb * CH;
#pragma unroll 2
            for (int k = 0; k < cnt; ++k) {
                const float *xk = xs + k * SB;
                const float4 r4 = p64_ld4(xk + ro), c0 = p64_ld4(xk + co), c1 = p64_ld4(xk + co + 4);
                float xr[4] = {r4.x, r4.y, r4.z, r4.w};
                const float xc[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                float al = 1.f;
                if (HAS_A) {
                    al = as[k];
#pragma unroll
                    for (int i = 0; i < 4; ++i) xr[i] *= al;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 8; q += 2) fma2(acc[i][q], acc[i][q + 1], xr[i], xr[i], xc[q], xc[q + 1]);
                if (dg) {  // diagonal lanes: gradient and upper-left 4 x 4 (lower triangle) of the tile
                    const float ek = HAS_A ? es[k] * al : es[k];
#pragma unroll
                    for (int q = 0; q < 8; q += 2) fma2(g[q], g[q + 1], ek, ek, xc[q], xc[q + 1]);
                    const float m0 = xc[0] * al, m1 = xc[1] * al, m2 = xc[2] * al, m3 = xc[3] * al;
                    up[0][0] = fmaf(m0, xc[0], up[0][0]);
                    fma2(up[1][0], up[1][1], m1, m1, xc[0], xc[1]);
                    fma2(up[2][0], up[2][1], m2, m2, xc[0], xc[1]);
                    up[2][2] = fmaf(m2, xc[2], up[2][2]);
                    fma2(up[3][0], up[3][1], m3, m3, xc[0], xc[1]);
                    fma2(up[3][2], up[3][3], m3, m3, xc[2], xc[3]);
                }
            }
        };
        p64_pipeline(pr, nch, stage0, stage1, body);
        if (dg) {  // the diagonal tile is exactly symmetric: upper entries from the lower ones
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 5 + i; j < 8; ++j) acc[i][j] = acc[j - 4][4 + i];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = i + 1; j < 4; ++j) up[i][j] = up[j][i];
        }
        if (tk.slot >= 0) {  // chunk of a long row: lower tiles and gradient to its slot
            float *Pp = a.part + (int64_t)tk.slot * (B * B + B);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                p64_st4(Pp + (ro + i) * B + co, acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
                p64_st4(Pp + (ro + i) * B + co + 4, acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
            }
            if (dg) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    p64_st4(Pp + (co + i) * B + co, up[i][0], up[i][1], up[i][2], up[i][3]);
                    p64_st4(Pp + (co + i) * B + co + 4, acc[0][i], acc[1][i], acc[2][i], acc[3][i]);
                }
                p64_st4(Pp + B * B + co, g[0], g[1], g[2], g[3]);
                p64_st4(Pp + B * B + co + 4, g[4], g[5], g[6], g[7]);
            }
            continue;
        }
        float *M = S.stage;
        // the system (both triangles) in the solve layout, the right-hand side to dl
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ro + i;
            p64_st4(M + p64_at(r, 0, tj), acc[i][0], acc[i][2], acc[i][4], acc[i][6]);
            p64_st4(M + p64_at(r, 1, tj), acc[i][1], acc[i][3], acc[i][5], acc[i][7]);
        }
        if (!dg) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {  // mirror: row co + j, columns ro .. ro + 3
                const int r = co + j;
                *reinterpret_cast<float2 *>(M + p64_at(r, 0, ti) + 2 * hh) = make_float2(acc[0][j], acc[2][j]);
                *reinterpret_cast<float2 *>(M + p64_at(r, 1, ti) + 2 * hh) = make_float2(acc[1][j], acc[3][j]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) {  // rows co .. co + 3 of the diagonal tile
                const int r = co + i;
                p64_st4(M + p64_at(r, 0, tj), up[i][0], up[i][2], acc[0][i], acc[2][i]);
                p64_st4(M + p64_at(r, 1, tj), up[i][1], up[i][3], acc[1][i], acc[3][i]);
            }
            p64_st4(S.dl + co, g[0], g[1], g[2], g[3]);
            p64_st4(S.dl + co + 4, g[4], g[5], g[6], g[7]);
        }
        pair_sync(pr);
        const int rq = pt >> 1, chh = pt & 1;
        float A[2][32], gr[2], x[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int r = 2 * rq + t;
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
                const float4 u = p64_ld4(M + p64_at(r, chh, q4));
                A[t][4 * q4] = u.x; A[t][4 * q4 + 1] = u.y; A[t][4 * q4 + 2] = u.z; A[t][4 * q4 + 3] = u.w;
            }
            gr[t] = S.dl[r];
        }
        const int rown = 2 * rq + chh;  // the row whose diagonal entry this thread holds
        const float dorig = M[p64_at(rown, chh, rq >> 2) + (rq & 3)];
        const int vote = p64_gj(A, gr, dorig, S.gjb, pr, pt, a.force_fp64 != 0, x);
        if (vote) {
            if (pt == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        if (chh == 0) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                apply_delta(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + 2 * rq + t, x[t]);
                S.dl[2 * rq + t] = x[t];
            }
        }
        // residual update e_s -= <delta, f_{c_s, pi}>: two threads per interaction, 32 entries each
        const int k = pt >> 1, part = pt & 1;
        auto rbody = [&](int j, int sb, int ib) {
            const int cnt = cnt_of(j);
            float t = 0.f;
            if (k < cnt) {  // float4 groups 0-3, 8-11 (part 0) and 4-7, 12-15 (part 1): no bank conflicts
                const float *xk = S.stage + sb * C::STAGE + k * SB + 16 * part;
                const float *dv = S.dl + 16 * part;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int m = 4 * (u & 3) + 32 * (u >> 2);
                    const float4 f = p64_ld4(xk + m), w = p64_ld4(dv + m);
                    t = fmaf(w.x, f.x, t);
                    t = fmaf(w.y, f.y, t);
                    t = fmaf(w.z, f.z, t);
                    t = fmaf(w.w, f.w, t);
                }
            }
            t += __shfl_xor_sync(kFull, t, 1);
            if (k < cnt && part == 0) {
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + k] : tk.begin + (int64_t)j * CH + k;
                a.e[q] -= t;
            }
        };
        auto rstage1 = [&](int i, int sb, int ib) {
            const int cnt = cnt_of(i);
            const int *ids = S.ci + ib * CH;
            float *buf = S.stage + sb * C::STAGE;
            for (int f = pt; f < cnt * (B / 4); f += 64) {
                const int kk = f >> 4, v = f & 15;
                cp_async16(buf + kk * SB + 4 * v, a.F + (int64_t)ids[kk] * a.d + a.p0 + 4 * v);
            }
        };
        p64_pipeline(pr, nch, stage0, rstage1, rbody);
    }
}

template <bool PERM, bool HAS_A>
cudaError_t launch_sparse_pair64_all(const StepArgs &a, cudaStream_t s) {
    using C = Pair64;
    using CF = CtaCfg<64>;
    static bool attr_done = false;
    static int per_sm = 0;
    auto kern = k_sparse_pair64<PERM, HAS_A>;
    if (!attr_done) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_split_solve_rc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      RcCfg<64>::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_retry_cta<64, PERM, HAS_A, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, retry_cta_smem<64>())) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM_BYTES)) != cudaSuccess)
            return e;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    if (a.n_tasks > 0) {
        int grid = 152 * per_sm;
        const int need = (a.n_tasks + C::PAIRS - 1) / C::PAIRS;
        if (grid > need) grid = need;
        prof_mark(a.prof, K_SPARSE, s);
        kern<<<grid, C::THREADS, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 4 ? a.n_split : 152 * 4;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve_rc<64, false><<<g2, RcCfg<64>::THREADS, RcCfg<64>::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    {  // always called: the first call sizes the grid, outside any stream capture
        const cudaError_t e = launch_split_resid_reg<64, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry_cta<64, PERM, HAS_A, false><<<kRetryBlocks, CF::THREADS, retry_cta_smem<64>(), s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ BF16 statistics

// Entry (r, c) of the solve layout of p64_gj.
__device__ __forceinline__ float *p64_entry(float *M, int r, int c) {
    const int m = c >> 1;
    return M + p64_at(r, c & 1, m >> 2) + (m & 3);
}

// Pair warp PW does the tile lists of the CTA kernel's warps 2 PW and 2 PW + 1
// (k_sparse_cta_bf16.cuh): two 16-row blocks of the lower triangle, both halves,
// and their gradient tiles, as compensated hi/lo mma.sync products; the
// fragments of the blocks the two lists share are loaded once.
template <int PW>
__device__ __forceinline__ void pbf_kstep(float (&acc)[2][5][4], float (&gac)[2][4], const __nv_bfloat16 *th,
                                          const __nv_bfloat16 *tl, int ks, int lane) {
    using W0 = CtaBfWarp<64, 2 * PW>;
    using W1 = CtaBfWarp<64, 2 * PW + 1>;
    constexpr int MT = 4, SBH = CtaBfCfg<64>::SBH, NPT = CtaBfCfg<64>::NPT;
    constexpr unsigned MASK = W0::blocks() | W1::blocks();
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
    ldsm_x4_t(E, (mj < 2 ? th : tl) + (ks * 16 + (mj & 1) * 8 + mr) * SBH + 64);
#pragma unroll
    for (int s = 0; s < NPT; ++s) {
        {
            const int i = W0::ti(s), n = W0::tn(s), g2 = n >> 1, h = n & 1;
            mma_bf16(acc[0][s], Rh[i], Rh[g2][h], Rh[g2][h + 2]);
            mma_bf16(acc[0][s], Rh[i], Rl[g2][h], Rl[g2][h + 2]);
            mma_bf16(acc[0][s], Rl[i], Rh[g2][h], Rh[g2][h + 2]);
        }
        {
            const int i = W1::ti(s), n = W1::tn(s), g2 = n >> 1, h = n & 1;
            mma_bf16(acc[1][s], Rh[i], Rh[g2][h], Rh[g2][h + 2]);
            mma_bf16(acc[1][s], Rh[i], Rl[g2][h], Rl[g2][h + 2]);
            mma_bf16(acc[1][s], Rl[i], Rh[g2][h], Rh[g2][h + 2]);
        }
    }
    mma_bf16(gac[0], Rh[W0::GRAD], E[0], E[1]);
    mma_bf16(gac[0], Rh[W0::GRAD], E[2], E[3]);
    mma_bf16(gac[0], Rl[W0::GRAD], E[0], E[1]);
    mma_bf16(gac[1], Rh[W1::GRAD], E[0], E[1]);
    mma_bf16(gac[1], Rh[W1::GRAD], E[2], E[3]);
    mma_bf16(gac[1], Rl[W1::GRAD], E[0], E[1]);
}

// Tile list W's accumulators into the solve layout (entries on or below the
// diagonal, mirrored, so the system is exactly symmetric) or, for a chunk of a
// long row, into its slot (lower 8 x 8 tiles, diagonal tiles mirrored); the
// gradient into rhs (length 64).
template <int W, bool SLOT>
__device__ __forceinline__ void pbf_store(const float (&acc)[5][4], const float (&gac)[4], float *M, float *rhs,
                                          int lane) {
    using WT = CtaBfWarp<64, W>;
    const int r = lane >> 2, c2 = 2 * (lane & 3);
#pragma unroll
    for (int s = 0; s < CtaBfCfg<64>::NPT; ++s) {
        const int i = WT::ti(s), n = WT::tn(s);
#pragma unroll
        for (int hr = 0; hr < 2; ++hr)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int rr = 16 * i + r + 8 * hr, cc = 8 * n + c2 + e;
                const float v = acc[s][2 * hr + e];
                if (cc <= rr) {
                    if (SLOT) {
                        M[rr * 64 + cc] = v;
                        if (cc < rr && (cc >> 3) == (rr >> 3)) M[cc * 64 + rr] = v;
                    } else {
                        *p64_entry(M, rr, cc) = v;
                        if (cc < rr) *p64_entry(M, cc, rr) = v;
                    }
                }
            }
    }
    if ((lane & 3) == 0) {
        rhs[16 * WT::GRAD + r] = gac[0];
        rhs[16 * WT::GRAD + r + 8] = gac[2];
    }
}

template <bool PERM, bool HAS_A>
__global__ void __launch_bounds__(Pair64Bf::THREADS, 2) k_sparse_pair64_bf16(const StepArgs a) {
    using C = Pair64Bf;
    constexpr int B = 64, CH = C::CH, SBH = C::SBH, NPT = CtaBfCfg<64>::NPT;
    extern __shared__ float4 smem4[];
    const int pr = threadIdx.x >> 6, pt = threadIdx.x & 63, pw = pt >> 5, lane = pt & 31;
    const PairSmem<C> S(reinterpret_cast<float *>(smem4) + pr * C::FLOATS);
    if (pt == 0) S.flag[0] = atomicAdd(a.counter, 1);
    for (;;) {
        pair_sync(pr);
        const int tsk = S.flag[0];
        if (tsk >= a.n_tasks) break;
        pair_sync(pr);
        if (pt == 0) S.flag[0] = atomicAdd(a.counter, 1);
        const Task tk = a.tasks[tsk];
        const int nch = (tk.len + CH - 1) / CH;
        float acc[2][NPT][4], gac[2][4];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
#pragma unroll
            for (int t = 0; t < NPT; ++t)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[l][t][q] = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) gac[l][q] = 0.f;
        }
        if (tk.slot < 0) {  // alpha0 G_pipi + lambda_r I and the row term
            const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
            if (pw == 0) {
                cta_bf_init<64, 0>(acc[0], gac[0], a, tk.row, lam, lane);
                cta_bf_init<64, 1>(acc[1], gac[1], a, tk.row, lam, lane);
            } else {
                cta_bf_init<64, 2>(acc[0], gac[0], a, tk.row, lam, lane);
                cta_bf_init<64, 3>(acc[1], gac[1], a, tk.row, lam, lane);
            }
        }
        auto cnt_of = [&](int c) { return min(CH, tk.len - c * CH); };
        auto stage0 = [&](int i, int ib) {
            const int cnt = cnt_of(i);
            const int64_t s0 = tk.begin + (int64_t)i * CH;
            if (pt < cnt) cp_async4(S.ci + ib * CH + pt, a.idx + s0 + pt);
            if (PERM && pt >= 32 && pt - 32 < cnt) cp_async4(S.cq + ib * CH + pt - 32, a.pos + s0 + pt - 32);
        };
        auto gather = [&](int i, int sb, int ib) {  // hi and lo slices of chunk i
            const int cnt = cnt_of(i);
            const int *ids = S.ci + ib * CH;
            __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * C::STAGE), *tl = th + C::TILE;
            for (int f = pt; f < cnt * 16; f += 64) {
                const int k = f >> 4, v = f & 15, half = v >> 3, vc = v & 7;
                cp_async16((half ? tl : th) + k * SBH + vc * 8,
                           (half ? a.Fl : a.Fh) + (int64_t)ids[k] * a.d + a.p0 + vc * 8);
            }
        };
        auto stage1 = [&](int i, int sb, int ib) {
            const int cnt = cnt_of(i);
            __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * C::STAGE), *tl = th + C::TILE;
            const int rows16 = (cnt + 15) & ~15;  // rows cnt .. rows16 - 1 take part in the k-steps: zero
            for (int rr = cnt + pt; rr < rows16; rr += 64) {
#pragma unroll
                for (int v = 0; v < SBH / 8; ++v) {
                    reinterpret_cast<uint4 *>(th + rr * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                    reinterpret_cast<uint4 *>(tl + rr * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
            gather(i, sb, ib);
            if (pt < cnt) {
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + pt] : tk.begin + (int64_t)i * CH + pt;
                cp_async4(S.she + sb * CH + pt, a.e + q);
                if (HAS_A) cp_async4(S.sha + sb * CH + pt, a.alpha + q);
            }
        };
        auto body = [&](int j, int sb, int) {
            const int cnt = cnt_of(j);
            __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * C::STAGE), *tl = th + C::TILE;
            if (HAS_A) {  // weighted: row and residual times sqrt(alpha), split into hi / lo again
                const int k = pt >> 1, hf = pt & 1;
                if (k < cnt) {
                    const float sa = sqrtf(S.sha[sb * CH + k]);
#pragma unroll
                    for (int v = 4 * hf; v < 4 * hf + 4; ++v) {
                        uint4 hv = reinterpret_cast<uint4 *>(th + k * SBH)[v];
                        uint4 lv = reinterpret_cast<uint4 *>(tl + k * SBH)[v];
                        __nv_bfloat162 *h2 = reinterpret_cast<__nv_bfloat162 *>(&hv);
                        __nv_bfloat162 *l2 = reinterpret_cast<__nv_bfloat162 *>(&lv);
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const float2 hf2 = __bfloat1622float2(h2[q]), lf2 = __bfloat1622float2(l2[q]);
                            const float x0 = (hf2.x + lf2.x) * sa, x1 = (hf2.y + lf2.y) * sa;
                            const __nv_bfloat162 nh = __floats2bfloat162_rn(x0, x1);
                            const float2 nhf = __bfloat1622float2(nh);
                            h2[q] = nh;
                            l2[q] = __floats2bfloat162_rn(x0 - nhf.x, x1 - nhf.y);
                        }
                        reinterpret_cast<uint4 *>(th + k * SBH)[v] = hv;
                        reinterpret_cast<uint4 *>(tl + k * SBH)[v] = lv;
                    }
                    if (hf == 0) {
                        const float e = S.she[sb * CH + k] * sa;
                        const __nv_bfloat16 h = __float2bfloat16_rn(e);
                        th[k * SBH + B] = h;
                        tl[k * SBH + B] = __float2bfloat16_rn(e - __bfloat162float(h));
                    }
                }
            } else if (pt < cnt) {  // the residual column, hi / lo
                const float e = S.she[sb * CH + pt];
                const __nv_bfloat16 h = __float2bfloat16_rn(e);
                th[pt * SBH + B] = h;
                tl[pt * SBH + B] = __float2bfloat16_rn(e - __bfloat162float(h));
            }
            pair_sync(pr);
            const int ksteps = (cnt + 15) >> 4;
            for (int ks = 0; ks < ksteps; ++ks) {
                if (pw == 0) pbf_kstep<0>(acc, gac, th, tl, ks, lane);
                else pbf_kstep<1>(acc, gac, th, tl, ks, lane);
            }
        };
        p64_pipeline(pr, nch, stage0, stage1, body);
        if (tk.slot >= 0) {  // chunk of a long row: its statistics to the slot
            float *Pp = a.part + (int64_t)tk.slot * (B * B + B);
            if (pw == 0) {
                pbf_store<0, true>(acc[0], gac[0], Pp, Pp + B * B, lane);
                pbf_store<1, true>(acc[1], gac[1], Pp, Pp + B * B, lane);
            } else {
                pbf_store<2, true>(acc[0], gac[0], Pp, Pp + B * B, lane);
                pbf_store<3, true>(acc[1], gac[1], Pp, Pp + B * B, lane);
            }
            continue;
        }
        float *M = S.stage;
        if (pw == 0) {
            pbf_store<0, false>(acc[0], gac[0], M, S.dl, lane);
            pbf_store<1, false>(acc[1], gac[1], M, S.dl, lane);
        } else {
            pbf_store<2, false>(acc[0], gac[0], M, S.dl, lane);
            pbf_store<3, false>(acc[1], gac[1], M, S.dl, lane);
        }
        pair_sync(pr);
        const int rq = pt >> 1, chh = pt & 1;
        float A[2][32], gr[2], x[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int r = 2 * rq + t;
#pragma unroll
            for (int q4 = 0; q4 < 8; ++q4) {
                const float4 u = p64_ld4(M + p64_at(r, chh, q4));
                A[t][4 * q4] = u.x; A[t][4 * q4 + 1] = u.y; A[t][4 * q4 + 2] = u.z; A[t][4 * q4 + 3] = u.w;
            }
            gr[t] = S.dl[r];
        }
        const float dorig = *p64_entry(M, 2 * rq + chh, 2 * rq + chh);
        const int vote = p64_gj(A, gr, dorig, S.gjb, pr, pt, a.force_fp64 != 0, x);
        if (vote) {
            if (pt == 0) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tk.row;
            }
            continue;
        }
        if (chh == 0) {
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                apply_delta(a.X, a.Xh, a.Xl, (int64_t)tk.row * a.d + a.p0 + 2 * rq + t, x[t]);
                S.dl[2 * rq + t] = x[t];
            }
        }
        // residual update from the re-gathered hi + lo slices: two threads per
        // interaction, 16-byte chunks u + 4 part of the row
        const int k = pt >> 1, part = pt & 1;
        auto rbody = [&](int j, int sb, int ib) {
            const int cnt = cnt_of(j);
            const __nv_bfloat16 *th = reinterpret_cast<const __nv_bfloat16 *>(S.stage + sb * C::STAGE);
            const __nv_bfloat16 *tl = th + C::TILE;
            float t = 0.f;
            if (k < cnt) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int c8 = u + 4 * part;
                    const uint4 hv = *reinterpret_cast<const uint4 *>(th + k * SBH + 8 * c8);
                    const uint4 lv = *reinterpret_cast<const uint4 *>(tl + k * SBH + 8 * c8);
                    const float4 w0 = p64_ld4(S.dl + 8 * c8), w1 = p64_ld4(S.dl + 8 * c8 + 4);
                    const float w[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                    const __nv_bfloat162 *h2 = reinterpret_cast<const __nv_bfloat162 *>(&hv);
                    const __nv_bfloat162 *l2 = reinterpret_cast<const __nv_bfloat162 *>(&lv);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float2 hf2 = __bfloat1622float2(h2[q]), lf2 = __bfloat1622float2(l2[q]);
                        t = fmaf(w[2 * q], hf2.x + lf2.x, t);
                        t = fmaf(w[2 * q + 1], hf2.y + lf2.y, t);
                    }
                }
            }
            t += __shfl_xor_sync(kFull, t, 1);
            if (k < cnt && part == 0) {
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + k] : tk.begin + (int64_t)j * CH + k;
                a.e[q] -= t;
            }
        };
        p64_pipeline(pr, nch, stage0, gather, rbody);
    }
}

template <bool PERM, bool HAS_A>
cudaError_t launch_sparse_pair64_bf16_all(const StepArgs &a, cudaStream_t s) {
    using C = Pair64Bf;
    using CF = CtaCfg<64>;
    static bool attr_done = false;
    static int per_sm = 0;
    auto kern = k_sparse_pair64_bf16<PERM, HAS_A>;
    if (!attr_done) {
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_split_solve_rc<64, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      RcCfg<64>::SMEM_BYTES)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_retry_cta<64, PERM, HAS_A, false>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, retry_cta_smem<64>())) != cudaSuccess)
            return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C::THREADS, C::SMEM_BYTES)) != cudaSuccess)
            return e;
        if (per_sm < 1) per_sm = 1;
        attr_done = true;
    }
    if (a.n_tasks > 0) {
        int grid = 152 * per_sm;
        const int need = (a.n_tasks + C::PAIRS - 1) / C::PAIRS;
        if (grid > need) grid = need;
        prof_mark(a.prof, K_SPARSE, s);
        kern<<<grid, C::THREADS, C::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    if (a.n_split > 0) {
        const int g2 = a.n_split < 152 * 4 ? a.n_split : 152 * 4;
        prof_mark(a.prof, K_SPLIT_SOLVE, s);
        k_split_solve_rc<64, false><<<g2, RcCfg<64>::THREADS, RcCfg<64>::SMEM_BYTES, s>>>(a);
        prof_mark(a.prof, -1, s);
    }
    {
        const cudaError_t e = launch_split_resid_reg_bf16<64, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry_cta<64, PERM, HAS_A, false><<<kRetryBlocks, CF::THREADS, retry_cta_smem<64>(), s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

}  // namespace ials
