// Block step of Algorithm 3 at block size b = 64, FP32 and BF16 statistics,
// with the row systems solved one per warp.
//
// A CTA of four warps takes four tasks at a time.  All threads accumulate the
// statistics of the four tasks in turn (Eqs. 11-12): FP32 as 8 x 8 register
// tiles (three interaction groups of 36 tile owners, summed in group order),
// BF16 as compensated hi/lo mma.sync tiles (the tile lists of
// k_sparse_cta_bf16.cuh); each result goes to one of four shared 64 x 64
// systems, both triangles, with the right-hand side as row 64.  Then every
// warp solves one system in registers (Eq. 9): lane l holds rows l and l + 32
// and runs the Gauss-Jordan elimination with 2 x 2 pivot blocks of
// k_sparse_impl.cuh, which needs only warp-level synchronisation, so the four
// solves proceed independently and every lane works at every step.  Finally
// the four rows are applied and their residuals updated (Eq. 7).
//
// The gathers are what the step waits for, so the batch's chunks (32
// interactions each) run through one software pipeline: the column ids and
// positions of chunk j + 4 and the slices and residuals of chunk j + 2 are in
// flight (cp.async) while chunk j is multiplied; the residual update runs the
// same pipeline over the solved rows' chunks.
#pragma once

#include "k_sparse_cta_bf16.cuh"
#include "k_sparse_rc.cuh"

namespace ials {

struct Gj64 {
    static constexpr int B = 64, R = 4, WARPS = 8, THREADS = 256;
    static constexpr int NTL = 36, NG = 3;              // FP32 statistics: tiles x groups
    static constexpr int SB = B + 4, CH = 32, BUF = CH * SB;
    static constexpr int P = 2;                         // slices of chunk j + P in flight at chunk j
    static constexpr int NS = P + 1, NI = 2 * P + 1;    // slice stages; id / position stages
    // one slice stage: FP32 rows, or BF16 hi and lo tiles (CtaBfCfg<64>::BUF bf16 = half as many floats)
    static constexpr int STAGE = BUF > CtaBfCfg<64>::BUF / 2 ? BUF : CtaBfCfg<64>::BUF / 2;
    static constexpr int MSZ = (B + 1) * SB;            // one system: 64 rows + right-hand side
    static constexpr int CB = B + 4;                    // solver column buffer: 64 entries, g, pad
    static constexpr int CBW = 4 * CB;                  // per system: two steps x two columns
    // floats: slice stages, e and alpha per stage, ids and positions per id stage,
    // systems, solver buffers, deltas, flags
    static constexpr int SMEM_FLOATS = NS * STAGE + 2 * NS * CH + 2 * NI * CH + R * MSZ + R * CBW + R * B + 16;
    static constexpr int SMEM_BYTES = SMEM_FLOATS * 4;
};

template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}

// The chunks of a batch: rows r < nr taken (use[r]), max(1, ceil(len / CH))
// chunks each (an empty row has one empty chunk), in row order.
struct ChunkSeq {
    int start[Gj64::R + 1];
    __device__ __forceinline__ void init(const Task *tks, int nr, const bool (&use)[Gj64::R]) {
        start[0] = 0;
#pragma unroll
        for (int r = 0; r < Gj64::R; ++r) {
            const int n = (r < nr && use[r]) ? max(1, (tks[r].len + Gj64::CH - 1) / Gj64::CH) : 0;
            start[r + 1] = start[r] + n;
        }
    }
    __device__ __forceinline__ int total() const { return start[Gj64::R]; }
    // row r and chunk c of chunk i; last = whether it is row r's last chunk
    __device__ __forceinline__ void locate(int i, int &r, int &c, bool &last) const {
        r = 0;
        int s0 = 0, s1 = start[1];
#pragma unroll
        for (int q = 1; q < Gj64::R; ++q)
            if (i >= start[q]) {
                r = q;
                s0 = start[q];
                s1 = start[q + 1];
            }
        c = i - s0;
        last = i + 1 == s1;
    }
};

// Software pipeline over `total` chunks.  stage0(i, ib): cp.async of chunk i's
// column ids / positions into id stage ib; stage1(i, sb, ib): the gathers of
// chunk i (reading its ids from id stage ib) into slice stage sb; body(j, sb, ib):
// the work on chunk j.  Every iteration commits one cp.async group, so waiting
// for all but the last P - 1 groups leaves chunk j's slices (and chunk j + P's
// ids) complete.  All threads call it.
template <typename S0, typename S1, typename Body>
__device__ __forceinline__ void gj64_pipeline(int total, S0 stage0, S1 stage1, Body body) {
    constexpr int P = Gj64::P, NS = Gj64::NS, NI = Gj64::NI;
    for (int i = 0; i < 2 * P && i < total; ++i) stage0(i, i % NI);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    for (int i = 0; i < P; ++i) {
        if (i < total) stage1(i, i % NS, i % NI);
        cp_async_commit();
    }
#pragma unroll 1
    for (int j = 0; j < total; ++j) {
        cp_async_wait_group<P - 1>();
        __syncthreads();
        const int n1 = j + P, n0 = j + 2 * P;
        if (n1 < total) stage1(n1, n1 % NS, n1 % NI);
        if (n0 < total) stage0(n0, n0 % NI);
        cp_async_commit();
        body(j, j % NS, j % NI);
    }
    cp_async_wait_all();
    __syncthreads();
}

// Barrier of the two warps (64 threads) that solve system `sys` (ids 1 .. R;
// id 0 is __syncthreads).
__device__ __forceinline__ void pair_sync(int sys) {
    asm volatile("bar.sync %0, 64;\n" ::"r"(sys + 1) : "memory");
}

// Gauss-Jordan solve of one 64 x 64 SPD system by two warps: lane l of warp
// half h holds row 32 h + l (both triangles) in A and its right-hand side in g.
// Step m eliminates the columns k = 2m, k + 1 with the 2 x 2 pivot block P =
// [[a, b], [b, c]] (a principal Schur complement, SPD): every row publishes its
// entries in columns k, k + 1 (by symmetry of the trailing block, the pivot
// rows' trailing entries), the pivot rows their right-hand sides; every other
// row then eliminates with [s1, s2] = [A[row][k], A[row][k+1]] P^{-1},
//   A[row][j] -= s1 A[k][j] + s2 A[k+1][j] (j > k + 1),  g_row -= s1 g_k + s2 g_{k+1}.
// At the end the system is block diagonal and each pivot pair solves its 2 x 2
// block (the partner row is the neighbouring lane).  The published columns are
// double-buffered in cb (4 x CB floats, 16-byte aligned) so one barrier of the
// pair per step suffices.  Pivots of A = L D L^T are checked against the
// original diagonal (not below 1e-5 of it, finite).  `vote` (2 ints) collects
// the two warps' verdicts.  Returns false (uniform over the pair) on a bad pivot
// or a non-finite solution; else x holds solution entry 32 h + l.
__device__ __forceinline__ bool gj_solve64_pair(float (&A)[64], float g, float *cb, int *vote, int sys, int h,
                                                int lane, bool force_fail, float &x) {
    constexpr int B = 64, CB = Gj64::CB;
    const int row = 32 * h + lane;
    float dorig = 0.f;
#pragma unroll
    for (int j = 0; j < B; ++j)
        if (j == row) dorig = A[j];
    bool bad = force_fail;
    float pa = 1.f, pb = 0.f, pc = 1.f;
#pragma unroll
    for (int k = 0; k < B; k += 2) {
        float *v1 = cb + ((k >> 1) & 1) * 2 * CB, *v2 = v1 + CB;
        v1[row] = A[k];
        v2[row] = A[k + 1];
        if (row == k) v1[B] = g;
        if (row == k + 1) v2[B] = g;
        pair_sync(sys);
        const float a = v1[k], b = v1[k + 1], c = v2[k + 1];
        const float gk = v1[B], gk1 = v2[B];
        const float rdet = rcp_approx(a * c - b * b);
        const bool piv = row == k || row == k + 1;
        const float xk = A[k], yk = A[k + 1];
        const float s1 = piv ? 0.f : (xk * c - yk * b) * rdet;
        const float s2 = piv ? 0.f : (yk * a - xk * b) * rdet;
        if (row == k) bad = bad || !(a > 1e-5f * dorig) || !(a <= 3.0e38f);
        if (row == k + 1) {
            const float d1 = c - b * b * rcp_approx(a);
            bad = bad || !(d1 > 1e-5f * dorig) || !(d1 <= 3.0e38f);
        }
        if (piv) {
            pa = a;
            pb = b;
            pc = c;
        }
#pragma unroll
        for (int j0 = (k + 2) & ~3; j0 < B; j0 += 4) {
            const float4 q1 = *reinterpret_cast<const float4 *>(v1 + j0);
            const float4 q2 = *reinterpret_cast<const float4 *>(v2 + j0);
            if (j0 > k + 1) {
                fma2(A[j0], A[j0 + 1], -s1, -s1, q1.x, q1.y);
                fma2(A[j0], A[j0 + 1], -s2, -s2, q2.x, q2.y);
            }
            fma2(A[j0 + 2], A[j0 + 3], -s1, -s1, q1.z, q1.w);
            fma2(A[j0 + 2], A[j0 + 3], -s2, -s2, q2.z, q2.w);
        }
        g -= s1 * gk + s2 * gk1;
    }
    const float gp = __shfl_xor_sync(kFull, g, 1);
    const float rd = rcp_approx(pa * pc - pb * pb);
    x = (lane & 1) ? (pa * g - pb * gp) * rd : (pc * g - pb * gp) * rd;
    const bool fail = __any_sync(kFull, bad || !isfinite(x));
    if (lane == 0) vote[h] = fail ? 1 : 0;
    pair_sync(sys);
    return !(vote[0] | vote[1]);
}

// Chunk of a long row: the (lower tiles of the) summed statistics to its slot.
__device__ __forceinline__ void gj64_store_slot(const StepArgs &a, const Task &tk, const float *Mr) {
    constexpr int B = 64, SB = Gj64::SB;
    float *P = a.part + (int64_t)tk.slot * (B * B + B);
    for (int e = threadIdx.x; e < B * B; e += blockDim.x) {
        const int i = e / B, j = e % B;
        if ((j >> 3) <= (i >> 3)) P[e] = Mr[i * SB + j];
    }
    for (int j = threadIdx.x; j < B; j += blockDim.x) P[B * B + j] = Mr[B * SB + j];
}

// Shared-memory layout of the b = 64 kernels.
struct Gj64Smem {
    float *stage, *she, *sha, *M, *cbase, *dl;
    int *ci, *cq, *flag;
    __device__ __forceinline__ Gj64Smem(float *smem) {
        using C = Gj64;
        stage = smem;
        she = stage + C::NS * C::STAGE;
        sha = she + C::NS * C::CH;
        ci = reinterpret_cast<int *>(sha + C::NS * C::CH);
        cq = ci + C::NI * C::CH;
        M = reinterpret_cast<float *>(cq + C::NI * C::CH);
        cbase = M + C::R * C::MSZ;
        dl = cbase + C::R * C::CBW;  // one solver buffer per system
        flag = reinterpret_cast<int *>(dl + C::R * C::B);  // [0] next batch, [1..4] solved
    }
};

// cp.async of the column ids (and, on the item side, residual positions) of
// `cnt` interactions from CSR position s0 into id stage ib.
template <bool PERM>
__device__ __forceinline__ void gj64_ids(const StepArgs &a, const Gj64Smem &S, int64_t s0, int cnt, int ib) {
    const int tid = threadIdx.x;
    if (tid < cnt) cp_async4(S.ci + ib * Gj64::CH + tid, a.idx + s0 + tid);
    if (PERM && tid >= 32 && tid - 32 < cnt) cp_async4(S.cq + ib * Gj64::CH + tid - 32, a.pos + s0 + tid - 32);
}

// Slice gathers of `cnt` interactions (ids from id stage ib) into slice stage sb.
template <bool BF>
__device__ __forceinline__ void gj64_slices(const StepArgs &a, const Gj64Smem &S, int cnt, int sb, int ib) {
    constexpr int B = 64;
    const int *ids = S.ci + ib * Gj64::CH;
    if (BF) {
        using CBf = CtaBfCfg<64>;
        constexpr int HC = B / 8;
        __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * Gj64::STAGE), *tl = th + CBf::TILE;
        for (int f = threadIdx.x; f < cnt * 2 * HC; f += blockDim.x) {
            const int k = f / (2 * HC), v = f % (2 * HC), half = v / HC, vc = v % HC;
            const int64_t c = ids[k];
            cp_async16((half ? tl : th) + k * CBf::SBH + vc * 8, (half ? a.Fl : a.Fh) + c * a.d + a.p0 + vc * 8);
        }
    } else {
        constexpr int V = B / 4;
        float *buf = S.stage + sb * Gj64::STAGE;
        for (int f = threadIdx.x; f < cnt * V; f += blockDim.x) {
            const int k = f / V, v = f % V;
            const int64_t c = ids[k];
            cp_async16(buf + k * Gj64::SB + 4 * v, a.F + c * a.d + a.p0 + 4 * v);
        }
    }
}

// Residual update of the solved rows of the batch, pipelined over their chunks:
// four threads per interaction, each a quarter of the slice (FP32) or of the hi
// and lo slices (BF16), e_s -= <delta, f_{c_s,pi}>.
template <bool PERM, bool BF>
__device__ __forceinline__ void gj64_residuals(const StepArgs &a, const Gj64Smem &S, const Task *tks, int nr,
                                               const bool (&use)[Gj64::R]) {
    constexpr int CH = Gj64::CH;
    using CBf = CtaBfCfg<64>;
    ChunkSeq seq;
    seq.init(tks, nr, use);
    // eight threads per interaction; thread part p takes the float4 groups p and p + 8
    // of the slice (conflict-free shared loads)
    const int tid = threadIdx.x, k = tid >> 3, part = tid & 7;
    auto cnt_of = [&](int i, int &r, int &c) {
        bool last;
        seq.locate(i, r, c, last);
        return max(0, min(CH, tks[r].len - c * CH));
    };
    auto stage0 = [&](int i, int ib) {
        int r, c;
        const int cnt = cnt_of(i, r, c);
        gj64_ids<PERM>(a, S, tks[r].begin + (int64_t)c * CH, cnt, ib);
    };
    auto stage1 = [&](int i, int sb, int ib) {
        int r, c;
        gj64_slices<BF>(a, S, cnt_of(i, r, c), sb, ib);
    };
    auto body = [&](int j, int sb, int ib) {
        int r, c;
        const int cnt = cnt_of(j, r, c);
        const float *x = S.dl + r * Gj64::B;
        float t = 0.f;
        if (k < cnt) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int o = 4 * (part + 8 * u);
                const float4 w = *reinterpret_cast<const float4 *>(x + o);
                float v[4];
                if (BF) {
                    const __nv_bfloat16 *hr = reinterpret_cast<const __nv_bfloat16 *>(S.stage + sb * Gj64::STAGE) +
                                              k * CBf::SBH + o;
                    const __nv_bfloat16 *lr = hr + CBf::TILE;
#pragma unroll
                    for (int q = 0; q < 4; ++q) v[q] = __bfloat162float(hr[q]) + __bfloat162float(lr[q]);
                } else {
                    const float4 f = *reinterpret_cast<const float4 *>(S.stage + sb * Gj64::STAGE + k * Gj64::SB + o);
                    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
                }
                t = fmaf(w.x, v[0], t);
                t = fmaf(w.y, v[1], t);
                t = fmaf(w.z, v[2], t);
                t = fmaf(w.w, v[3], t);
            }
        }
        t += __shfl_xor_sync(kFull, t, 1);
        t += __shfl_xor_sync(kFull, t, 2);
        t += __shfl_xor_sync(kFull, t, 4);
        if (k < cnt && part == 0) {
            const int64_t q = PERM ? (int64_t)S.cq[ib * CH + k] : tks[r].begin + (int64_t)c * CH + k;
            a.e[q] -= t;
        }
    };
    gj64_pipeline(seq.total(), stage0, stage1, body);
}

// Solve of the batch (one system per pair of warps), then apply and residual
// update of each solved row.
template <bool PERM, bool BF>
__device__ __forceinline__ void gj64_finish(const StepArgs &a, const Gj64Smem &S, const Task *tks, int nr) {
    constexpr int B = 64, SB = Gj64::SB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int sys = warp >> 1, h = warp & 1, row = 32 * h + lane;
    int *ok = S.flag + 1, *vote = S.flag + 8 + 2 * sys;
    if (sys < nr && tks[sys].slot < 0) {
        const float *Mr = S.M + sys * Gj64::MSZ;
        float A[64];
#pragma unroll
        for (int j = 0; j < B; j += 4) {
            const float4 u = *reinterpret_cast<const float4 *>(Mr + row * SB + j);
            A[j] = u.x; A[j + 1] = u.y; A[j + 2] = u.z; A[j + 3] = u.w;
        }
        float x;
        const bool good = gj_solve64_pair(A, Mr[B * SB + row], S.cbase + sys * Gj64::CBW, vote, sys, h, lane,
                                          a.force_fp64 != 0, x);
        if (good) S.dl[sys * B + row] = x;
        if (tid == 64 * sys) {
            ok[sys] = good ? 1 : 0;
            if (!good) {
                const int i = atomicAdd(a.retry, 1);
                a.retry[1 + i] = tks[sys].row;
            }
        }
    }
    __syncthreads();
    bool use[Gj64::R];
#pragma unroll
    for (int r = 0; r < Gj64::R; ++r) use[r] = r < nr && tks[r].slot < 0 && ok[r];
#pragma unroll
    for (int r = 0; r < Gj64::R; ++r)
        if (use[r])
            for (int j = tid; j < B; j += blockDim.x)
                apply_delta(a.X, a.Xh, a.Xl, (int64_t)tks[r].row * a.d + a.p0 + j, S.dl[r * B + j]);
    gj64_residuals<PERM, BF>(a, S, tks, nr, use);
}

template <bool PERM, bool HAS_A>
__global__ void __launch_bounds__(Gj64::THREADS, 1) k_sparse_gj64(const StepArgs a) {
    using C = Gj64;
    constexpr int B = 64, SB = C::SB, CH = C::CH, NTL = C::NTL, NG = C::NG;
    extern __shared__ float4 smem4[];
    const Gj64Smem S(reinterpret_cast<float *>(smem4));
    __shared__ Task tks[C::R];
    const int tid = threadIdx.x;
    const bool active = tid < NTL * NG;
    const int grp = active ? tid / NTL : NG;
    const int kstart = active ? grp : CH;
    int ti = 0, tj = 0;
    tri_index(tid % NTL, ti, tj);
    if (tid == 0) S.flag[0] = atomicAdd(a.counter, C::R);
    for (;;) {
        __syncthreads();
        const int base = S.flag[0];
        if (base >= a.n_tasks) break;
        const int nr = min(C::R, a.n_tasks - base);
        if (tid < nr) tks[tid] = a.tasks[base + tid];
        __syncthreads();  // every thread has read flag[0]; tks is set
        if (tid == 0) S.flag[0] = atomicAdd(a.counter, C::R);
        bool all[C::R];
#pragma unroll
        for (int r = 0; r < C::R; ++r) all[r] = true;
        ChunkSeq seq;
        seq.init(tks, nr, all);
        float t[8][8], g[8];
        auto cnt_of = [&](int i, int &r, int &c) {
            bool last;
            seq.locate(i, r, c, last);
            return max(0, min(CH, tks[r].len - c * CH));
        };
        auto stage0 = [&](int i, int ib) {
            int r, c;
            const int cnt = cnt_of(i, r, c);
            gj64_ids<PERM>(a, S, tks[r].begin + (int64_t)c * CH, cnt, ib);
        };
        auto stage1 = [&](int i, int sb, int ib) {
            int r, c;
            const int cnt = cnt_of(i, r, c);
            gj64_slices<false>(a, S, cnt, sb, ib);
            if (tid < cnt) {  // residual (and weight) of each interaction
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + tid] : tks[r].begin + (int64_t)c * CH + tid;
                cp_async4(S.she + sb * CH + tid, a.e + q);
                if (HAS_A) cp_async4(S.sha + sb * CH + tid, a.alpha + q);
            }
        };
        auto body = [&](int j, int sb, int ib) {
            int r, c;
            bool last;
            seq.locate(j, r, c, last);
            const int cnt = max(0, min(CH, tks[r].len - c * CH));
            const Task &tk = tks[r];
            if (c == 0) {  // first chunk of row r: the dense terms (whole rows, group 0) or zero
                const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
                if (tk.slot < 0 && grp == 0) {
                    rc_dense_init<B, false>(a, ti, tj, tk.row, lam, t, g);
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        g[i] = 0.f;
#pragma unroll
                        for (int q = 0; q < 8; ++q) t[i][q] = 0.f;
                    }
                }
            }
            const float *bp = S.stage + sb * C::STAGE;
            const float *se = S.she + sb * CH, *sa = S.sha + sb * CH;
            for (int k = kstart; k < cnt; k += NG) {
                const float *xk = bp + k * SB;
                float xa[8], xb[8];
                load_seg<8>(xk + 8 * ti, xa);
                load_seg<8>(xk + 8 * tj, xb);
                float ek = se[k];
                if (HAS_A) {
                    const float ak = sa[k];
                    ek *= ak;
#pragma unroll
                    for (int i = 0; i < 8; ++i) g[i] = fmaf(ek, xa[i], g[i]);
#pragma unroll
                    for (int i = 0; i < 8; ++i) xa[i] *= ak;
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) g[i] = fmaf(ek, xa[i], g[i]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int q = 0; q < 8; q += 2) fma2(t[i][q], t[i][q + 1], xa[i], xa[i], xb[q], xb[q + 1]);
            }
            if (!last) return;  // more chunks of row r follow
            // last chunk of row r: group partials summed in group order into system r,
            // both triangles (mirrored, so exactly symmetric); gradient blocks into row 64
            float *Mr = S.M + r * C::MSZ;
            if (ti == tj) {  // a diagonal tile takes its lower triangle on both sides
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int q = i + 1; q < 8; ++q) t[i][q] = t[q][i];
            }
#pragma unroll 1
            for (int ph = 0; ph < NG; ++ph) {
                __syncthreads();
                if (active && grp == ph) {
                    // rows of the tile, then (off the diagonal) rows of its transpose; every
                    // entry and its mirror receive the same sums in the same order
#pragma unroll
                    for (int i = 0; i < 8; ++i) store_tile<8>(Mr + (8 * ti + i) * SB + 8 * tj, t[i], ph > 0);
                    if (ti != tj) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            float col[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) col[i] = t[i][q];
                            store_tile<8>(Mr + (8 * tj + q) * SB + 8 * ti, col, ph > 0);
                        }
                    }
                    if (tj == 0) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            float *p = Mr + B * SB + 8 * ti + i;
                            *p = ph ? *p + g[i] : g[i];
                        }
                    }
                }
            }
            __syncthreads();
            if (tk.slot >= 0) gj64_store_slot(a, tk, Mr);
        };
        gj64_pipeline(seq.total(), stage0, stage1, body);
        gj64_finish<PERM, false>(a, S, tks, nr);
    }
}

// BF16 statistics (compensated hi/lo mma.sync, the warp tile lists of
// k_sparse_cta_bf16.cuh) with the batched warp solves.  The residuals arrive
// as floats and are split into the hi / lo residual column of the staged tile
// before the products.
template <bool PERM, bool HAS_A>
__global__ void __launch_bounds__(Gj64::THREADS, 2) k_sparse_gj64_bf16(const StepArgs a) {
    using C = Gj64;
    using CBf = CtaBfCfg<64>;
    constexpr int B = 64, CH = C::CH, SBH = CBf::SBH, NPT = CBf::NPT;
    extern __shared__ float4 smem4[];
    const Gj64Smem S(reinterpret_cast<float *>(smem4));
    __shared__ Task tks[C::R];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
    for (int i = tid; i < C::NS * C::STAGE / 4; i += nt)
        reinterpret_cast<float4 *>(S.stage)[i] = make_float4(0.f, 0.f, 0.f, 0.f);  // padding columns stay zero
    if (tid == 0) S.flag[0] = atomicAdd(a.counter, C::R);
    for (;;) {
        __syncthreads();
        const int base = S.flag[0];
        if (base >= a.n_tasks) break;
        const int nr = min(C::R, a.n_tasks - base);
        if (tid < nr) tks[tid] = a.tasks[base + tid];
        __syncthreads();
        if (tid == 0) S.flag[0] = atomicAdd(a.counter, C::R);
        bool all[C::R];
#pragma unroll
        for (int r = 0; r < C::R; ++r) all[r] = true;
        ChunkSeq seq;
        seq.init(tks, nr, all);
        float acc[NPT][4], gac[4];
        auto cnt_of = [&](int i, int &r, int &c) {
            bool last;
            seq.locate(i, r, c, last);
            return max(0, min(CH, tks[r].len - c * CH));
        };
        auto stage0 = [&](int i, int ib) {
            int r, c;
            const int cnt = cnt_of(i, r, c);
            gj64_ids<PERM>(a, S, tks[r].begin + (int64_t)c * CH, cnt, ib);
        };
        auto stage1 = [&](int i, int sb, int ib) {
            int r, c;
            const int cnt = cnt_of(i, r, c);
            __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * C::STAGE), *tl = th + CBf::TILE;
            // rows cnt .. next multiple of 16 stay zero (the tile products run over whole 16-row steps)
            const int rows16 = (cnt + 15) & ~15;
            for (int rr = cnt + tid; rr < rows16; rr += nt) {
#pragma unroll
                for (int v = 0; v < SBH / 8; ++v) {
                    reinterpret_cast<uint4 *>(th + rr * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                    reinterpret_cast<uint4 *>(tl + rr * SBH)[v] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
            gj64_slices<true>(a, S, cnt, sb, ib);
            if (tid < cnt) {
                const int64_t q = PERM ? (int64_t)S.cq[ib * CH + tid] : tks[r].begin + (int64_t)c * CH + tid;
                cp_async4(S.she + sb * CH + tid, a.e + q);
                if (HAS_A) cp_async4(S.sha + sb * CH + tid, a.alpha + q);
            }
        };
        auto body = [&](int j, int sb, int ib) {
            int r, c;
            bool last;
            seq.locate(j, r, c, last);
            const int cnt = max(0, min(CH, tks[r].len - c * CH));
            const Task &tk = tks[r];
            if (c == 0) {
#pragma unroll
                for (int s = 0; s < NPT; ++s)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[s][q] = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q) gac[q] = 0.f;
                const float lam = a.lambda * (1.0f + a.nu * (float)tk.len);
                if (tk.slot < 0 && warp < CBf::WARPS) cta_bf_init_any<B>(warp, acc, gac, a, tk.row, lam, lane);
            }
            __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(S.stage + sb * C::STAGE), *tl = th + CBf::TILE;
            if (tid < cnt) {  // residual column: hi / lo split (weighted: row and residual times sqrt(alpha))
                float e = S.she[sb * CH + tid];
                if (HAS_A) {
                    const float sa = sqrtf(S.sha[sb * CH + tid]);
                    e *= sa;
#pragma unroll
                    for (int v = 0; v < B / 8; ++v) {
                        uint4 hv = reinterpret_cast<uint4 *>(th + tid * SBH)[v];
                        uint4 lv = reinterpret_cast<uint4 *>(tl + tid * SBH)[v];
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
                        reinterpret_cast<uint4 *>(th + tid * SBH)[v] = hv;
                        reinterpret_cast<uint4 *>(tl + tid * SBH)[v] = lv;
                    }
                }
                const __nv_bfloat16 h = __float2bfloat16_rn(e);
                th[tid * SBH + B] = h;
                tl[tid * SBH + B] = __float2bfloat16_rn(e - __bfloat162float(h));
            }
            __syncthreads();
            const int ksteps = (cnt + 15) >> 4;
            if (warp < CBf::WARPS)  // the tile lists cover four warps; the others wait
                for (int ks = 0; ks < ksteps; ++ks) cta_bf_kstep_any<B>(warp, acc, gac, th, tl, ks, lane);
            if (!last) return;
            float *Mr = S.M + r * C::MSZ;
            __syncthreads();
            if (warp < CBf::WARPS) cta_bf_store_any<B>(warp, acc, gac, Mr, lane);
            __syncthreads();
            // the upper triangle from the lower one (exactly symmetric)
            for (int e = tid; e < B * B; e += nt) {
                const int i = e / B, q = e % B;
                if (q > i) Mr[i * C::SB + q] = Mr[q * C::SB + i];
            }
            __syncthreads();
            if (tk.slot >= 0) gj64_store_slot(a, tk, Mr);
        };
        gj64_pipeline(seq.total(), stage0, stage1, body);
        gj64_finish<PERM, true>(a, S, tks, nr);
    }
}

template <bool PERM, bool HAS_A, bool BF>
cudaError_t launch_sparse_gj64_all(const StepArgs &a, cudaStream_t s) {
    using C = Gj64;
    using CF = CtaCfg<64>;
    static bool attr_done = false;
    static int per_sm = 0;
    auto kern = BF ? (void (*)(const StepArgs))k_sparse_gj64_bf16<PERM, HAS_A> : (void (*)(const StepArgs))k_sparse_gj64<PERM, HAS_A>;
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
        const int batches = (a.n_tasks + C::R - 1) / C::R;
        if (grid > batches) grid = batches;
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
        const cudaError_t e = BF ? launch_split_resid_reg_bf16<64, PERM>(a, s) : launch_split_resid_reg<64, PERM>(a, s);
        if (e != cudaSuccess) return e;
    }
    prof_mark(a.prof, K_RETRY, s);
    k_retry_cta<64, PERM, HAS_A, false><<<kRetryBlocks, CF::THREADS, retry_cta_smem<64>(), s>>>(a);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

}  // namespace ials
