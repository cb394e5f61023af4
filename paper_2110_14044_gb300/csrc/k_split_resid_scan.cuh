// Residual update of the item side's split rows (Eq. 7) in user-major order.
//
// After the split-row solve of an item step, every interaction (u, c) of a split
// item row c needs e_q -= <delta_c, w_{u,pi}>, q being its position in the
// user-major residual array.  Visiting them row by row (item-major) reaches the
// residuals through the position map, one 32-byte sector per 4-byte residual,
// and gathers one user slice per interaction.  Here they are visited in
// user-major order instead: split_pos lists the positions whose item is a split
// row, in increasing order, and split_row the split row of each.  Each warp takes
// a contiguous piece of the list, lane i on entry k0 + i, so the residual reads
// and writes of a warp fall in a few sectors, and the lanes that share a user
// read the same slice.  The deltas of all split rows of the step sit in shared
// memory, rows of B floats; lane l reads the 16-byte pieces of its row starting
// at piece l (rotated), so that the eight lanes of a quarter warp meet eight
// different bank groups whatever rows they read (B >= 32; for the BF16 slices
// the two pieces of each group of eight features are read in opposite orders by
// the two halves of a quarter warp, to the same end).
//
// A lane finds the user of its position by counting user boundaries: the warp
// holds a user `base` at or before every position still to come and the next 32
// boundaries optr[base + 1 .. base + 32], one per lane; each lane counts those at
// or below its position with a five-step binary search over the lanes
// (shuffles).  A position past all 32 moves the window on by 32 users, and a
// window three quarters used restarts at the chunk's last user.  List entries
// are loaded two chunks ahead and residuals one chunk ahead.  Each e_q is
// written by one lane, its dot product summed in a fixed order for that entry,
// so the result does not depend on the schedule.
#pragma once

#include <algorithm>

#include "ials_internal.cuh"

namespace ials {

constexpr int kScanThreads = 1024;

template <int B>
constexpr int scan_smem_bytes(int n_split) {
    return n_split * B * 4;
}

template <int B, bool BF>
__global__ void __launch_bounds__(kScanThreads) k_split_resid_scan(const StepArgs a, int32_t piece) {
    static_assert(B % 8 == 0 && (B & (B - 1)) == 0, "slices are read in 16-byte pieces");
    constexpr int NV4 = B / 4, NV8 = B / 8;
    extern __shared__ float4 sdel4[];
    {
        const float4 *d4 = reinterpret_cast<const float4 *>(a.delta);
        for (int i = threadIdx.x; i < a.n_split * NV4; i += blockDim.x) sdel4[i] = d4[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t kb = warp * piece;
    if (kb >= a.n_spos) return;
    const int64_t ke = min(kb + (int64_t)piece, a.n_spos);
    const int64_t *optr = a.optr;
    const int n_u = a.n_orows;
    const int64_t qb = a.split_pos[kb];

    // the user holding qb: optr[lo] <= qb < optr[hi], narrowed about 32-fold per
    // round (lane k probes lo + (hi - lo)(k + 1) / 32; the lanes whose probe is at
    // or below qb form a prefix because optr does not decrease)
    int lo = 0, hi = n_u;
    while (hi - lo > 1) {
        const int m = lo + (int)((int64_t)(hi - lo) * (lane + 1) / 32);
        const bool le = m == lo || (m < hi && optr[m] <= qb);
        const int c = __popc(__ballot_sync(kFull, le));  // lane 31 probes hi: c <= 31
        const int nlo = __shfl_sync(kFull, m, c > 0 ? c - 1 : 0);
        const int nhi = __shfl_sync(kFull, m, c);
        if (c > 0) lo = nlo;
        hi = nhi;
    }

    // user boundaries optr[base + 1 + lane]: the window stays in registers while
    // the positions advance through it
    int base = lo;
    int bj = (int)optr[min(base + 1 + lane, n_u)];
    // an entry past the piece has position INT_MAX and split row -1
    auto fetch = [&](int64_t kc, int &q, int &sr) {
        const int64_t k = kc + lane;
        q = 0x7fffffff;
        sr = -1;
        if (k < ke) {
            q = a.split_pos[k];
            sr = a.split_row[k];
        }
    };
    int qA, sA, qB, sB;
    fetch(kb, qA, sA);
    fetch(kb + 32, qB, sB);
    float eA = sA >= 0 ? a.e[qA] : 0.f;
    for (int64_t k0 = kb; k0 < ke; k0 += 32) {
        int qC, sC;
        fetch(k0 + 64, qC, sC);
        const float eB = sB >= 0 ? a.e[qB] : 0.f;
        const bool in = sA >= 0;
        const int q = qA;
        int my_u = -1;
        for (;;) {  // count the window's boundaries at or below q; past the window: next 32 users
            int c = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1) {
                const int v = __shfl_sync(kFull, bj, c + st - 1);
                if (v <= q) c += st;
            }
            const int last = __shfl_sync(kFull, bj, 31);  // every lane takes part in each shuffle
            if (c == 31 && last <= q) c = 32;
            if (in && my_u < 0 && c < 32) my_u = base + c;
            if (!__any_sync(kFull, in && my_u < 0) || base + 32 >= n_u) break;
            base += 32;
            bj = (int)optr[min(base + 1 + lane, n_u)];
        }
        const int u31 = __shfl_sync(kFull, my_u, 31);
        if (u31 >= base + 24) {  // the window is mostly used: restart it at the last user
            base = u31;
            bj = (int)optr[min(base + 1 + lane, n_u)];
        }
        if (in && my_u >= 0) {
            const float4 *dl = sdel4 + (int64_t)sA * NV4;
            const int64_t off = (int64_t)my_u * a.d + a.p0;
            float tx = 0.f, ty = 0.f, tz = 0.f, tw = 0.f;  // four partial sums, added in a fixed order
            if constexpr (!BF) {
                const float4 *f4 = reinterpret_cast<const float4 *>(a.F + off);
#pragma unroll 8
                for (int v = 0; v < NV4; ++v) {
                    const int vv = (v + lane) & (NV4 - 1);
                    const float4 f = __ldg(f4 + vv);
                    const float4 w = dl[vv];
                    tx = fmaf(w.x, f.x, tx);
                    ty = fmaf(w.y, f.y, ty);
                    tz = fmaf(w.z, f.z, tz);
                    tw = fmaf(w.w, f.w, tw);
                }
            } else {  // f = hi + lo, formed in FP32 as the BF16 kernels do
                const uint4 *h8 = reinterpret_cast<const uint4 *>(a.Fh + off);
                const uint4 *l8 = reinterpret_cast<const uint4 *>(a.Fl + off);
                const int sw = (lane >> 2) & 1;
#pragma unroll 4
                for (int v = 0; v < NV8; ++v) {
                    const int vv = (v + lane) & (NV8 - 1);
                    const uint4 hv = __ldg(h8 + vv), lv = __ldg(l8 + vv);
                    const float4 wa = dl[2 * vv + sw], wb = dl[2 * vv + 1 - sw];
                    const float4 w0 = sw ? wb : wa, w1 = sw ? wa : wb;
                    const unsigned hw[4] = {hv.x, hv.y, hv.z, hv.w}, lw[4] = {lv.x, lv.y, lv.z, lv.w};
                    const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float2 fh = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hw[r]));
                        const float2 fl = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&lw[r]));
                        float &t0 = (r & 1) ? tz : tx;
                        float &t1 = (r & 1) ? tw : ty;
                        t0 = fmaf(wv[2 * r], fh.x + fl.x, t0);
                        t1 = fmaf(wv[2 * r + 1], fh.y + fl.y, t1);
                    }
                }
            }
            a.e[q] = eA - ((tx + ty) + (tz + tw));
        }
        qA = qB;
        sA = sB;
        eA = eB;
        qB = qC;
        sB = sC;
    }
}

// Whether the scan serves this step: the item side (position map present) with a
// user-major split list and a delta table that fits in shared memory.
template <int B>
__host__ bool split_scan_applies(const StepArgs &a) {
    return B % 8 == 0 && a.pos != nullptr && a.split_pos != nullptr && a.n_split > 0 && a.n_spos > 0 &&
           scan_smem_bytes<B>(a.n_split) <= kScanSmemMax;
}

// Kernel attributes and register count, set on the first call; every context
// makes that call outside any stream capture (its warm-up step).
template <int B, bool BF>
cudaError_t split_scan_prepare(int *regs_out) {
    static int regs = 0;
    if (regs == 0) {
        auto kern = k_split_resid_scan<B, BF>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kScanSmemMax);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa{};
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        regs = fa.numRegs > 0 ? fa.numRegs : 1;
    }
    if (regs_out) *regs_out = regs;
    return cudaSuccess;
}

template <int B, bool BF>
cudaError_t launch_split_resid_scan(const StepArgs &a, cudaStream_t s) {
    int regs = 0;
    cudaError_t e = split_scan_prepare<B, BF>(&regs);
    if (e != cudaSuccess) return e;
    const int smem = scan_smem_bytes<B>(a.n_split);
    // resident blocks per SM from the warp, register and shared-memory limits
    // (registers allocated per warp in units of 256, 1 KB of shared memory
    // reserved per block, 228 KB per SM)
    const int warps = kScanThreads / 32;
    const int per_warp_regs = (regs * 32 + 255) / 256 * 256;
    int per_sm = 64 / warps;
    per_sm = std::min(per_sm, 65536 / (warps * per_warp_regs));
    per_sm = std::min(per_sm, (228 * 1024) / (smem + 1024));
    if (per_sm < 1) per_sm = 1;
    const int64_t total_warps = (int64_t)152 * per_sm * warps;
    int64_t piece = (a.n_spos + total_warps - 1) / total_warps;
    piece = std::max<int64_t>(256, (piece + 31) / 32 * 32);
    const int64_t need = (a.n_spos + piece - 1) / piece;  // warps with a piece
    const int grid = (int)((need + warps - 1) / warps);
    prof_mark(a.prof, K_SPLIT_RESID, s);
    k_split_resid_scan<B, BF><<<grid, kScanThreads, smem, s>>>(a, (int32_t)piece);
    prof_mark(a.prof, -1, s);
    return cudaGetLastError();
}

}  // namespace ials
