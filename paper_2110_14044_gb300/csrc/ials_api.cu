// Host side of libials: the C ABI declared in include/ials.h.
//
// A context owns, in device memory (row-major float32 unless noted):
//   W (n_users x d), H (n_items x d), the residual cache e (nnz, user-major),
//   optional y / alpha (nnz), both CSR views of S (int64 row pointers, int32
//   column ids), the item-major -> user-major position map (int32), the work
//   decomposition of both sides (tasks sorted by decreasing length, long rows
//   cut into chunks), and the workspaces of one block-side step: partial
//   Gramian G^{pi} (d x b), its split-K partials, row terms R (rows x b),
//   split-row partial statistics and deltas, counters.
//
// One epoch (Algorithm 3) = residual recompute, then for k = 0 .. d/b - 1 the
// user step and the item step of block k.  Each block-side step launches:
//   Gramian tile + reduce (Eq. 10), row terms (Eq. 11 dense part), the sparse
//   warp kernel (Eqs. 11-12, solve, apply, residual update), split-row solve
//   and residual kernels, FP64 retry.
#include "ials_internal.cuh"
#include "../../include/ials.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace ials;

namespace {

thread_local std::string g_last_error;

ials_status fail(ials_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

}  // namespace

namespace ials {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace ials

namespace {

ials_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // do not leak a non-sticky error into the next call
    return IALS_ECUDA;
}

#define IALS_CUDA(call, what)                          \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
ials_status fetch(const T *src, int64_t count, std::vector<T> &dst, const char *what) {
    try {
        dst.resize((size_t)count);
    } catch (const std::bad_alloc &) {
        return fail(IALS_ENOMEM, std::string("host allocation for ") + what);
    }
    if (count == 0) return IALS_OK;
    if (is_device_ptr(src)) {
        IALS_CUDA(cudaMemcpy(dst.data(), src, sizeof(T) * count, cudaMemcpyDeviceToHost), what);
    } else {
        std::memcpy(dst.data(), src, sizeof(T) * count);
    }
    return IALS_OK;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct SideDev {
    int32_t n_rows = 0;
    int64_t *ptr = nullptr;
    int32_t *idx = nullptr;
    int32_t *pos = nullptr;  // item side only
    // item side: user-major positions whose item is a split row (increasing) and
    // the split row of each, for the residual update in user-major order
    int32_t *split_pos = nullptr, *split_row = nullptr;
    int64_t n_spos = 0;
    Task *tasks = nullptr;
    int32_t n_tasks = 0;
    SplitRow *split = nullptr;
    int32_t n_split = 0;
    Task *stasks = nullptr;
    int32_t n_stasks = 0;
    int32_t n_slots = 0;
};

bool valid_block(int b) {
    return b == 1 || b == 2 || b == 4 || b == 8 || b == 16 || b == 32 || b == 64 || b == 128 || b == 256;
}

cudaError_t launch_sparse(const StepArgs &a, cudaStream_t s) {
    switch (a.b) {
        case 1: return launch_sparse_b1(a, s);
        case 2: return launch_sparse_b2(a, s);
        case 4: return launch_sparse_b4(a, s);
        case 8: return launch_sparse_b8(a, s);
        case 16: return launch_sparse_b16(a, s);
        case 32: return launch_sparse_b32(a, s);
        case 64: return launch_sparse_b64(a, s);
        case 128: return launch_sparse_b128(a, s);
        case 256: return launch_sparse_b256(a, s);
        default: return a.b > 256 ? launch_ials_big(a, s) : cudaErrorInvalidValue;
    }
}

}  // namespace

struct ials_ctx {
    ials_params p{};
    int32_t n_users = 0, n_items = 0;
    int64_t nnz = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<DevBuf> bufs;
    float *W = nullptr, *H = nullptr, *e = nullptr, *y = nullptr, *alpha = nullptr;
    __nv_bfloat16 *Wh = nullptr, *Wl = nullptr, *Hh = nullptr, *Hl = nullptr;  // BF16 mode shadows
    GramMaps maps[2];          // BF16 mode: tensor maps of the W (0) and H (1) shadows
    RowMaps rmaps[2];          // BF16 mode: row-term maps of the users (0) and items (1) side
    __nv_bfloat16 *gth = nullptr, *gtl = nullptr;  // BF16 mode: G^T hi/lo (b x d)
    int32_t *dev_err = nullptr;  // nonzero if a bounded device wait gave up
    SideDev side[2];
    float *G = nullptr, *gram_ws = nullptr, *R = nullptr, *part = nullptr, *delta = nullptr;
    int32_t *ctl = nullptr;    // [0] work counter, [1] retry count, [2..] retry rows
    int64_t *stats = nullptr;  // [0] FP64 retries, [1] not positive definite
    double *obj = nullptr;     // [0] observed, [1] all pairs, [2] L2
    double *obj_part = nullptr;
    int32_t n_obj_part = 0;
    double *g64a = nullptr, *g64b = nullptr, *g64ws = nullptr;
    double *retry_ws = nullptr;  // b > 128: FP64 re-solve systems
    float *big_ws = nullptr;     // b = d > 256 (iALS): per-block row systems, FP32 and FP64
    double *big_ws64 = nullptr;
    // iCD path (b = 1): Gramian columns (two of d), their partials, completion counter
    float *icd_g = nullptr, *icd_gpart = nullptr;
    float *WT = nullptr, *HT = nullptr;  // transposed factors (d x n), kept current by the passes
    float *e_i = nullptr, *alpha_i = nullptr;  // item-major residual copy and weights
    float *dU = nullptr, *dI = nullptr, *icd_xold = nullptr;  // per-row deltas of the last passes
    int32_t *icd_done = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool own_stream = false;
    bool e_stale = false;  // W or H replaced since the residual cache was last computed
    // per side, for the work model: interactions in unsplit rows / split rows,
    // number of unsplit rows, split rows, partial slots, tasks
    int64_t nnz_unsplit[2] = {0, 0}, nnz_split[2] = {0, 0};
    int64_t rows_unsplit[2] = {0, 0};

    template <typename T>
    ials_status alloc(T *&out, int64_t count, const char *what) {
        void *p = nullptr;
        size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(IALS_ENOMEM, std::string("cudaMalloc failed for ") + what + " (" +
                                         std::to_string(bytes) + " bytes)");
        }
        bufs.push_back({p, bytes});
        out = static_cast<T *>(p);
        return IALS_OK;
    }
    ~ials_ctx() {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto &b : bufs) cudaFree(b.p);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

// Work decomposition of one side: one task per row, long rows cut into chunks.
struct HostTasks {
    std::vector<Task> tasks;
    std::vector<SplitRow> split;
    std::vector<Task> stasks;
    int32_t n_slots = 0;
};

constexpr int64_t kResidPiece = 128;  // interactions per residual-update piece of a split row

HostTasks build_tasks(const std::vector<int64_t> &ptr, int32_t n_rows, int64_t split_len) {
    HostTasks ht;
    ht.tasks.reserve(n_rows);
    for (int32_t r = 0; r < n_rows; ++r) {
        const int64_t n = ptr[r + 1] - ptr[r];
        if (n <= split_len) {
            ht.tasks.push_back({ptr[r], (int32_t)n, r, -1, -1});
            continue;
        }
        const int64_t nchunks = (n + split_len - 1) / split_len;
        int64_t chunk = (n + nchunks - 1) / nchunks;
        chunk = (chunk + 31) / 32 * 32;
        const int32_t srow = (int32_t)ht.split.size();
        const int32_t slot0 = ht.n_slots;
        int32_t ns = 0;
        for (int64_t b = 0; b < n; b += chunk) {
            const int64_t len = std::min(chunk, n - b);
            Task t{ptr[r] + b, (int32_t)len, r, slot0 + ns, srow};
            ht.tasks.push_back(t);
            ++ns;
        }
        // residual-update pieces of the row (any cut works: no reduction)
        for (int64_t b = 0; b < n; b += kResidPiece) {
            const int64_t len = std::min<int64_t>(kResidPiece, n - b);
            ht.stasks.push_back({ptr[r] + b, (int32_t)len, r, -1, srow});
        }
        ht.split.push_back({ptr[r], (int32_t)n, r, slot0, ns});
        ht.n_slots += ns;
    }
    std::stable_sort(ht.tasks.begin(), ht.tasks.end(),
                     [](const Task &a, const Task &b) { return a.len > b.len; });
    std::stable_sort(ht.stasks.begin(), ht.stasks.end(),
                     [](const Task &a, const Task &b) { return a.len > b.len; });
    return ht;
}

ials_status upload(ials_ctx *c, const void *src, void *dst, size_t bytes, const char *what) {
    if (bytes == 0) return IALS_OK;
    IALS_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->stream), what);
    return IALS_OK;
}

// Residual cache e = W H^T - y (Alg. 3 "Compute yhat") over the user-side tasks.
cudaError_t residual_enqueue(ials_ctx *c) {
    return launch_residual_tasks(c->side[0].tasks, c->side[0].n_tasks, c->side[0].idx, c->W, c->H, c->y,
                                 c->p.d, c->e, c->ctl, c->stream);
}

// After ials_set_factors the cache is rebuilt lazily: every epoch starts with
// its own recompute, so only the calls that read it outside an epoch rebuild it.
cudaError_t ensure_residuals(ials_ctx *c) {
    if (!c->e_stale) return cudaSuccess;
    cudaError_t err = residual_enqueue(c);
    if (err == cudaSuccess) c->e_stale = false;
    return err;
}

cudaError_t launch_sparse_bf16(int32_t b, const StepArgs &a, cudaStream_t s) {
    switch (b) {
        case 16: return launch_sparse_bf16_b16(a, s);
        case 32: return launch_sparse_bf16_b32(a, s);
        case 64: return launch_sparse_bf16_b64(a, s);
        case 128: return launch_sparse_bf16_b128(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// Arguments of one block-side step on the context's buffers.
StepArgs step_args(ials_ctx *c, int side, int p0, Profiler *prof) {
    SideDev &sd = c->side[side];
    StepArgs a{};
    a.ptr = sd.ptr;
    a.idx = sd.idx;
    a.pos = side == 1 ? sd.pos : nullptr;
    a.e = c->e;
    a.alpha = c->alpha;
    a.y = c->y;
    a.X = side == 0 ? c->W : c->H;
    a.F = side == 0 ? c->H : c->W;
    a.G = c->G;
    a.R = c->R;
    a.n_rows = sd.n_rows;
    a.d = c->p.d;
    a.b = c->p.b;
    a.p0 = p0;
    a.alpha0 = (float)c->p.alpha0;
    a.lambda = (float)c->p.lambda;
    a.nu = (float)c->p.nu;
    a.tasks = sd.tasks;
    a.n_tasks = sd.n_tasks;
    a.split = sd.split;
    a.n_split = sd.n_split;
    a.stasks = sd.stasks;
    a.n_stasks = sd.n_stasks;
    a.part = c->part;
    a.delta = c->delta;
    a.counter = c->ctl;
    a.retry = c->ctl + 1;
    a.stats = c->stats;
    a.force_fp64 = (c->p.flags & IALS_FLAG_FORCE_FP64) ? 1 : 0;
    a.retry_ws = c->retry_ws;
    a.big_ws = c->big_ws;
    a.big_ws64 = c->big_ws64;
    a.prof = prof;
    if (side == 1 && sd.split_pos) {
        a.optr = c->side[0].ptr;
        a.split_pos = sd.split_pos;
        a.split_row = sd.split_row;
        a.n_spos = sd.n_spos;
        a.n_orows = c->n_users;
    }
    a.Xh = side == 0 ? c->Wh : c->Hh;
    a.Xl = side == 0 ? c->Wl : c->Hl;
    a.Fh = side == 0 ? c->Hh : c->Wh;
    a.Fl = side == 0 ? c->Hl : c->Wl;
    return a;
}

// The iCD path (Algorithm 2) runs for b = 1 unless the general path is forced.
bool use_icd(const ials_ctx *c) { return c->p.b == 1 && !(c->p.flags & IALS_FLAG_GENERAL); }

// Transposed copies of W and H for the iCD passes (each pass then keeps them current).
cudaError_t icd_transpose(ials_ctx *c, Profiler *prof) {
    prof_mark(prof, K_RESIDUAL, c->stream);  // data movement at the epoch start
    cudaError_t e = launch_transpose(c->W, c->n_users, c->p.d, c->WT, c->stream);
    if (e == cudaSuccess) e = launch_transpose(c->H, c->n_items, c->p.d, c->HT, c->stream);
    prof_mark(prof, -1, c->stream);
    return e;
}

// One iCD pass: side `side`, coordinate f, fixed-side Gramian column in g_in;
// forms the updated side's column fn (>= 0) into g_out on the way.  The side's
// own residual copy must be current except for the previous pass's deltas
// when `pending` (user pass: the item pass at f - 1; item pass: the user pass at f).
ials_status icd_pass_enqueue(ials_ctx *c, int side, int f, int fn, const float *g_in, float *g_out,
                             bool pending, Profiler *prof) {
    IcdArgs a;
    a.s = step_args(c, side, f, prof);
    a.eo = side == 0 ? c->e : c->e_i;
    a.alpha_o = side == 0 ? c->alpha : c->alpha_i;
    a.dprev = pending ? (side == 0 ? c->dI : c->dU) : nullptr;
    a.fprev = side == 0 ? f - 1 : f;
    a.dself = side == 0 ? c->dU : c->dI;
    a.xold = c->icd_xold;
    a.f = f;
    a.fn = fn;
    a.g_in = g_in;
    a.g_out = g_out;
    a.gpart = c->icd_gpart;
    a.done = c->icd_done;
    a.grid = icd_row_grid(a.s.n_tasks, c->p.d);
    a.FT = side == 0 ? c->HT : c->WT;
    a.XT = side == 0 ? c->WT : c->HT;
    a.n_fixed = side == 0 ? c->n_items : c->n_users;
    IALS_CUDA(launch_icd(a, c->stream), "iCD pass");
    return IALS_OK;
}

// The iALS path (Algorithm 1) runs for b = d >= 64 unless the general path is forced (which
// creation refuses above b = 256).
bool use_ials(const ials_ctx *c) {
    return c->p.b == c->p.d && c->p.b >= 64 && !(c->p.flags & IALS_FLAG_GENERAL);
}

// One iALS epoch (Algorithm 1): per side the full Gramian G of the fixed side,
// then every row solved directly from Eq. 3 (statistics sum alpha f f^T and
// sum alpha y f, dense terms alpha0 G + lambda_r I).  No residual cache is
// read or kept.
ials_status direct_epoch_enqueue(ials_ctx *c, Profiler *prof) {
    const int32_t d = c->p.d;
    cudaStream_t s = c->stream;
    for (int side = 0; side < 2; ++side) {
        const int64_t n_fixed = side == 0 ? c->n_items : c->n_users;
        prof_mark(prof, K_GRAM, s);
        if (c->p.precision == IALS_PREC_BF16) {
            IALS_CUDA(launch_gram_tc(c->maps[side == 0 ? 1 : 0], n_fixed, d, 0, d, c->G, c->gram_ws, c->dev_err, s),
                      "Gramian (tcgen05)");
        } else {
            IALS_CUDA(launch_gram(side == 0 ? c->H : c->W, n_fixed, d, 0, d, c->G, c->gram_ws, s), "Gramian");
        }
        prof_mark(prof, -1, s);
        IALS_CUDA(cudaMemsetAsync(c->ctl, 0, 2 * sizeof(int32_t), s), "counter reset");
        StepArgs a = step_args(c, side, 0, prof);
        a.direct = 1;
        if (c->p.precision == IALS_PREC_BF16) {
            IALS_CUDA(launch_sparse_bf16(d, a, s), "iALS row solves (BF16)");
        } else {
            IALS_CUDA(launch_sparse(a, s), "iALS row solves");
        }
    }
    return IALS_OK;
}

// One iCD epoch: for every coordinate f the user pass, then the item pass
// (Algorithm 2).  H's column 0 is formed once; every later column comes out of
// the pass before the one that needs it.
ials_status icd_epoch_enqueue(ials_ctx *c, Profiler *prof) {
    const int d = c->p.d;
    float *gH = c->icd_g, *gW = c->icd_g + d;
    IALS_CUDA(icd_transpose(c, prof), "transposed factors");
    prof_mark(prof, K_RESIDUAL, c->stream);
    IALS_CUDA(launch_perm_gather(c->e, c->side[1].pos, c->nnz, c->e_i, c->stream), "item-major residuals");
    prof_mark(prof, K_GRAM, c->stream);
    IALS_CUDA(launch_gram(c->H, c->n_items, d, 0, 1, gH, c->gram_ws, c->stream), "Gramian column");
    prof_mark(prof, -1, c->stream);
    for (int f = 0; f < d; ++f) {
        ials_status st = icd_pass_enqueue(c, 0, f, f, gH, gW, f > 0, prof);
        if (st != IALS_OK) return st;
        st = icd_pass_enqueue(c, 1, f, f + 1 < d ? f + 1 : -1, gW, gH, true, prof);
        if (st != IALS_OK) return st;
    }
    return IALS_OK;
}

ials_status step_enqueue(ials_ctx *c, int side, int block, Profiler *prof = nullptr) {
    if (use_icd(c)) {  // one coordinate: its Gramian column of the fixed side, then the pass
        IALS_CUDA(icd_transpose(c, prof), "transposed factors");
        const float *F = side == 0 ? c->H : c->W;
        const int64_t n_fixed = side == 0 ? c->n_items : c->n_users;
        prof_mark(prof, K_GRAM, c->stream);
        IALS_CUDA(launch_gram(F, n_fixed, c->p.d, block, 1, c->icd_g, c->gram_ws, c->stream), "Gramian column");
        prof_mark(prof, -1, c->stream);
        if (side == 0) return icd_pass_enqueue(c, 0, block, -1, c->icd_g, nullptr, false, prof);
        // the item pass on an item-major copy of the (current) user-major cache, written back
        IALS_CUDA(launch_perm_gather(c->e, c->side[1].pos, c->nnz, c->e_i, c->stream), "item-major residuals");
        ials_status st = icd_pass_enqueue(c, 1, block, -1, c->icd_g, nullptr, false, prof);
        if (st != IALS_OK) return st;
        IALS_CUDA(launch_perm_scatter(c->e_i, c->side[1].pos, c->nnz, c->e, c->stream), "user-major residuals");
        return IALS_OK;
    }
    const int32_t d = c->p.d, b = c->p.b, p0 = block * b;
    SideDev &sd = c->side[side];
    float *X = side == 0 ? c->W : c->H;
    const float *F = side == 0 ? c->H : c->W;
    const int64_t n_fixed = side == 0 ? c->n_items : c->n_users;
    cudaStream_t s = c->stream;
    prof_mark(prof, K_GRAM, s);
    if (c->p.precision == IALS_PREC_BF16) {
        IALS_CUDA(launch_gram_tc(c->maps[side == 0 ? 1 : 0], n_fixed, d, p0, b, c->G, c->gram_ws, c->dev_err, s),
                  "partial Gramian (tcgen05)");
    } else {
        IALS_CUDA(launch_gram(F, n_fixed, d, p0, b, c->G, c->gram_ws, s), "partial Gramian");
    }
    prof_mark(prof, K_ROWTERM, s);
    if (c->p.precision == IALS_PREC_BF16) {
        IALS_CUDA(launch_rowterm_tc(c->rmaps[side], c->G, c->gth, c->gtl, X, sd.ptr, sd.n_rows, d, p0, b,
                                    (float)c->p.alpha0, (float)c->p.lambda, (float)c->p.nu, c->R, c->dev_err, s),
                  "row terms (tcgen05)");
    } else {
        IALS_CUDA(launch_rowterm(X, sd.ptr, sd.n_rows, d, p0, b, c->G, (float)c->p.alpha0,
                                 (float)c->p.lambda, (float)c->p.nu, c->R, s),
                  "row terms");
    }
    prof_mark(prof, -1, s);
    IALS_CUDA(cudaMemsetAsync(c->ctl, 0, 2 * sizeof(int32_t), s), "counter reset");
    StepArgs a = step_args(c, side, p0, prof);
    if (c->p.precision == IALS_PREC_BF16) {
        IALS_CUDA(launch_sparse_bf16(b, a, s), "sparse block step (BF16)");
    } else {
        IALS_CUDA(launch_sparse(a, s), "sparse block step");
    }
    return IALS_OK;
}

ials_status epoch_enqueue(ials_ctx *c, Profiler *prof = nullptr) {
    if (use_ials(c)) return direct_epoch_enqueue(c, prof);
    prof_mark(prof, K_RESIDUAL, c->stream);
    IALS_CUDA(residual_enqueue(c), "residual recompute");
    prof_mark(prof, -1, c->stream);
    if (use_icd(c)) return icd_epoch_enqueue(c, prof);
    const int nb = c->p.d / c->p.b;
    for (int k = 0; k < nb; ++k)
        for (int side = 0; side < 2; ++side) {
            ials_status st = step_enqueue(c, side, k, prof);
            if (st != IALS_OK) return st;
        }
    return IALS_OK;
}

ials_status finish(ials_ctx *c) {
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    int64_t st[2];
    IALS_CUDA(cudaMemcpy(st, c->stats, sizeof(st), cudaMemcpyDeviceToHost), "stats");
    int32_t derr = 0;
    IALS_CUDA(cudaMemcpy(&derr, c->dev_err, sizeof(derr), cudaMemcpyDeviceToHost), "device error flag");
    if (derr != 0)
        return fail(IALS_ETIMEDOUT, "a bounded device wait gave up (code " + std::to_string(derr) + ")");
    if (st[1] > 0)
        return fail(IALS_ENOTPD, std::to_string(st[1]) +
                                     " row(s) had a Hessian that is not positive definite in FP64");
    return IALS_OK;
}

ials_status objective_enqueue(ials_ctx *c) {
    cudaStream_t s = c->stream;
    const int32_t d = c->p.d;
    IALS_CUDA(cudaMemsetAsync(c->obj, 0, 3 * sizeof(double), s), "objective reset");
    IALS_CUDA(launch_sq_loss(c->side[0].ptr, c->side[0].idx, c->W, c->H, c->y, c->alpha,
                             c->n_users, d, c->obj_part, c->n_obj_part, c->obj + 0, s),
              "observed loss");
    IALS_CUDA(launch_gram64(c->W, c->n_users, d, c->g64a, c->g64ws, s), "Gramian of W");
    IALS_CUDA(launch_gram64(c->H, c->n_items, d, c->g64b, c->g64ws, s), "Gramian of H");
    IALS_CUDA(launch_frobenius(c->g64a, c->g64b, d, c->p.alpha0, c->obj + 1, s), "all-pairs term");
    IALS_CUDA(launch_reg_loss(c->side[0].ptr, c->W, c->n_users, d, c->p.lambda, c->p.nu,
                              c->obj_part, c->n_obj_part, c->obj + 2, s),
              "L2 term (users)");
    IALS_CUDA(launch_reg_loss(c->side[1].ptr, c->H, c->n_items, d, c->p.lambda, c->p.nu,
                              c->obj_part, c->n_obj_part, c->obj + 2, s),
              "L2 term (items)");
    return IALS_OK;
}

ials_status objective_read(ials_ctx *c, double *out) {
    double v[3];
    IALS_CUDA(cudaMemcpyAsync(v, c->obj, sizeof(v), cudaMemcpyDeviceToHost, c->stream), "objective");
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    *out = v[0] + v[1] + v[2];
    return IALS_OK;
}

}  // namespace

extern "C" {

const char *ials_last_error(void) { return g_last_error.c_str(); }

ials_status ials_create(const ials_params *params, int32_t n_users, int32_t n_items, int64_t nnz,
                        const int64_t *u_indptr, const int32_t *u_items, const int64_t *i_indptr,
                        const int32_t *i_users, const float *y, const float *alpha,
                        void *cuda_stream, ials_ctx **out) {
    g_last_error.clear();
    if (!params || !out) return fail(IALS_EINVAL, "params and out must not be NULL");
    *out = nullptr;
    const ials_params p = *params;
    if (p.d < 4 || p.d > 4096 || p.d % 4 != 0) return fail(IALS_EINVAL, "d must be a multiple of 4 in [4, 4096]");
    const bool big = p.b == p.d && ials_big_supported(p.d);  // iALS only (Algorithm 1)
    if (!big && (!valid_block(p.b) || p.d % p.b != 0))
        return fail(IALS_EINVAL, "b must be a power of two <= 256 that divides d, or b = d (a multiple of 64 up "
                                 "to 1024)");
    if (big && (p.flags & IALS_FLAG_GENERAL))
        return fail(IALS_EINVAL, "the general block step needs b <= 256; b = d above 256 runs iALS only");
    if (!(p.alpha0 >= 0) || !(p.lambda >= 0) || !(p.nu >= 0) || !std::isfinite(p.alpha0) ||
        !std::isfinite(p.lambda) || !std::isfinite(p.nu))
        return fail(IALS_EINVAL, "alpha0, lambda, nu must be finite and >= 0");
    if (p.precision != IALS_PREC_FP32 && p.precision != IALS_PREC_BF16)
        return fail(IALS_EINVAL, "unknown precision");
    if (p.precision == IALS_PREC_BF16 && ((p.b != 16 && p.b != 32 && p.b != 64 && p.b != 128) || p.d % 8 != 0))
        return fail(IALS_EINVAL, "BF16 precision needs b in {16, 32, 64, 128} and d % 8 == 0");
    if (p.split_len != 0 && (p.split_len < 32 || p.split_len > (1 << 24)))
        return fail(IALS_EINVAL, "split_len must be 0 or in [32, 2^24]");
    if (p.reserved != 0) return fail(IALS_EINVAL, "reserved must be 0");
    if (n_users <= 0 || n_items <= 0) return fail(IALS_EINVAL, "n_users and n_items must be > 0");
    if (nnz < 0 || nnz >= (int64_t)1 << 31) return fail(IALS_EINVAL, "nnz must be in [0, 2^31)");
    if (!u_indptr || (nnz > 0 && !u_items)) return fail(IALS_EINVAL, "user CSR missing");
    if ((i_indptr && nnz > 0 && !i_users) || (!i_indptr && i_users))
        return fail(IALS_EINVAL, "item CSR must be given completely or not at all");

    // ---- inputs to host and validation
    std::vector<int64_t> uptr;
    std::vector<int32_t> uidx;
    ials_status st;
    if ((st = fetch(u_indptr, (int64_t)n_users + 1, uptr, "user indptr")) != IALS_OK) return st;
    if ((st = fetch(u_items, nnz, uidx, "user items")) != IALS_OK) return st;
    if (uptr[0] != 0 || uptr[n_users] != nnz) return fail(IALS_EINVAL, "user indptr must start at 0 and end at nnz");
    for (int32_t u = 0; u < n_users; ++u)
        if (uptr[u + 1] < uptr[u]) return fail(IALS_EINVAL, "user indptr must be non-decreasing");
    {
        std::vector<int32_t> stamp(n_items, -1);
        for (int32_t u = 0; u < n_users; ++u)
            for (int64_t s = uptr[u]; s < uptr[u + 1]; ++s) {
                const int32_t i = uidx[s];
                if (i < 0 || i >= n_items) return fail(IALS_EINVAL, "item id out of range");
                if (stamp[i] == u) return fail(IALS_EINVAL, "repeated item within a user row");
                stamp[i] = u;
            }
    }
    // item-major view (users ascending within each item) and position map
    std::vector<int64_t> iptr(n_items + 1, 0);
    std::vector<int32_t> iidx(nnz), ipos(nnz);
    for (int64_t s = 0; s < nnz; ++s) iptr[uidx[s] + 1]++;
    for (int32_t i = 0; i < n_items; ++i) iptr[i + 1] += iptr[i];
    {
        std::vector<int64_t> fillp(iptr.begin(), iptr.end() - 1);
        for (int32_t u = 0; u < n_users; ++u)
            for (int64_t s = uptr[u]; s < uptr[u + 1]; ++s) {
                const int64_t t = fillp[uidx[s]]++;
                iidx[t] = u;
                ipos[t] = (int32_t)s;
            }
    }
    if (i_indptr) {
        std::vector<int64_t> gptr;
        std::vector<int32_t> gidx;
        if ((st = fetch(i_indptr, (int64_t)n_items + 1, gptr, "item indptr")) != IALS_OK) return st;
        if ((st = fetch(i_users, nnz, gidx, "item users")) != IALS_OK) return st;
        for (int32_t i = 0; i <= n_items; ++i)
            if (gptr[i] != iptr[i]) return fail(IALS_EINVAL, "item CSR is not the transpose of the user CSR");
        for (int32_t i = 0; i < n_items; ++i) {
            std::sort(gidx.begin() + gptr[i], gidx.begin() + gptr[i + 1]);
            for (int64_t t = gptr[i]; t < gptr[i + 1]; ++t)
                if (gidx[t] != iidx[t]) return fail(IALS_EINVAL, "item CSR is not the transpose of the user CSR");
        }
    }
    std::vector<float> hy, ha;
    if (y) {
        if ((st = fetch(y, nnz, hy, "y")) != IALS_OK) return st;
        for (float v : hy)
            if (!std::isfinite(v)) return fail(IALS_EINVAL, "y must be finite");
    }
    if (alpha) {
        if ((st = fetch(alpha, nnz, ha, "alpha")) != IALS_OK) return st;
        for (float v : ha)
            if (!(v > 0.f) || !std::isfinite(v)) return fail(IALS_EINVAL, "alpha must be finite and > 0");
    }

    int dev = 0;
    IALS_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    cudaDeviceProp prop;
    IALS_CUDA(cudaGetDeviceProperties(&prop, dev), "cudaGetDeviceProperties");
    if (prop.major * 10 + prop.minor != 103)
        return fail(IALS_ECUDA, "libials is built for sm_103a (GB300); device is sm_" +
                                    std::to_string(prop.major * 10 + prop.minor));

    ials_ctx *c = new (std::nothrow) ials_ctx;
    if (!c) return fail(IALS_ENOMEM, "context");
    c->p = p;
    c->n_users = n_users;
    c->n_items = n_items;
    c->nnz = nnz;
    c->device = dev;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (!c->stream) {
        // The legacy default stream cannot be captured into a graph: use a
        // private stream that still orders with it (a blocking stream).
        cudaError_t se = cudaStreamCreate(&c->stream);
        if (se != cudaSuccess) { c->stream = nullptr; delete c; return cuda_fail(se, "stream"); }
        c->own_stream = true;
    }

    // ---- work decomposition
    const int64_t split_len = p.split_len > 0 ? (int64_t)p.split_len
                                              : std::max<int64_t>(256, std::min<int64_t>(8192, nnz / (152 * 16 * 2)));
    HostTasks ht[2] = {build_tasks(uptr, n_users, split_len), build_tasks(iptr, n_items, split_len)};
    for (int sd = 0; sd < 2; ++sd)
        for (const Task &t : ht[sd].tasks) {
            if (t.slot < 0) { c->nnz_unsplit[sd] += t.len; c->rows_unsplit[sd] += 1; }
            else c->nnz_split[sd] += t.len;
        }

    const int32_t d = p.d, b = p.b;
#define ALLOC(ptr, n, what)                                   \
    do {                                                      \
        ials_status _s = c->alloc(ptr, (int64_t)(n), what);    \
        if (_s != IALS_OK) { delete c; return _s; }            \
    } while (0)
    ALLOC(c->W, (int64_t)n_users * d, "W");
    ALLOC(c->H, (int64_t)n_items * d, "H");
    if (p.precision == IALS_PREC_BF16) {
        ALLOC(c->Wh, (int64_t)n_users * d, "W hi");
        ALLOC(c->Wl, (int64_t)n_users * d, "W lo");
        ALLOC(c->Hh, (int64_t)n_items * d, "H hi");
        ALLOC(c->Hl, (int64_t)n_items * d, "H lo");
        ALLOC(c->gth, (int64_t)b * d, "G^T hi");
        ALLOC(c->gtl, (int64_t)b * d, "G^T lo");
    }
    ALLOC(c->e, nnz, "residuals");
    if (y) ALLOC(c->y, nnz, "y");
    if (alpha) ALLOC(c->alpha, nnz, "alpha");
    for (int sd = 0; sd < 2; ++sd) {
        SideDev &S = c->side[sd];
        S.n_rows = sd == 0 ? n_users : n_items;
        ALLOC(S.ptr, (int64_t)S.n_rows + 1, "CSR indptr");
        ALLOC(S.idx, nnz, "CSR indices");
        if (sd == 1) ALLOC(S.pos, nnz, "position map");
        // the item side's split rows update their residuals in user-major order
        // when they hold at least an eighth of the interactions
        if (sd == 1 && b % 8 == 0 && b <= 256 && !(b == d && b >= 64 && !(p.flags & IALS_FLAG_GENERAL)) &&
            !ht[1].split.empty() && c->nnz_split[1] * 8 >= nnz) {
            S.n_spos = c->nnz_split[1];
            ALLOC(S.split_pos, S.n_spos, "split positions");
            ALLOC(S.split_row, S.n_spos, "split rows of the positions");
        }
        S.n_tasks = (int32_t)ht[sd].tasks.size();
        S.n_split = (int32_t)ht[sd].split.size();
        S.n_stasks = (int32_t)ht[sd].stasks.size();
        S.n_slots = ht[sd].n_slots;
        ALLOC(S.tasks, S.n_tasks, "tasks");
        ALLOC(S.split, S.n_split, "split rows");
        ALLOC(S.stasks, S.n_stasks, "split tasks");
    }
    const int64_t max_rows = std::max(n_users, n_items);
    const int32_t max_slots = std::max(c->side[0].n_slots, c->side[1].n_slots);
    const int32_t max_split = std::max(c->side[0].n_split, c->side[1].n_split);
    ALLOC(c->G, (int64_t)d * b, "partial Gramian");
    ALLOC(c->gram_ws, std::max(std::max(gram_ws_floats(n_items, d, b), gram_ws_floats(n_users, d, b)),
                               std::max(gram_tc_ws_floats(n_items, d, b), gram_tc_ws_floats(n_users, d, b))),
          "Gramian workspace");
    ALLOC(c->dev_err, 1, "error flag");
    const bool big_ials = b > 256;  // iALS at b = d > 256: whole rows, no row terms or split partials
    ALLOC(c->R, big_ials ? 1 : max_rows * b, "row terms");
    ALLOC(c->part, big_ials ? 1 : (int64_t)max_slots * (b * b + b), "split partials");
    ALLOC(c->delta, big_ials ? 1 : (int64_t)max_split * b, "split deltas");
    if (big_ials) {
        ALLOC(c->big_ws, ials_big_ws_floats(d), "iALS row systems");
        ALLOC(c->big_ws64, ials_big_ws_doubles(d), "iALS FP64 row systems");
    }
    ALLOC(c->ctl, max_rows + 2, "counters");
    ALLOC(c->stats, 2, "stats");
    ALLOC(c->obj, 3, "objective");
    c->n_obj_part = 4 * 152;
    ALLOC(c->obj_part, c->n_obj_part, "objective partials");
    if (b == 1) {
        ALLOC(c->icd_g, 2 * (int64_t)d, "Gramian columns");
        ALLOC(c->icd_gpart, (int64_t)(icd_row_grid(std::max(c->side[0].n_tasks, c->side[1].n_tasks), d) +
                                      icd_split_grid(max_split, d)) * d,
              "Gramian column partials");
        ALLOC(c->WT, (int64_t)n_users * d, "W transposed");
        ALLOC(c->HT, (int64_t)n_items * d, "H transposed");
        ALLOC(c->e_i, nnz, "item-major residuals");
        if (alpha) ALLOC(c->alpha_i, nnz, "item-major weights");
        ALLOC(c->dU, n_users, "user deltas");
        ALLOC(c->dI, n_items, "item deltas");
        ALLOC(c->icd_xold, max_split, "long-row coordinates");
        ALLOC(c->icd_done, 1, "completion counter");
    }
    if (sparse_retry_ws_doubles(b) > 0) ALLOC(c->retry_ws, sparse_retry_ws_doubles(b), "FP64 re-solve workspace");
    ALLOC(c->g64a, (int64_t)d * d, "FP64 Gramian");
    ALLOC(c->g64b, (int64_t)d * d, "FP64 Gramian");
    ALLOC(c->g64ws, std::max(gram64_ws_doubles(n_users, d), gram64_ws_doubles(n_items, d)),
          "FP64 Gramian workspace");
#undef ALLOC

    ials_status us = IALS_OK;
    auto up = [&](const void *src, void *dst, size_t bytes, const char *what) {
        if (us == IALS_OK) us = upload(c, src, dst, bytes, what);
    };
    up(uptr.data(), c->side[0].ptr, sizeof(int64_t) * (n_users + 1), "user indptr");
    up(uidx.data(), c->side[0].idx, sizeof(int32_t) * nnz, "user items");
    up(iptr.data(), c->side[1].ptr, sizeof(int64_t) * (n_items + 1), "item indptr");
    up(iidx.data(), c->side[1].idx, sizeof(int32_t) * nnz, "item users");
    up(ipos.data(), c->side[1].pos, sizeof(int32_t) * nnz, "position map");
    if (c->side[1].split_pos) {
        std::vector<int32_t> sq(nnz, -1);
        for (size_t r = 0; r < ht[1].split.size(); ++r) {
            const SplitRow &sr = ht[1].split[r];
            for (int64_t t = sr.begin; t < sr.begin + sr.len; ++t) sq[ipos[t]] = (int32_t)r;
        }
        std::vector<int32_t> lp, lr;
        lp.reserve(c->side[1].n_spos);
        lr.reserve(c->side[1].n_spos);
        for (int64_t q = 0; q < nnz; ++q)
            if (sq[q] >= 0) { lp.push_back((int32_t)q); lr.push_back(sq[q]); }
        up(lp.data(), c->side[1].split_pos, sizeof(int32_t) * lp.size(), "split positions");
        up(lr.data(), c->side[1].split_row, sizeof(int32_t) * lr.size(), "split rows of the positions");
    }
    if (y) up(hy.data(), c->y, sizeof(float) * nnz, "y");
    if (alpha) up(ha.data(), c->alpha, sizeof(float) * nnz, "alpha");
    for (int sd = 0; sd < 2; ++sd) {
        up(ht[sd].tasks.data(), c->side[sd].tasks, sizeof(Task) * ht[sd].tasks.size(), "tasks");
        up(ht[sd].split.data(), c->side[sd].split, sizeof(SplitRow) * ht[sd].split.size(), "split rows");
        up(ht[sd].stasks.data(), c->side[sd].stasks, sizeof(Task) * ht[sd].stasks.size(), "split tasks");
    }
    if (us != IALS_OK) { delete c; return us; }
    if (c->alpha_i) {
        const cudaError_t ge = launch_perm_gather(c->alpha, c->side[1].pos, nnz, c->alpha_i, c->stream);
        if (ge != cudaSuccess) { delete c; return cuda_fail(ge, "item-major weights"); }
    }
    cudaError_t e1 = launch_init_normal(c->W, (int64_t)n_users * d, p.init_std, p.seed, 1, c->stream);
    cudaError_t e2 = launch_init_normal(c->H, (int64_t)n_items * d, p.init_std, p.seed, 2, c->stream);
    cudaError_t e3 = cudaMemsetAsync(c->stats, 0, 2 * sizeof(int64_t), c->stream);
    if (e3 == cudaSuccess && c->Wh) e3 = launch_split_bf16(c->W, (int64_t)n_users * d, c->Wh, c->Wl, c->stream);
    if (e3 == cudaSuccess && c->Hh) e3 = launch_split_bf16(c->H, (int64_t)n_items * d, c->Hh, c->Hl, c->stream);
    if (e3 == cudaSuccess) e3 = cudaMemsetAsync(c->dev_err, 0, sizeof(int32_t), c->stream);
    if (e3 == cudaSuccess && c->icd_done) e3 = cudaMemsetAsync(c->icd_done, 0, sizeof(int32_t), c->stream);
    if (e3 == cudaSuccess && c->Wh &&
        (!make_gram_maps(c->maps[0], c->Wh, c->Wl, n_users, d, b) ||
         !make_gram_maps(c->maps[1], c->Hh, c->Hl, n_items, d, b) ||
         !make_row_maps(c->rmaps[0], c->Wh, c->Wl, n_users, d, c->gth, c->gtl, b) ||
         !make_row_maps(c->rmaps[1], c->Hh, c->Hl, n_items, d, c->gth, c->gtl, b))) {
        delete c;
        return fail(IALS_ECUDA, "could not encode TMA tensor maps (cuTensorMapEncodeTiled)");
    }
    cudaError_t e4 = cudaStreamSynchronize(c->stream);
    cudaError_t e5 = residual_enqueue(c);
    cudaError_t e6 = cudaStreamSynchronize(c->stream);
    // Set kernel attributes of both sides' sparse variants now, outside any
    // stream capture: an empty step launches nothing but the (idle) retry kernel.
    cudaError_t e7 = b > 256 ? ials_big_prepare() : cudaSuccess;
    for (int k = 0; k < (use_ials(c) ? 4 : 2) && e7 == cudaSuccess; ++k) {
        if (b > 256 && !(k >> 1)) continue;  // above b = 256 only the iALS path exists
        const int sd = k & 1;
        StepArgs a = step_args(c, sd, 0, nullptr);
        a.n_tasks = a.n_split = a.n_stasks = 0;
        a.n_rows = 0;
        a.direct = k >> 1;  // the iALS path's variants too
        e7 = cudaMemsetAsync(c->ctl, 0, 2 * sizeof(int32_t), c->stream);
        if (e7 == cudaSuccess) {
            if (p.precision == IALS_PREC_BF16)
                e7 = launch_sparse_bf16(b, a, c->stream);
            else
                e7 = launch_sparse(a, c->stream);
        }
    }
    if (e7 == cudaSuccess && b == 1) e7 = icd_prepare();
    if (e7 == cudaSuccess) e7 = dense_prepare();
    cudaError_t e8 = cudaStreamSynchronize(c->stream);
    for (cudaError_t e : {e1, e2, e3, e4, e5, e6, e7, e8})
        if (e != cudaSuccess) { delete c; return cuda_fail(e, "context initialisation"); }
    *out = c;
    return IALS_OK;
}

ials_status ials_destroy(ials_ctx *ctx) {
    if (!ctx) return IALS_OK;
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
    return IALS_OK;
}

ials_status ials_epoch(ials_ctx *c, int32_t n_epochs, double *objective_after) {
    if (!c || n_epochs < 0) return fail(IALS_EINVAL, "bad context or epoch count");
    IALS_CUDA(cudaMemsetAsync(c->stats, 0, 2 * sizeof(int64_t), c->stream), "stats reset");
    if (c->p.flags & IALS_FLAG_GRAPH) {
        if (!c->graph) {
            cudaGraph_t g = nullptr;
            IALS_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
            ials_status st = epoch_enqueue(c);
            cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
            if (st != IALS_OK) { if (g) cudaGraphDestroy(g); return st; }
            if (ce != cudaSuccess) return cuda_fail(ce, "end capture");
            ce = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) { c->graph = nullptr; return cuda_fail(ce, "graph instantiate"); }
        }
        for (int t = 0; t < n_epochs; ++t) IALS_CUDA(cudaGraphLaunch(c->graph, c->stream), "graph launch");
    } else {
        for (int t = 0; t < n_epochs; ++t) {
            ials_status st = epoch_enqueue(c);
            if (st != IALS_OK) return st;
        }
    }
    // each epoch recomputed the cache first; the iALS path keeps none, and the iCD
    // path leaves the user-major copy one item pass behind
    if (n_epochs > 0) c->e_stale = use_ials(c) || use_icd(c);
    ials_status st = finish(c);
    if (objective_after && (st == IALS_OK || st == IALS_ENOTPD)) {
        ials_status s2 = objective_enqueue(c);
        if (s2 != IALS_OK) return s2;
        s2 = objective_read(c, objective_after);
        if (s2 != IALS_OK) return s2;
    }
    return st;
}

ials_status ials_objective(ials_ctx *c, double *out) {
    if (!c || !out) return fail(IALS_EINVAL, "bad arguments");
    ials_status st = objective_enqueue(c);
    if (st != IALS_OK) return st;
    return objective_read(c, out);
}

ials_status ials_get_factors(ials_ctx *c, float *W, float *H) {
    if (!c) return fail(IALS_EINVAL, "bad context");
    const size_t wb = sizeof(float) * (size_t)c->n_users * c->p.d, hb = sizeof(float) * (size_t)c->n_items * c->p.d;
    if (W) IALS_CUDA(cudaMemcpyAsync(W, c->W, wb, cudaMemcpyDefault, c->stream), "copy W out");
    if (H) IALS_CUDA(cudaMemcpyAsync(H, c->H, hb, cudaMemcpyDefault, c->stream), "copy H out");
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return IALS_OK;
}

ials_status ials_set_factors(ials_ctx *c, const float *W, const float *H) {
    if (!c) return fail(IALS_EINVAL, "bad context");
    const size_t wb = sizeof(float) * (size_t)c->n_users * c->p.d, hb = sizeof(float) * (size_t)c->n_items * c->p.d;
    if (W) IALS_CUDA(cudaMemcpyAsync(c->W, W, wb, cudaMemcpyDefault, c->stream), "copy W in");
    if (H) IALS_CUDA(cudaMemcpyAsync(c->H, H, hb, cudaMemcpyDefault, c->stream), "copy H in");
    if (W && c->Wh)
        IALS_CUDA(launch_split_bf16(c->W, (int64_t)c->n_users * c->p.d, c->Wh, c->Wl, c->stream), "W shadow");
    if (H && c->Hh)
        IALS_CUDA(launch_split_bf16(c->H, (int64_t)c->n_items * c->p.d, c->Hh, c->Hl, c->stream), "H shadow");
    // the residual cache is a function of W and H: rebuilt before it is next read
    c->e_stale = true;
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return IALS_OK;
}

ials_status ials_recompute_residuals(ials_ctx *c) {
    if (!c) return fail(IALS_EINVAL, "bad context");
    IALS_CUDA(residual_enqueue(c), "residual recompute");
    c->e_stale = false;
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return IALS_OK;
}

ials_status ials_block_step(ials_ctx *c, int32_t side, int32_t block) {
    if (!c || side < 0 || side > 1 || block < 0 || block >= c->p.d / c->p.b)
        return fail(IALS_EINVAL, "bad side or block");
    if (c->p.b > 256) return fail(IALS_EINVAL, "block steps need b <= 256 (at b = d above 256 the epoch runs iALS)");
    IALS_CUDA(cudaMemsetAsync(c->stats, 0, 2 * sizeof(int64_t), c->stream), "stats reset");
    IALS_CUDA(ensure_residuals(c), "residual recompute");
    ials_status st = step_enqueue(c, side, block);
    if (st != IALS_OK) return st;
    return finish(c);
}

ials_status ials_get_residuals(ials_ctx *c, float *e) {
    if (!c || !e) return fail(IALS_EINVAL, "bad arguments");
    IALS_CUDA(ensure_residuals(c), "residual recompute");
    IALS_CUDA(cudaMemcpyAsync(e, c->e, sizeof(float) * (size_t)c->nnz, cudaMemcpyDefault, c->stream),
              "copy residuals out");
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    return IALS_OK;
}

ials_status ials_last_stats(ials_ctx *c, int64_t *n_fp64_retry, int64_t *n_not_pd) {
    if (!c) return fail(IALS_EINVAL, "bad context");
    int64_t st[2];
    IALS_CUDA(cudaMemcpy(st, c->stats, sizeof(st), cudaMemcpyDeviceToHost), "stats");
    if (n_fp64_retry) *n_fp64_retry = st[0];
    if (n_not_pd) *n_not_pd = st[1];
    return IALS_OK;
}

ials_status ials_profile_epochs(ials_ctx *c, int32_t n_epochs, double *kernel_ms,
                                int64_t *launches, int32_t n_kinds, double *total_ms) {
    if (!c || n_epochs < 0 || n_kinds < 0 || (n_kinds > 0 && (!kernel_ms || !launches)))
        return fail(IALS_EINVAL, "bad profiling arguments");
    Profiler prof;
    IALS_CUDA(cudaMemsetAsync(c->stats, 0, 2 * sizeof(int64_t), c->stream), "stats reset");
    IALS_CUDA(cudaStreamSynchronize(c->stream), "synchronize");
    prof_mark(&prof, -1, c->stream);
    for (int t = 0; t < n_epochs; ++t) {
        ials_status st = epoch_enqueue(c, &prof);
        if (st != IALS_OK) return st;
    }
    if (n_epochs > 0) c->e_stale = use_ials(c) || use_icd(c);
    prof_mark(&prof, -1, c->stream);
    ials_status st = finish(c);
    if (st != IALS_OK && st != IALS_ENOTPD) return st;
    for (int k = 0; k < n_kinds; ++k) { kernel_ms[k] = 0.0; launches[k] = 0; }
    for (size_t i = 0; i + 1 < prof.ev.size(); ++i) {
        const int k = prof.kind[i];
        if (k < 0 || k >= n_kinds) continue;
        float ms = 0.f;
        IALS_CUDA(cudaEventElapsedTime(&ms, prof.ev[i], prof.ev[i + 1]), "event time");
        kernel_ms[k] += ms;
        launches[k] += 1;
    }
    if (total_ms) {
        float ms = 0.f;
        IALS_CUDA(cudaEventElapsedTime(&ms, prof.ev.front(), prof.ev.back()), "event time");
        *total_ms = ms;
    }
    return st;
}

ials_status ials_work_model(ials_ctx *c, double *bytes, double *flops, int32_t n_kinds) {
    if (!c || !bytes || !flops || n_kinds < 0) return fail(IALS_EINVAL, "bad arguments");
    double B[K_COUNT] = {0}, F[K_COUNT] = {0};
    const double d = c->p.d, b = c->p.b, nb = c->p.d / c->p.b, nnz = (double)c->nnz;
    const double nu = c->n_users, ni = c->n_items;
    // residual recompute: index, y (if given), residual write, w_u once per row, h_i per interaction
    B[K_RESIDUAL] = nnz * (4 + 4 + 4 * d + (c->y ? 4 : 0)) + nu * (8 + 4 * d);
    F[K_RESIDUAL] = 2 * d * nnz;
    for (int sd = 0; sd < 2; ++sd) {
        const SideDev &S = c->side[sd];
        const double rows = S.n_rows, fixed = sd == 0 ? ni : nu;
        const double per_nz_read = 4 + 4 * b + 4 + (sd == 1 ? 4 : 0) + (c->alpha ? 4 : 0);
        // Gramian: the fixed side read once, G written (Eq. 10)
        B[K_GRAM] += nb * (fixed * d * 4 + d * b * 4);
        F[K_GRAM] += nb * 2 * fixed * d * b;
        // row terms: x_r read, G read, R written
        B[K_ROWTERM] += nb * (rows * d * 4 + d * b * 4 + rows * (b * 4 + 8));
        F[K_ROWTERM] += nb * 2 * rows * d * b;
        // sparse: per interaction index, slice, residual (+ position map, weight);
        // unsplit rows also write the residual, read R and read/write x_{r,pi}
        const double nz_u = (double)c->nnz_unsplit[sd], nz_s = (double)c->nnz_split[sd];
        const double r_u = (double)c->rows_unsplit[sd];
        B[K_SPARSE] += nb * (nz_u * (per_nz_read + 4) + nz_s * per_nz_read +
                             r_u * (4 * b + 8 * b + 16) + S.n_tasks * (double)sizeof(Task));
        F[K_SPARSE] += nb * ((nz_u + nz_s) * (b * b + 3 * b) + nz_u * 2 * b +
                             r_u * (b * b * b / 3 + 2 * b * b));
        B[K_SPLIT_SOLVE] += nb * (S.n_slots * (b * b + b) * 4 + S.n_split * (4 * b + 12 * b + 24));
        F[K_SPLIT_SOLVE] += nb * (S.n_slots * (b * b + b) + S.n_split * (b * b * b / 3 + 2 * b * b));
        if (S.split_pos && (int64_t)S.n_split * b * 4 <= kScanSmemMax)  // user-major list
            B[K_SPLIT_RESID] += nb * (nz_s * (8 + 8) + nu * (8 + 4 * b) + S.n_split * 4.0 * b);
        else
            B[K_SPLIT_RESID] += nb * (nz_s * (4 + 4 * b + 8 + (sd == 1 ? 4 : 0)) +
                                      S.n_stasks * ((double)sizeof(Task) + 4 * b));
        F[K_SPLIT_RESID] += nb * nz_s * 2 * b;
    }
    for (int k = 0; k < n_kinds; ++k) {
        bytes[k] = k < K_COUNT ? B[k] : 0.0;
        flops[k] = k < K_COUNT ? F[k] : 0.0;
    }
    return IALS_OK;
}

ials_status ials_partial_gramian_bf16(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                                      float *G, void *cuda_stream) {
    if (!X || !G || n < 0 || d < 8 || d % 8 != 0 || (bs != 16 && bs != 32 && bs != 64 && bs != 128) || p0 < 0 ||
        p0 % 8 != 0 || p0 + bs > d)
        return fail(IALS_EINVAL, "bad BF16 Gramian arguments (d % 8 == 0, bs in {16, 32, 64, 128}, p0 % 8 == 0)");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t count = n * (int64_t)d;
    const int64_t wsn = std::max<int64_t>(gram_tc_ws_floats(n, d, bs), 1);
    void *buf = nullptr;
    const size_t bytes = sizeof(__nv_bfloat16) * 2 * (size_t)std::max<int64_t>(count, 1) + sizeof(float) * wsn + 256;
    if (cudaMalloc(&buf, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(IALS_ENOMEM, "BF16 Gramian workspace");
    }
    __nv_bfloat16 *hi = static_cast<__nv_bfloat16 *>(buf), *lo = hi + std::max<int64_t>(count, 1);
    float *ws = reinterpret_cast<float *>(lo + std::max<int64_t>(count, 1));
    int32_t *err = reinterpret_cast<int32_t *>(ws + wsn);
    GramMaps maps;
    ials_status st = IALS_OK;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_split_bf16(X, count, hi, lo, s);
    if (e == cudaSuccess && n > 0 && !make_gram_maps(maps, hi, lo, n, d, bs)) st = fail(IALS_ECUDA, "tensor maps");
    if (e == cudaSuccess && st == IALS_OK) e = launch_gram_tc(maps, n, d, p0, bs, G, ws, err, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    int32_t derr = 0;
    if (e == cudaSuccess && e2 == cudaSuccess) cudaMemcpy(&derr, err, sizeof(derr), cudaMemcpyDeviceToHost);
    cudaFree(buf);
    if (st != IALS_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "BF16 partial Gramian");
    if (e2 != cudaSuccess) return cuda_fail(e2, "synchronize");
    if (derr) return fail(IALS_ETIMEDOUT, "a bounded device wait gave up");
    return IALS_OK;
}

ials_status ials_partial_gramian(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                                 float *G, void *cuda_stream) {
    if (!X || !G || n < 0 || d < 1 || bs < 1 || p0 < 0 || p0 + bs > d)
        return fail(IALS_EINVAL, "bad Gramian arguments");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    IALS_CUDA(dense_prepare(), "kernel attributes");
    float *ws = nullptr;
    const int64_t wsn = gram_ws_floats(n, d, bs);
    if (cudaMalloc(&ws, sizeof(float) * (size_t)std::max<int64_t>(wsn, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(IALS_ENOMEM, "Gramian workspace");
    }
    cudaError_t e = launch_gram(X, n, d, p0, bs, G, ws, s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(ws);
    if (e != cudaSuccess) return cuda_fail(e, "partial Gramian");
    if (e2 != cudaSuccess) return cuda_fail(e2, "synchronize");
    return IALS_OK;
}

}  // extern "C"
