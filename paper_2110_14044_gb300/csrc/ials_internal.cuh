// Internal declarations shared by the CUDA translation units of libials.
// Nothing here is part of the public ABI (see include/ials.h).
#pragma once

#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace ials {

// Kernel kinds reported by the profiling entry point (must match include/ials.h).
enum KernelKind {
    K_RESIDUAL = 0, K_GRAM = 1, K_ROWTERM = 2, K_SPARSE = 3, K_SPLIT_SOLVE = 4,
    K_SPLIT_RESID = 5, K_RETRY = 6, K_OBJECTIVE = 7, K_COUNT = 8
};

// Host-side event marks around kernel launches (measurement only).  mark(k)
// opens a segment of kind k (k < 0: a gap that is not attributed).
struct Profiler {
    std::vector<cudaEvent_t> ev;
    std::vector<int> kind;
    cudaError_t mark(int k, cudaStream_t s) {
        cudaEvent_t e;
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) return err;
        ev.push_back(e);
        kind.push_back(k);
        return cudaEventRecord(e, s);
    }
    ~Profiler() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

inline void prof_mark(Profiler *p, int k, cudaStream_t s) {
    if (p) p->mark(k, s);
}

#ifdef __CUDACC__
// x = v for one coordinate, keeping the BF16 hi/lo shadow current (BF16 mode).
__device__ __forceinline__ void set_value(float *X, __nv_bfloat16 *Xh, __nv_bfloat16 *Xl, int64_t i, float v) {
    X[i] = v;
    if (Xh) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        Xh[i] = h;
        Xl[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

// x -= delta for one coordinate, keeping the BF16 hi/lo shadow current (BF16 mode).
__device__ __forceinline__ void apply_delta(float *X, __nv_bfloat16 *Xh, __nv_bfloat16 *Xl,
                                            int64_t i, float delta) {
    const float x = X[i] - delta;
    X[i] = x;
    if (Xh) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        Xh[i] = h;
        Xl[i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}
#endif

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;
// shared memory for the delta table of the user-major split-row residual scan
constexpr int kScanSmemMax = 200 * 1024;

// One unit of sparse work: a whole row, or a chunk of a long ("split") row.
struct Task {
    int64_t begin;  // first CSR position
    int32_t len;    // number of interactions
    int32_t row;    // row being updated
    int32_t slot;   // partial-statistics slot for split rows, -1 otherwise
    int32_t srow;   // index into the split-row table for split rows, -1 otherwise
};

// A row whose statistics are accumulated by several tasks.
struct SplitRow {
    int64_t begin;   // CSR range of the whole row
    int32_t len;
    int32_t row;
    int32_t slot0;   // first partial slot; the row owns [slot0, slot0 + nslots)
    int32_t nslots;
};

// Arguments of one block-side step (side = users or items).
struct StepArgs {
    // CSR of the side being updated: rows of this side, column ids index the fixed side
    const int64_t *ptr;
    const int32_t *idx;
    const int32_t *pos;     // side 1: CSR position -> user-major residual index; nullptr on side 0
    float *e;               // residual cache r = yhat - y, user-major order
    const float *alpha;     // per interaction weights (user-major) or nullptr
    const float *y;         // per interaction labels (user-major) or nullptr (all ones)
    float *X;               // updated side, n_rows x d
    const float *F;         // fixed side, n_fixed x d
    // BF16 mode: hi/lo shadows (x = hi + lo to ~16 bits) of the updated and fixed sides;
    // nullptr in FP32 mode
    __nv_bfloat16 *Xh, *Xl;
    const __nv_bfloat16 *Fh, *Fl;
    const float *G;         // partial Gramian of F, d x b (row-major)
    const float *R;         // row terms alpha0 x_r G + lambda_r x_{r,pi}, n_rows x b
    int32_t n_rows, d, b, p0;
    float alpha0, lambda, nu;
    // work decomposition
    const Task *tasks;
    int32_t n_tasks;
    const SplitRow *split;
    int32_t n_split;
    const Task *stasks;     // the tasks of split rows (for the residual update)
    int32_t n_stasks;
    float *part;            // split partials: slot -> (b*b Hessian, b gradient)
    float *delta;           // split rows: srow -> delta (b)
    int32_t *counter;       // work-stealing counter (zeroed before launch)
    int32_t *retry;         // [0] = count, [1..] = rows to redo in FP64
    int64_t *stats;         // [0] = FP64 retries, [1] = not positive definite
    int32_t force_fp64;     // fault injection: every FP32 pivot counts as failed
    int32_t direct;         // b = d (Algorithm 1): solve for x_r itself from sum alpha y f, no residuals
    double *retry_ws;       // b > 128: FP64 systems of the re-solve kernel's blocks
    float *big_ws;          // b = d > 256: per-block row systems of the iALS kernel
    double *big_ws64;       // and of its FP64 re-solve
    // item side with split rows: the user-major view, for the split rows' residual
    // update in user-major order (nullptr / 0 otherwise)
    const int64_t *optr;      // user CSR row pointers (n_orows + 1)
    const int32_t *split_pos; // user-major positions whose item is a split row, increasing
    const int32_t *split_row; // the split row of each
    int64_t n_spos;           // entries of the two lists
    int32_t n_orows;          // users
    Profiler *prof;         // host only: event marks around launches, or nullptr
};

// One iCD pass (b = 1, Algorithm 2) over one side for coordinate f
// (k_icd.cu).  part holds two floats per chunk slot, delta one per long row.
struct IcdArgs {
    StepArgs s;
    int32_t f;           // coordinate updated by the pass
    int32_t fn;          // column of the updated side's Gramian formed on the way (-1: none)
    const float *g_in;   // column f of the fixed side's Gramian (d floats)
    float *g_out;        // column fn of the updated side's Gramian after the pass (d floats)
    float *gpart;        // partial columns: icd_row_grid blocks, then icd_split_grid blocks (d each)
    int32_t *done;       // completion counter of the final reduction (0 between passes)
    int32_t grid;        // blocks of the row kernel: icd_row_grid(n_tasks, d)
    const float *FT;     // fixed side transposed, d x n_fixed
    float *XT;           // updated side transposed, d x n_rows (kept current)
    int64_t n_fixed;
    float *eo;           // residuals in this side's CSR order
    const float *alpha_o;  // weights in this side's CSR order, or nullptr
    const float *dprev;  // deltas of the previous pass (other side, by column id), or nullptr
    int32_t fprev;       // coordinate of the updated row that dprev multiplies
    float *dself;        // this pass's delta per row (n_rows)
    float *xold;         // long rows: the fprev coordinate before the update (n_split)
};
int32_t icd_row_grid(int32_t n_tasks, int32_t d);
int32_t icd_split_grid(int32_t n_split, int32_t d);
// X (n x d) -> XT (d x n)
cudaError_t launch_transpose(const float *X, int64_t n, int32_t d, float *XT, cudaStream_t s);
// dst[t] = src[pos[t]] and dst[pos[t]] = src[t], t < n
cudaError_t launch_perm_gather(const float *src, const int32_t *pos, int64_t n, float *dst, cudaStream_t s);
cudaError_t launch_perm_scatter(const float *src, const int32_t *pos, int64_t n, float *dst, cudaStream_t s);
cudaError_t launch_icd(const IcdArgs &a, cudaStream_t s);
// Kernel attributes of the iCD kernels; call once outside any stream capture.
cudaError_t icd_prepare();

// One fold-in request inside the server's workspace arena (byte offsets; the
// items start at arena + off, the others are relative to that).
struct FoldReq {
    int64_t off, y_off, e_off, l_off, w_off;
    int32_t n, has_y;
};

struct FoldArgs {
    const FoldReq *req;
    int32_t n_req;
    const int32_t *list;  // the requests this launch serves (indices into req)
    int32_t n_list;
    uint8_t *arena;
    const float *H;   // frozen item factors, n_items x d
    const float *G;   // G^I = H^T H, d x d
    int32_t d, b, sweeps;
    float alpha0, lambda, nu;
    int32_t *status;     // per request: 0 ok, 4 not positive definite
    float *w_host;       // mapped host memory: the embeddings, n_req x d
    int32_t *done_host;  // mapped host memory: per request 1 + status once finished
};
// Requests longer than kFoldLong interactions run on a cluster of kFoldCluster CTAs.
constexpr int kFoldLong = 384;
constexpr int kFoldCluster = 8;

// ---------------------------------------------------------------- launchers
// dense kernels (k_dense.cu)
// e = W H^T - y over the user-side task list (persistent, work-stealing over an
// atomic counter, which the launcher zeroes on the stream first).
cudaError_t launch_residual_tasks(const Task *tasks, int32_t n_tasks, const int32_t *u_idx,
                                  const float *W, const float *H, const float *y, int32_t d, float *e,
                                  int32_t *counter, cudaStream_t s);
// Sum over S of alpha (yhat - y)^2 in FP64, recomputing yhat from W, H.
// Writes one double per block into part (n_part >= grid) and the total into out.
cudaError_t launch_sq_loss(const int64_t *u_ptr, const int32_t *u_idx, const float *W,
                           const float *H, const float *y, const float *alpha,
                           int32_t n_users, int32_t d, double *part, int32_t n_part,
                           double *out, cudaStream_t s);
// sum_r lambda (1 + nu n_r) |x_r|^2 in FP64 -> out (adds to *out if accumulate)
cudaError_t launch_reg_loss(const int64_t *ptr, const float *X, int32_t n_rows, int32_t d,
                            double lambda, double nu, double *part, int32_t n_part,
                            double *out, cudaStream_t s);
// <A, B>_F of two d x d FP64 matrices -> *out += result
cudaError_t launch_frobenius(const double *A, const double *B, int32_t n, double alpha0,
                             double *out, cudaStream_t s);

// Kernel attributes of the dense kernels; call once outside any stream capture.
cudaError_t dense_prepare();
// Split-K partial Gramian G = X^T X[:, p0:p0+bs] (d x bs).
// ws must hold gram_ws_floats(n, d, bs) floats.
int64_t gram_ws_floats(int64_t n, int32_t d, int32_t bs);
cudaError_t launch_gram(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs, float *G,
                        float *ws, cudaStream_t s);
// The same split-K Gramian with a caller-provided workspace of max_floats
// floats: the row ranges are lengthened until the partials fit.
// gram_ws_floats_capped returns the floats used, or -1 if d * bs > max_floats.
int64_t gram_ws_floats_capped(int64_t n, int32_t d, int32_t bs, int64_t max_floats);
cudaError_t launch_gram_capped(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                               float *G, float *ws, int64_t max_floats, cudaStream_t s);
// Full FP64-accumulated Gramian G64 = X^T X (d x d); ws holds gram64_ws_doubles(n, d).
int64_t gram64_ws_doubles(int64_t n, int32_t d);
cudaError_t launch_gram64(const float *X, int64_t n, int32_t d, double *G64, double *ws,
                          cudaStream_t s);

// tcgen05 partial Gramian (k_tc_gram.cu): TMA descriptors of one BF16 hi/lo pair
// (opaque CUtensorMap storage) and the launcher; err receives a nonzero code if
// a bounded wait gave up.
struct alignas(64) GramMaps {
    unsigned char ah[128], al[128], bh[128], bl[128];
};
// Columns col0 .. col0+cols-1 of G (row stride ldg) = fixed-order sum of nsplit
// partial rows x cols blocks.
cudaError_t launch_gram_reduce_cols(const float *ws, int nsplit, int32_t rows, int32_t cols, float *G, int32_t ldg,
                                    int32_t col0, cudaStream_t s);
bool make_gram_maps(GramMaps &g, const __nv_bfloat16 *hi, const __nv_bfloat16 *lo, int64_t rows, int32_t d,
                    int32_t b);
int64_t gram_tc_ws_floats(int64_t n, int32_t d, int32_t bs);
// tcgen05 row terms: tensor maps of the updated side's hi/lo shadows (K-major
// boxes of 64 x 128) and of G^T hi/lo (b x d); the launcher first writes G^T.
struct alignas(64) RowMaps {
    unsigned char xh[128], xl[128], gh[128], gl[128];
};
bool make_row_maps(RowMaps &m, const __nv_bfloat16 *xh, const __nv_bfloat16 *xl, int64_t rows, int32_t d,
                   const __nv_bfloat16 *gth, const __nv_bfloat16 *gtl, int32_t b);
cudaError_t launch_rowterm_tc(const RowMaps &m, const float *G, __nv_bfloat16 *gth, __nv_bfloat16 *gtl,
                              const float *X, const int64_t *ptr, int32_t n_rows, int32_t d, int32_t p0, int32_t b,
                              float alpha0, float lambda, float nu, float *R, int32_t *err, cudaStream_t s);
cudaError_t launch_gram_tc(const GramMaps &g, int64_t n, int32_t d, int32_t p0, int32_t bs, float *G, float *ws,
                           int32_t *err, cudaStream_t s);

// Row terms R[r] = alpha0 * X[r] G + lambda (1 + nu n_r) X[r, p0:p0+bs]  (n_rows x bs)
cudaError_t launch_rowterm(const float *X, const int64_t *ptr, int32_t n_rows, int32_t d,
                           int32_t p0, int32_t bs, const float *G, float alpha0, float lambda,
                           float nu, float *R, cudaStream_t s);
// BF16 hi/lo split of count floats: hi = bf16(x), lo = bf16(x - hi)
cudaError_t launch_split_bf16(const float *X, int64_t count, __nv_bfloat16 *hi, __nv_bfloat16 *lo,
                              cudaStream_t s);
// N(0, std^2) draws from a counter-based hash (SplitMix64 + Box-Muller)
cudaError_t launch_init_normal(float *X, int64_t count, double std, uint64_t seed,
                               uint64_t stream_id, cudaStream_t s);

// sparse kernels (k_sparse_b*.cu): statistics, solve, apply and residual
// update of one block-side step for block size B (1, 2, 4, 8, 16, 32).
cudaError_t launch_sparse_b1(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b2(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b4(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b8(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b16(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b32(const StepArgs &a, cudaStream_t s);
// block sizes 64, 128 and 256 (k_sparse_b64.cu, k_sparse_b128.cu, k_sparse_b256.cu)
cudaError_t launch_sparse_b64(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b128(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_b256(const StepArgs &a, cudaStream_t s);
// iALS at b = d above 256 (k_ials_big.cu): d a multiple of 64 up to 1024, FP32 with
// an FP64 re-solve; row systems in global workspaces of the given sizes
bool ials_big_supported(int32_t d);
int64_t ials_big_ws_floats(int32_t d);
int64_t ials_big_ws_doubles(int32_t d);
cudaError_t ials_big_prepare();  // kernel attributes; call once outside any stream capture
cudaError_t launch_ials_big(const StepArgs &a, cudaStream_t s);
// doubles of FP64 re-solve workspace a block size needs (0 up to b = 128)
int64_t sparse_retry_ws_doubles(int32_t b);
// fold-in (k_foldin.cu): one CTA per request, or (cluster) one cluster of
// kFoldCluster CTAs per request; factors per request: foldin_factor_floats
cudaError_t launch_foldin(const FoldArgs &a, bool cluster, cudaStream_t s);
int64_t foldin_factor_floats(int32_t d, int32_t b);
// BF16 mode (k_sparse_bf16.cu): tensor-core statistics for block sizes 16 and 32
cudaError_t launch_sparse_bf16_b16(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_bf16_b32(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_bf16_b64(const StepArgs &a, cudaStream_t s);
cudaError_t launch_sparse_bf16_b128(const StepArgs &a, cudaStream_t s);

}  // namespace ials
