/*
 * ials.h — C ABI of the GB300 iALS++ library (libials.so).
 *
 * iALS++ (Rendle, Krichene, Zhang, Koren, arXiv 2110.14044) learns the
 * implicit-feedback matrix factorisation yhat(u,i) = <w_u, h_i> (Eq. 1) by
 * minimising
 *
 *   L(W,H) = sum_{(u,i,y,a) in S} a (yhat(u,i) - y)^2
 *          + alpha0 sum_{u in U} sum_{i in I} yhat(u,i)^2
 *          + sum_u lambda_u |w_u|^2 + sum_i lambda_i |h_i|^2          (Eq. 2)
 *
 * with lambda_r = lambda (1 + nu |S_r|) (nu = 0 gives Eq. 2 as printed), by
 * subspace coordinate descent: Algorithm 3 visits the coordinate blocks
 * pi = [k b, (k+1) b) in order and, per block, solves every user's and then
 * every item's b-dimensional sub-problem exactly with one Newton step
 * (Eqs. 8-9, sufficient statistics Eqs. 10-12).
 *
 * Conventions shared by every entry point:
 *  - Every call returns an ials_status; nothing throws across the ABI.  On an
 *    error, ials_last_error() returns a message for the calling thread.
 *  - Array arguments may be host or device pointers (told apart with
 *    cudaPointerGetAttributes).  Inputs are copied; the caller keeps ownership
 *    of its arrays.  The library owns W, H, residuals and all workspaces until
 *    ials_destroy / ials_foldin_close.
 *  - Matrices are row-major float32: W is n_users x d, H is n_items x d.
 *  - All device work of a context runs on the stream given at creation (NULL:
 *    a private stream that orders with the legacy default stream; the legacy
 *    stream itself cannot be captured into a CUDA graph).  Calls on one context must not overlap
 *    (a context is single-threaded); submit/poll on a fold-in server are
 *    thread-safe.
 *  - The library runs on the current CUDA device at creation time; it needs an
 *    sm_103a GPU and fails with IALS_ECUDA otherwise.
 */
#ifndef IALS_H
#define IALS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ials_ctx ials_ctx;
typedef struct ials_srv ials_srv;

typedef enum {
    IALS_OK = 0,
    IALS_EINVAL = 1,     /* bad argument or inconsistent input */
    IALS_ENOMEM = 2,     /* device or host allocation failed */
    IALS_ECUDA = 3,      /* a CUDA call failed (message in ials_last_error) */
    IALS_ENOTPD = 4,     /* some row's Hessian was not positive definite even in FP64 */
    IALS_EAGAIN = 5,     /* fold-in: not admitted now / result pending */
    IALS_ETIMEDOUT = 6,  /* fold-in: poll deadline passed */
    IALS_ENOTFOUND = 7   /* fold-in: unknown ticket */
} ials_status;

/* Arithmetic of the block step. */
enum {
    IALS_PREC_FP32 = 0,  /* FP32 everywhere (FP64 objective, FP64 retry of failed pivots) */
    IALS_PREC_BF16 = 1   /* BF16 tensor-core statistics: x = hi + lo split into two bf16,
                          * products hi*hi + hi*lo + lo*hi accumulated in FP32 (about 16
                          * bits); weighted interactions enter as rows scaled by
                          * sqrt(alpha); FP32 solve with FP64 retry, FP64 objective.
                          * At b = 128 the row statistics are FP32 (register tiles,
                          * measured faster there); the Gramian and row terms stay
                          * on the tensor cores.  Needs b in {16, 32, 64, 128} and
                          * d % 8 == 0. */
};

/* ials_params.flags */
enum {
    IALS_FLAG_GRAPH = 1,      /* capture one epoch as a CUDA graph and replay it */
    IALS_FLAG_FORCE_FP64 = 2, /* fault injection: treat every FP32 pivot as failed */
    IALS_FLAG_GENERAL = 4     /* run the general block path also at the end points b = 1
                               * (otherwise iCD, Algorithm 2) and b = d (otherwise iALS,
                               * Algorithm 1) */
};

typedef struct {
    int32_t d;          /* embedding dimension; multiple of 4, 4 <= d <= 4096 */
    int32_t b;          /* block size |pi|; a power of two <= 256 that divides d (BF16: 16 .. 128),
                         * or, FP32 only, b = d for d a multiple of 64 up to 1024 (iALS,
                         * Algorithm 1; ials_block_step then refuses) */
    double alpha0;      /* weight of the all-pairs term, >= 0 */
    double lambda;      /* L2 weight, >= 0 */
    double nu;          /* regularisation scaling: lambda_r = lambda (1 + nu |S_r|), >= 0 */
    double init_std;    /* W, H drawn N(0, init_std^2) at creation (seeded) */
    uint64_t seed;
    int32_t precision;  /* IALS_PREC_* */
    int32_t flags;      /* IALS_FLAG_* */
    int32_t split_len;  /* work decomposition: a row with more interactions than this is cut
                         * into chunks (about equal, multiples of 32) whose statistics are
                         * summed in chunk order; 0 = the library's choice from nnz
                         * (clamp(nnz / 4864, 256, 8192)); else 32 <= split_len <= 2^24.
                         * Ignored by ials_foldin_open. */
    int32_t reserved;   /* must be 0 */
} ials_params;

/* Create a training context (Section 2 problem setting, Algorithm 3 state).
 *
 * S is given user-major: u_indptr (n_users + 1, int64, u_indptr[0] = 0,
 * non-decreasing, u_indptr[n_users] = nnz) and u_items (nnz, int32 item ids in
 * [0, n_items), no repeats within a row).  i_indptr / i_users may give the
 * item-major view; if non-NULL it must hold exactly the same pairs (any order
 * within a row), else IALS_EINVAL.  If NULL the library builds it.
 * y and alpha are per interaction in user-major order; NULL means all ones
 * (binary implicit feedback).  alpha must be finite and > 0, y finite.
 * nnz must be < 2^31.  cuda_stream is a cudaStream_t (see the stream convention above).
 * On success *out receives the context; W and H hold the seeded initial draw. */
ials_status ials_create(const ials_params *params, int32_t n_users, int32_t n_items,
                        int64_t nnz, const int64_t *u_indptr, const int32_t *u_items,
                        const int64_t *i_indptr, const int32_t *i_users, const float *y,
                        const float *alpha, void *cuda_stream, ials_ctx **out);

/* Release every device and host resource of the context (NULL is a no-op). */
ials_status ials_destroy(ials_ctx *ctx);

/* Run n_epochs epochs of Algorithm 3: recompute the residual cache, then for
 * each block pi the user pass followed by the item pass.  If objective_after
 * is non-NULL it receives L(W,H) (FP64) after the last epoch.  Returns
 * IALS_ENOTPD if some row could not be solved even in FP64 (that row keeps its
 * old value); the epoch still completes. */
ials_status ials_epoch(ials_ctx *ctx, int32_t n_epochs, double *objective_after);

/* L(W,H) of Eq. 2 (with lambda_r), accumulated in FP64, from the current W, H. */
ials_status ials_objective(ials_ctx *ctx, double *out);

/* Copy W (n_users x d) and/or H (n_items x d) out; either pointer may be NULL. */
ials_status ials_get_factors(ials_ctx *ctx, float *W, float *H);

/* Overwrite W and/or H (either may be NULL); the residual cache is recomputed
 * from them before it is next read (an epoch recomputes it first anyway, and
 * ials_block_step / ials_get_residuals do so when the factors were replaced).
 * Used to resume from a checkpoint taken at an epoch boundary (Algorithm 3
 * recomputes the cache per epoch, so resuming is exact).  The host buffers
 * may be reused when the call returns. */
ials_status ials_set_factors(ials_ctx *ctx, const float *W, const float *H);

/* --- single steps of Algorithm 3 (for step-level checks and profiling) --- */

/* Residual cache e(u,i) = yhat(u,i) - y for all of S ("Compute yhat",
 * Algorithm 3; Eq. 1).  Stored unweighted, in user-major order. */
ials_status ials_recompute_residuals(ials_ctx *ctx);

/* One block-side step of Algorithm 3: side 0 updates users (fixed side H),
 * side 1 updates items (fixed side W); block k covers coordinates
 * [k b, (k+1) b).  Partial Gramian (Eq. 10), row terms and sparse statistics
 * (Eqs. 11-12), Newton solve, apply, and in-place residual update. */
ials_status ials_block_step(ials_ctx *ctx, int32_t side, int32_t block);

/* Copy the residual cache (nnz floats, user-major order) out. */
ials_status ials_get_residuals(ials_ctx *ctx, float *e);

/* Counters of the last ials_block_step / ials_epoch: rows re-solved in FP64
 * after a failed FP32 pivot, and rows left unchanged (not positive definite). */
ials_status ials_last_stats(ials_ctx *ctx, int64_t *n_fp64_retry, int64_t *n_not_pd);

/* Kernel kinds of ials_profile_epochs. */
enum {
    IALS_K_RESIDUAL = 0,     /* residual cache recompute */
    IALS_K_GRAM = 1,         /* partial Gramian (tile + reduce) */
    IALS_K_ROWTERM = 2,      /* alpha0 x_r G + lambda_r x_{r,pi} */
    IALS_K_SPARSE = 3,       /* sparse statistics, solve, apply, residual update */
    IALS_K_SPLIT_SOLVE = 4,  /* long rows: reduce partial statistics and solve */
    IALS_K_SPLIT_RESID = 5,  /* long rows: residual update */
    IALS_K_RETRY = 6,        /* FP64 re-solve of failed pivots */
    IALS_K_OBJECTIVE = 7,
    IALS_K_COUNT = 8
};

/* Measurement: run n_epochs epochs without graph capture, with a CUDA event
 * recorded on the context's stream before and after every kernel launch (or
 * launch pair, for the Gramian).  kernel_ms[k] and launches[k] (k < n_kinds)
 * receive the summed device time and the launch count per kind;
 * *total_ms (if non-NULL) the time from the first to the last event.
 * Returns like ials_epoch. */
ials_status ials_profile_epochs(ials_ctx *ctx, int32_t n_epochs, double *kernel_ms,
                                int64_t *launches, int32_t n_kinds, double *total_ms);

/* Algorithmic work of one epoch per kernel kind, from the context's own work
 * decomposition: bytes[k] = bytes a kernel of kind k must move (indices,
 * residuals, gathered b-slices of the fixed side, rows read and written),
 * flops[k] = floating-point operations counted as in the complexity analysis
 * (Table 1; symmetric b x b Hessian, b^3/3 Cholesky).  k < n_kinds. */
ials_status ials_work_model(ials_ctx *ctx, double *bytes, double *flops, int32_t n_kinds);

/* Partial Gramian G = X^T X[:, p0:p0+bs] (Eq. 10) of a row-major n x d float32
 * device matrix X into the d x bs row-major float32 device array G, on the
 * given stream, with the library's split-K kernel (precision IALS_PREC_FP32).
 * Workspace is allocated internally per call.  Synchronous. */
ials_status ials_partial_gramian(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                                 float *G, void *cuda_stream);

/* Partial Gramian on the tcgen05 tensor cores (Eq. 10): X is split into BF16
 * hi/lo halves and G = Xh^T Xh_pi + Xh^T Xl_pi + Xl^T Xh_pi is accumulated in
 * FP32 (about 16 bits).  Needs d % 8 == 0, bs in {16, 32, 64, 128}, p0 % 8 == 0
 * (blocks wider than 32 columns are formed 32 columns at a time).
 * X (n x d float32) and G (d x bs float32) are device arrays; temporaries are
 * allocated per call.  Synchronous.  IALS_ETIMEDOUT if a bounded device wait
 * gave up. */
ials_status ials_partial_gramian_bf16(const float *X, int64_t n, int32_t d, int32_t p0, int32_t bs,
                                      float *G, void *cuda_stream);

/* The same partial Gramian for callers that cannot allocate device memory:
 * code whose device memory belongs to another allocator (a framework's caching
 * allocator, a fixed arena) or a latency-bound loop in which cudaMalloc /
 * cudaFree, which may synchronise the device, are not acceptable.  The paper
 * has no counterpart; this is a library convenience.
 * The split-K partial sums live in one fixed device array of 2^21 floats
 * (8 MiB) that every GPU loading the library holds until the process exits;
 * calls with d * bs > 2^21 fail with IALS_EINVAL.  X (n x d) and G (d x bs)
 * are caller-owned device (or managed) arrays; unlike the other calls, host
 * arrays are not copied but refused with IALS_EINVAL.  Nothing is allocated or freed: no
 * cudaMalloc, cudaFree or allocating library routine is called.
 * The call only enqueues work on cuda_stream and returns; G is ready when the
 * stream reaches that point.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one array and it
 * keeps the last call's contents: calls that overlap on the GPU (another
 * stream, another thread) race on it and give wrong results, so serialise
 * them.  Every partial slot is written before it is read, so no clearing is
 * needed between calls. */
ials_status ials_partial_gramian_noalloc(const float *X, int64_t n, int32_t d, int32_t p0,
                                         int32_t bs, float *G, void *cuda_stream);

/* --- fold-in serving ----------------------------------------------------
 * New users are solved against frozen item factors, as the evaluation protocol
 * of Section 5.1.1 does for held-out users.  The paper gives no procedure;
 * this library starts from w = 0 and runs `sweeps` passes of the user-side
 * block steps of Algorithm 3 with H and G^I = H^T H fixed and
 * lambda_u = lambda (1 + nu n).  One sweep with b = d is Eq. 3.
 *
 * ials_foldin_open copies H (n_items x d, host or device) to the device,
 * forms G^I, and reserves workspace_bytes of device memory for requests.
 * params->d and params->b (16, 32, 64 or 128, dividing d), alpha0, lambda, nu
 * apply; precision and flags are ignored (FP32).  cuda_stream is used for the
 * set-up only.  A scheduler thread batches requests continuously: queued
 * requests are admitted in arrival order whenever their device memory fits the
 * free workspace and one of four stream slots is free, so new requests start
 * while earlier ones are still running.  A request longer than 384
 * interactions is split over a cluster of 8 CTAs; each request is published as
 * soon as it finishes.  A request's result does not depend on the requests it
 * is batched with. */
ials_status ials_foldin_open(const float *H, int32_t n_items, const ials_params *params,
                             size_t workspace_bytes, int32_t sweeps, void *cuda_stream,
                             ials_srv **out);

/* Queue one request: n item ids (host array, each in [0, n_items)) and
 * optional labels y (host array, NULL = all ones; weights are 1).  Thread-safe.
 * Returns IALS_EAGAIN if the queue is full and IALS_EINVAL if the request can
 * never fit the workspace.  *ticket identifies the request for poll. */
ials_status ials_foldin_submit(ials_srv *srv, const int32_t *items, const float *y, int32_t n,
                               uint64_t *ticket);

/* Wait up to timeout_us microseconds (<= 0: do not wait) for a request.  On
 * IALS_OK, w_out (host, d floats) receives the embedding and the ticket is
 * released.  IALS_EAGAIN: not ready (timeout_us <= 0); IALS_ETIMEDOUT: not ready
 * within timeout_us; IALS_ENOTFOUND: unknown or already collected ticket;
 * IALS_ENOTPD: a block Hessian was not positive definite (ticket released);
 * IALS_ECUDA: the batch holding the request failed on the device (ticket
 * released).  Thread-safe. */
ials_status ials_foldin_poll(ials_srv *srv, uint64_t ticket, float *w_out, int32_t timeout_us);

/* ials_foldin_poll that also returns, in *latency_us (if non-NULL), the time
 * from the request's submission to the moment its result reached host memory,
 * both taken by the library with a monotonic clock. */
ials_status ials_foldin_poll_timed(ials_srv *srv, uint64_t ticket, float *w_out, int32_t timeout_us,
                                   double *latency_us);

/* How a finished request was served (ials_foldin_poll_info). */
typedef struct {
    double latency_us;   /* submission to result in host memory, monotonic clock */
    uint64_t batch;      /* id of the batch it ran in (batches are numbered from 1) */
    int32_t batch_size;  /* requests in that batch */
    int32_t cluster;     /* 1: longer than the library's limit for one CTA, run on a CTA cluster */
} ials_foldin_info;

/* ials_foldin_poll that also describes, in *info (if non-NULL, filled when the
 * result is returned), how the request was served: latency, batch and whether
 * its interactions were split over a cluster of CTAs.  Thread-safe. */
ials_status ials_foldin_poll_info(ials_srv *srv, uint64_t ticket, float *w_out, int32_t timeout_us,
                                  ials_foldin_info *info);

/* Stop the scheduler, drop queued requests and release everything (NULL: no-op).
 * No other thread may be inside ials_foldin_submit / _poll on srv meanwhile. */
ials_status ials_foldin_close(ials_srv *srv);

/* Message of the last failed call on this thread ("" if none). */
const char *ials_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IALS_H */
