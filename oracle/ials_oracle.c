/*
 * FP64 CPU oracle for iALS++ (Rendle, Krichene, Zhang, Koren: "iALS++: Speeding
 * up Matrix Factorization with Subspace Optimization", arXiv 2110.14044).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header or helper with the CUDA library.
 *
 * Everything is double precision.  Each routine follows one passage of the
 * paper in the paper's order and notation:
 *
 *   oracle_predict         yhat(u,i) = <w_u, h_i>                 (Eq. 1)
 *   oracle_objective       L(W,H) with the Gramian trick           (Eq. 2, Eq. 4)
 *   oracle_halfstep        one block pi, one side of Algorithm 3  (Eqs. 10-12)
 *   oracle_ialspp          T epochs of Algorithm 3
 *   oracle_row_step        one row of oracle_halfstep, read-only  (Eqs. 11-12)
 *   oracle_rows_step       the same for a list of rows
 *   oracle_ials            T epochs of Algorithm 1 (closed form, Eq. 3)
 *   oracle_icd             T epochs of Algorithm 2 (Eqs. 5-7)
 *   oracle_foldin          new-user solve against frozen H (Section 5.1.1
 *                          protocol; the paper does not give the procedure,
 *                          see the reading in oracle_foldin); oracle_foldin_g
 *                          takes G^I from oracle_gramian instead of forming it
 *
 * Readings of the paper that this file fixes:
 *  - The 1/2 in front of the gradient and Hessian cancels in the Newton step
 *    delta = (Hessian)^-1 gradient; the un-halved sums of Algorithm 3 are used.
 *  - G^{I,pi} = sum_i h_i (x) h_{i,pi} is d x |pi| (the paper's R^{I x |pi|} is a
 *    typo); its pi rows form G^{I,pi}_pi.
 *  - "+ lambda" in a Hessian means + lambda * identity.
 *  - Blocks are contiguous coordinate ranges [k b, min((k+1) b, d)), visited in
 *    increasing k, the same every epoch.
 *  - The item pass of a block uses the Gramian of W after that block's user
 *    pass ("perform a similar pass over the item side").
 *  - Regularisation is scaled per row: lambda_r = lambda (1 + nu |S_r|), with
 *    |S_r| the number of interactions of row r; nu = 0 gives Eq. 2 exactly.
 *    The same lambda_r enters the objective.
 *  - The prediction cache yhat is recomputed at the start of every epoch.
 *
 * Data: the interaction set S is given twice, user-major and item-major CSR
 * (row pointer int64, column index int32).  y and alpha are per interaction in
 * user-major order (NULL means 1).  i_pos maps each item-major entry to the
 * position of the same (u,i) pair in user-major order; oracle_build_pos fills it.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n_users, n_items;
    int64_t nnz;
    const int64_t *u_ptr;
    const int32_t *u_idx;
    const int64_t *i_ptr;
    const int32_t *i_idx;
    const int64_t *i_pos; /* item-major entry -> user-major entry */
    const double *y;      /* NULL = all ones */
    const double *alpha;  /* NULL = all ones */
    int32_t d, b;
    double alpha0, lambda, nu;
    int32_t n_threads;
} oracle_problem;

enum { ORACLE_OK = 0, ORACLE_EINVAL = 1, ORACLE_ENOMEM = 2, ORACLE_ENOTPD = 4 };

static double yv(const oracle_problem *P, int64_t s) { return P->y ? P->y[s] : 1.0; }
static double av(const oracle_problem *P, int64_t s) { return P->alpha ? P->alpha[s] : 1.0; }

/* ---------------------------------------------------------------- helpers */

/* Solve A x = r for symmetric positive definite A (n x n, row-major) by the
 * textbook Cholesky factorisation A = L L^T followed by two triangular solves.
 * A and r are overwritten (A by L, r by x).  Returns nonzero on a non-positive
 * pivot. */
static int cholesky_solve(double *A, double *r, int n) {
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return 1;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    for (int i = 0; i < n; ++i) { /* L z = r */
        double t = r[i];
        for (int k = 0; k < i; ++k) t -= A[i * n + k] * r[k];
        r[i] = t / A[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) { /* L^T x = z */
        double t = r[i];
        for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * r[k];
        r[i] = t / A[i * n + i];
    }
    return 0;
}

/* Simple static row partition over worker threads. */
typedef struct {
    void (*fn)(void *ctx, int64_t lo, int64_t hi, int tid);
    void *ctx;
    int64_t lo, hi;
    int tid;
} task_t;

static void *run_task(void *p) {
    task_t *t = (task_t *)p;
    t->fn(t->ctx, t->lo, t->hi, t->tid);
    return NULL;
}

static void parallel_for(int64_t n, int n_threads, void *ctx,
                         void (*fn)(void *, int64_t, int64_t, int)) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_threads == 1 || n < 2 * n_threads) {
        fn(ctx, 0, n, 0);
        return;
    }
    pthread_t th[256];
    task_t tk[256];
    for (int t = 0; t < n_threads; ++t) {
        tk[t].fn = fn;
        tk[t].ctx = ctx;
        tk[t].lo = n * t / n_threads;
        tk[t].hi = n * (t + 1) / n_threads;
        tk[t].tid = t;
        pthread_create(&th[t], NULL, run_task, &tk[t]);
    }
    for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* --------------------------------------------------------------- mapping */

/* For every item-major entry (i, u) find the position of (u, i) in user u's
 * row of the user-major CSR.  Returns ORACLE_EINVAL unless the two CSRs hold
 * exactly the same pairs (every pair found, no position used twice). */
int oracle_build_pos(int32_t n_users, int32_t n_items, const int64_t *u_ptr,
                     const int32_t *u_idx, const int64_t *i_ptr, const int32_t *i_idx,
                     int64_t *i_pos) {
    const int64_t nnz = u_ptr[n_users];
    if (i_ptr[n_items] != nnz) return ORACLE_EINVAL;
    char *used = calloc(nnz > 0 ? (size_t)nnz : 1, 1);
    if (!used) return ORACLE_ENOMEM;
    int status = ORACLE_OK;
    for (int32_t i = 0; i < n_items && status == ORACLE_OK; ++i) {
        for (int64_t s = i_ptr[i]; s < i_ptr[i + 1]; ++s) {
            int32_t u = i_idx[s];
            int64_t found = -1;
            if (u < 0 || u >= n_users) { status = ORACLE_EINVAL; break; }
            for (int64_t q = u_ptr[u]; q < u_ptr[u + 1]; ++q)
                if (u_idx[q] == i) { found = q; break; }
            if (found < 0 || used[found]) { status = ORACLE_EINVAL; break; }
            used[found] = 1;
            i_pos[s] = found;
        }
    }
    free(used);
    return status;
}

/* ------------------------------------------------------------- model, loss */

/* Eq. 1: yhat(u,i) = <w_u, h_i> for every (u,i) in S, in user-major order. */
void oracle_predict(const oracle_problem *P, const double *W, const double *H, double *yhat) {
    const int d = P->d;
    for (int32_t u = 0; u < P->n_users; ++u)
        for (int64_t s = P->u_ptr[u]; s < P->u_ptr[u + 1]; ++s) {
            const double *w = W + (int64_t)u * d, *h = H + (int64_t)P->u_idx[s] * d;
            double t = 0.0;
            for (int f = 0; f < d; ++f) t += w[f] * h[f];
            yhat[s] = t;
        }
}

/* Gramian of a row-major n x d matrix X: G = sum_j x_j (x) x_j (Eq. 4). */
static void gramian(const double *X, int64_t n, int d, double *G) {
    memset(G, 0, sizeof(double) * d * d);
    for (int64_t j = 0; j < n; ++j) {
        const double *x = X + j * d;
        for (int f = 0; f < d; ++f)
            for (int g = 0; g < d; ++g) G[f * d + g] += x[f] * x[g];
    }
}

/* Eq. 2, with the unobserved term over all |U| x |I| pairs evaluated as
 * <W^T W, H^T H>_F (the Gramian identity behind Eq. 4), and per-row lambda. */
double oracle_objective(const oracle_problem *P, const double *W, const double *H) {
    const int d = P->d;
    double obs = 0.0;
    for (int32_t u = 0; u < P->n_users; ++u)
        for (int64_t s = P->u_ptr[u]; s < P->u_ptr[u + 1]; ++s) {
            const double *w = W + (int64_t)u * d, *h = H + (int64_t)P->u_idx[s] * d;
            double yh = 0.0;
            for (int f = 0; f < d; ++f) yh += w[f] * h[f];
            double r = yh - yv(P, s);
            obs += av(P, s) * r * r;
        }
    double *GW = malloc(sizeof(double) * d * d), *GH = malloc(sizeof(double) * d * d);
    if (!GW || !GH) { free(GW); free(GH); return NAN; }
    gramian(W, P->n_users, d, GW);
    gramian(H, P->n_items, d, GH);
    double unobs = 0.0;
    for (int k = 0; k < d * d; ++k) unobs += GW[k] * GH[k];
    free(GW);
    free(GH);
    double reg = 0.0;
    for (int32_t u = 0; u < P->n_users; ++u) {
        double lam = P->lambda * (1.0 + P->nu * (double)(P->u_ptr[u + 1] - P->u_ptr[u]));
        double n2 = 0.0;
        for (int f = 0; f < d; ++f) n2 += W[(int64_t)u * d + f] * W[(int64_t)u * d + f];
        reg += lam * n2;
    }
    for (int32_t i = 0; i < P->n_items; ++i) {
        double lam = P->lambda * (1.0 + P->nu * (double)(P->i_ptr[i + 1] - P->i_ptr[i]));
        double n2 = 0.0;
        for (int f = 0; f < d; ++f) n2 += H[(int64_t)i * d + f] * H[(int64_t)i * d + f];
        reg += lam * n2;
    }
    return obs + P->alpha0 * unobs + reg;
}

/* ---------------------------------------------------- Algorithm 3 (iALS++) */

/* One side of one block of Algorithm 3.  side 0 updates W (rows = users, the
 * fixed side is H); side 1 updates H (rows = items, the fixed side is W). */
typedef struct {
    const oracle_problem *P;
    int side, p0, bs;
    double *Upd;         /* matrix being updated */
    const double *Fix;   /* fixed matrix */
    const double *G;     /* d x bs partial Gramian of Fix */
    double *yhat;        /* prediction cache, user-major order */
    double *scratch;     /* per thread: bs*bs + bs */
    int status;
} half_ctx;

/* The Newton system of one row's block (Eqs. 9, 11, 12).  The loss restricted
 * to x_{r,pi} is quadratic, so its minimiser is one Newton step: with the
 * (un-halved) gradient g and Hessian A of Eqs. 11-12, delta = A^-1 g and the
 * block moves to x_{r,pi} - delta (Eq. 9).  Both statistics split into a part
 * that involves every row of the fixed side only through the partial Gramian
 * G^{pi} (Eq. 10) and a part summed over the row's own interactions S_r. */

/* The Gramian part: g = alpha0 x_r G^{pi} + lambda_r x_{r,pi} (Eq. 11) and
 * A = alpha0 G^{pi}_{pi} + lambda_r I (Eq. 12, "+ lambda" read as lambda_r I). */
static void gramian_terms(const oracle_problem *P, int p0, int bs, const double *x,
                          const double *G, double lam, double *A, double *g) {
    const int d = P->d;
    for (int f = 0; f < bs; ++f) {
        double xg = 0.0;
        for (int k = 0; k < d; ++k) xg += x[k] * G[k * bs + f];
        g[f] = P->alpha0 * xg + lam * x[p0 + f];
        for (int q = 0; q < bs; ++q)
            A[f * bs + q] = P->alpha0 * G[(p0 + f) * bs + q] + (f == q ? lam : 0.0);
    }
}

/* The observed part, added on: for every interaction (r, c) of S_r with weight
 * alpha and label y, g += alpha (yhat - y) f_{c,pi} and A += alpha f_{c,pi}
 * f_{c,pi}^T, where f_c is the fixed-side row of c (Eqs. 11-12).  On the item
 * side the prediction of (u, i) is found through i_pos. */
static void observed_terms(const oracle_problem *P, int side, int p0, int bs,
                           const double *Fix, const double *yhat, int64_t r, double *A,
                           double *g) {
    const int d = P->d;
    const int64_t *ptr = side == 0 ? P->u_ptr : P->i_ptr;
    const int32_t *idx = side == 0 ? P->u_idx : P->i_idx;
    for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
        const int64_t q = side == 0 ? s : P->i_pos[s];
        const double *f_c = Fix + (int64_t)idx[s] * d + p0;
        const double a = av(P, q), res = a * (yhat[q] - yv(P, q));
        for (int f = 0; f < bs; ++f) {
            g[f] += res * f_c[f];
            for (int t = 0; t < bs; ++t) A[f * bs + t] += a * f_c[f] * f_c[t];
        }
    }
}

/* Exact minimisation of L over x_{r,pi} (Eq. 8) by the Newton step of Eq. 9,
 * as Algorithm 3 does for every row of a half-step.  With apply = 1 the row
 * moves to x_{r,pi} - delta and every cached prediction of the row drops by
 * <delta, f_{c,pi}> (the prediction is linear in x_r, Eq. 1); with apply = 0
 * the new block goes to out_w and nothing changes.  A (bs x bs) and g (bs) are
 * scratch. */
static int row_update(const oracle_problem *P, int side, int p0, int bs, double *Upd,
                      const double *Fix, const double *G, double *yhat, int64_t r,
                      double *A, double *g, int apply, double *out_w) {
    const int d = P->d;
    const int64_t *ptr = side == 0 ? P->u_ptr : P->i_ptr;
    const int32_t *idx = side == 0 ? P->u_idx : P->i_idx;
    double *x = Upd + r * d;
    const double lam = P->lambda * (1.0 + P->nu * (double)(ptr[r + 1] - ptr[r]));

    gramian_terms(P, p0, bs, x, G, lam, A, g);
    observed_terms(P, side, p0, bs, Fix, yhat, r, A, g);
    if (cholesky_solve(A, g, bs)) return ORACLE_ENOTPD; /* g now holds delta */
    if (!apply) {
        for (int f = 0; f < bs; ++f) out_w[f] = x[p0 + f] - g[f];
        return ORACLE_OK;
    }
    for (int f = 0; f < bs; ++f) x[p0 + f] -= g[f];
    for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
        const int64_t q = side == 0 ? s : P->i_pos[s];
        const double *f_c = Fix + (int64_t)idx[s] * d + p0;
        double change = 0.0;
        for (int f = 0; f < bs; ++f) change += g[f] * f_c[f];
        yhat[q] -= change;
    }
    return ORACLE_OK;
}

static void half_rows(void *vp, int64_t lo, int64_t hi, int tid) {
    half_ctx *c = (half_ctx *)vp;
    double *A = c->scratch + (int64_t)tid * (c->bs * c->bs + c->bs);
    double *g = A + c->bs * c->bs;
    for (int64_t r = lo; r < hi; ++r)
        if (row_update(c->P, c->side, c->p0, c->bs, c->Upd, c->Fix, c->G, c->yhat, r, A, g,
                       1, NULL))
            c->status = ORACLE_ENOTPD;
}

/* Partial Gramian G^{pi} = sum_j x_j (x) x_{j,pi} (Eq. 10), d x bs. */
static void partial_gramian(const double *X, int64_t n, int d, int p0, int bs, double *G) {
    memset(G, 0, sizeof(double) * d * bs);
    for (int64_t j = 0; j < n; ++j) {
        const double *x = X + j * d;
        for (int k = 0; k < d; ++k)
            for (int f = 0; f < bs; ++f) G[k * bs + f] += x[k] * x[p0 + f];
    }
}

/* One block-side step of Algorithm 3 on block k (coordinates [k b, k b + bs)).
 * W, H, yhat are updated in place.  Returns ORACLE_ENOTPD if some row's
 * Hessian was not positive definite (that row is left unchanged). */
int oracle_halfstep(const oracle_problem *P, int side, int block, double *W, double *H,
                    double *yhat) {
    const int d = P->d, b = P->b;
    if (d <= 0 || b <= 0 || block < 0 || block * b >= d) return ORACLE_EINVAL;
    const int p0 = block * b, bs = (d - p0 < b) ? d - p0 : b;
    const int nt = P->n_threads > 0 ? P->n_threads : 1;
    half_ctx c;
    c.P = P;
    c.side = side;
    c.p0 = p0;
    c.bs = bs;
    c.Upd = side == 0 ? W : H;
    c.Fix = side == 0 ? H : W;
    c.yhat = yhat;
    c.status = ORACLE_OK;
    double *G = malloc(sizeof(double) * d * bs);
    double *scr = malloc(sizeof(double) * (size_t)nt * (bs * bs + bs));
    if (!G || !scr) { free(G); free(scr); return ORACLE_ENOMEM; }
    partial_gramian(c.Fix, side == 0 ? P->n_items : P->n_users, d, p0, bs, G);
    c.G = G;
    c.scratch = scr;
    parallel_for(side == 0 ? P->n_users : P->n_items, nt, &c, half_rows);
    free(G);
    free(scr);
    return c.status;
}

/* The new w_{r,pi} that oracle_halfstep would give row r, computed from the
 * current state without changing it.  out_w receives bs values. */
int oracle_row_step(const oracle_problem *P, int side, int block, const double *W,
                    const double *H, const double *yhat, int64_t r, double *out_w) {
    const int d = P->d, b = P->b;
    if (d <= 0 || b <= 0 || block < 0 || block * b >= d) return ORACLE_EINVAL;
    const int p0 = block * b, bs = (d - p0 < b) ? d - p0 : b;
    const double *Fix = side == 0 ? H : W;
    double *G = malloc(sizeof(double) * d * bs);
    double *A = malloc(sizeof(double) * (bs * bs + bs));
    if (!G || !A) { free(G); free(A); return ORACLE_ENOMEM; }
    partial_gramian(Fix, side == 0 ? P->n_items : P->n_users, d, p0, bs, G);
    int st = row_update(P, side, p0, bs, (double *)(side == 0 ? W : H), Fix, G,
                        (double *)yhat, r, A, A + bs * bs, 0, out_w);
    free(G);
    free(A);
    return st;
}

/* oracle_row_step for a list of rows (the partial Gramian is formed once).
 * out_w receives n_sel x bs values; status per row in out_status. */
int oracle_rows_step(const oracle_problem *P, int side, int block, const double *W,
                     const double *H, const double *yhat, const int64_t *rows, int64_t n_sel,
                     double *out_w, int32_t *out_status) {
    const int d = P->d, b = P->b;
    if (d <= 0 || b <= 0 || block < 0 || block * b >= d) return ORACLE_EINVAL;
    const int p0 = block * b, bs = (d - p0 < b) ? d - p0 : b;
    const double *Fix = side == 0 ? H : W;
    double *G = malloc(sizeof(double) * d * bs);
    double *A = malloc(sizeof(double) * (bs * bs + bs));
    if (!G || !A) { free(G); free(A); return ORACLE_ENOMEM; }
    partial_gramian(Fix, side == 0 ? P->n_items : P->n_users, d, p0, bs, G);
    for (int64_t k = 0; k < n_sel; ++k)
        out_status[k] = row_update(P, side, p0, bs, (double *)(side == 0 ? W : H), Fix, G,
                                   (double *)yhat, rows[k], A, A + bs * bs, 0, out_w + k * bs);
    free(G);
    free(A);
    return ORACLE_OK;
}

/* T epochs of Algorithm 3.  If trace is non-NULL it receives the objective
 * after every block-side step: epochs * 2 * ceil(d/b) values, in order. */
int oracle_ialspp(const oracle_problem *P, int epochs, double *W, double *H, double *yhat,
                  double *trace) {
    const int nb = (P->d + P->b - 1) / P->b;
    int status = ORACLE_OK;
    int64_t t = 0;
    for (int e = 0; e < epochs; ++e) {
        oracle_predict(P, W, H, yhat); /* Compute yhat */
        for (int k = 0; k < nb; ++k) {
            for (int side = 0; side < 2; ++side) {
                int st = oracle_halfstep(P, side, k, W, H, yhat);
                if (st == ORACLE_EINVAL || st == ORACLE_ENOMEM) return st;
                if (st) status = st;
                if (trace) trace[t++] = oracle_objective(P, W, H);
            }
        }
    }
    return status;
}

/* ---------------------------------------------- Algorithm 1 (iALS), Eq. 3 */

typedef struct {
    const oracle_problem *P;
    int side;
    double *Upd;
    const double *Fix;
    const double *G; /* full d x d Gramian of Fix */
    double *scratch;
    int status;
} ials_ctx;

static void ials_rows(void *vp, int64_t lo, int64_t hi, int tid) {
    ials_ctx *c = (ials_ctx *)vp;
    const oracle_problem *P = c->P;
    const int d = P->d;
    double *A = c->scratch + (int64_t)tid * (d * d + d), *rhs = A + d * d;
    const int64_t *ptr = c->side == 0 ? P->u_ptr : P->i_ptr;
    const int32_t *idx = c->side == 0 ? P->u_idx : P->i_idx;
    for (int64_t r = lo; r < hi; ++r) {
        const double lam = P->lambda * (1.0 + P->nu * (double)(ptr[r + 1] - ptr[r]));
        for (int f = 0; f < d; ++f) {
            rhs[f] = 0.0;
            for (int g = 0; g < d; ++g)
                A[f * d + g] = P->alpha0 * c->G[f * d + g] + (f == g ? lam : 0.0);
        }
        for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
            const int64_t q = c->side == 0 ? s : P->i_pos[s];
            const double *h = c->Fix + (int64_t)idx[s] * d;
            const double a = av(P, q), y = yv(P, q);
            for (int f = 0; f < d; ++f) {
                rhs[f] += a * y * h[f];
                for (int g = 0; g < d; ++g) A[f * d + g] += a * h[f] * h[g];
            }
        }
        if (cholesky_solve(A, rhs, d)) { c->status = ORACLE_ENOTPD; continue; }
        memcpy(c->Upd + r * d, rhs, sizeof(double) * d);
    }
}

/* T epochs of Algorithm 1: G^I, all users by Eq. 3, then G^U and all items. */
int oracle_ials(const oracle_problem *P, int epochs, double *W, double *H) {
    const int d = P->d, nt = P->n_threads > 0 ? P->n_threads : 1;
    double *G = malloc(sizeof(double) * d * d);
    double *scr = malloc(sizeof(double) * (size_t)nt * (d * d + d));
    if (!G || !scr) { free(G); free(scr); return ORACLE_ENOMEM; }
    int status = ORACLE_OK;
    for (int e = 0; e < epochs; ++e) {
        for (int side = 0; side < 2; ++side) {
            ials_ctx c;
            c.P = P;
            c.side = side;
            c.Upd = side == 0 ? W : H;
            c.Fix = side == 0 ? H : W;
            gramian(c.Fix, side == 0 ? P->n_items : P->n_users, d, G);
            c.G = G;
            c.scratch = scr;
            c.status = ORACLE_OK;
            parallel_for(side == 0 ? P->n_users : P->n_items, nt, &c, ials_rows);
            if (c.status) status = c.status;
        }
    }
    free(G);
    free(scr);
    return status;
}

/* ------------------------------------------- Algorithm 2 (iCD), Eqs. 5-7 */

/* T epochs of Algorithm 2: recompute yhat; for each coordinate f the user pass
 * (g^I = sum_i h_{i,f} h_i, then Eq. 6 / Eq. 5 / Eq. 7 per user) and then the
 * item pass with the roles of W and H exchanged. */
int oracle_icd(const oracle_problem *P, int epochs, double *W, double *H, double *yhat) {
    const int d = P->d;
    double *gv = malloc(sizeof(double) * d);
    if (!gv) return ORACLE_ENOMEM;
    int status = ORACLE_OK;
    for (int e = 0; e < epochs; ++e) {
        oracle_predict(P, W, H, yhat);
        for (int f = 0; f < d; ++f) {
            for (int side = 0; side < 2; ++side) {
                double *Upd = side == 0 ? W : H;
                const double *Fix = side == 0 ? H : W;
                const int64_t nf = side == 0 ? P->n_items : P->n_users;
                const int64_t nr = side == 0 ? P->n_users : P->n_items;
                const int64_t *ptr = side == 0 ? P->u_ptr : P->i_ptr;
                const int32_t *idx = side == 0 ? P->u_idx : P->i_idx;
                for (int k = 0; k < d; ++k) gv[k] = 0.0;
                for (int64_t j = 0; j < nf; ++j)
                    for (int k = 0; k < d; ++k) gv[k] += Fix[j * d + f] * Fix[j * d + k];
                for (int64_t r = 0; r < nr; ++r) {
                    double *w = Upd + r * d;
                    const double lam = P->lambda * (1.0 + P->nu * (double)(ptr[r + 1] - ptr[r]));
                    double num = 0.0;
                    for (int k = 0; k < d; ++k) num += w[k] * gv[k];
                    num = P->alpha0 * num + lam * w[f];
                    double den = P->alpha0 * gv[f] + lam;
                    for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
                        const int64_t q = side == 0 ? s : P->i_pos[s];
                        const double h = Fix[(int64_t)idx[s] * d + f];
                        num += av(P, q) * (yhat[q] - yv(P, q)) * h;
                        den += av(P, q) * h * h;
                    }
                    if (!(den > 0.0)) { status = ORACLE_ENOTPD; continue; }
                    const double delta = num / den;
                    w[f] -= delta;
                    for (int64_t s = ptr[r]; s < ptr[r + 1]; ++s) {
                        const int64_t q = side == 0 ? s : P->i_pos[s];
                        yhat[q] -= delta * Fix[(int64_t)idx[s] * d + f];
                    }
                }
            }
        }
    }
    free(gv);
    return status;
}

/* ------------------------------------------------------------- fold-in */

/* Embedding for one new user against frozen item factors H (n_items x d).
 * The paper's protocol gives held-out users' interactions at evaluation time
 * without saying how their embeddings are obtained.  Reading used here: start
 * from w = 0 (so yhat = 0 on the request's items) and run `sweeps` passes of
 * the user-side block steps of Algorithm 3 over all blocks in order, with H,
 * and hence G^I, fixed and lambda_u = lambda (1 + nu n).  One sweep with b = d
 * is Eq. 3; more sweeps converge to it for any b.
 * items/y/alpha: the request's n interactions (y, alpha may be NULL = 1). */
/* G^I = H^T H (Eq. 4), d x d, for callers that fold in many users against the
 * same frozen H (oracle_foldin_g). */
void oracle_gramian(const double *H, int32_t n_items, int32_t d, double *G) { gramian(H, n_items, d, G); }

/* oracle_foldin with G^I = H^T H given (from oracle_gramian), so that a
 * sequence of requests against one H forms it once.  Same arithmetic. */
int oracle_foldin_g(const double *H, const double *G, int32_t n_items, int32_t d, int32_t b, double alpha0,
                    double lambda, double nu, int32_t sweeps, const int32_t *items, const double *y,
                    const double *alpha, int32_t n, double *w_out);

int oracle_foldin(const double *H, int32_t n_items, int32_t d, int32_t b, double alpha0,
                  double lambda, double nu, int32_t sweeps, const int32_t *items,
                  const double *y, const double *alpha, int32_t n, double *w_out) {
    if (d <= 0 || b <= 0 || n < 0) return ORACLE_EINVAL;
    double *G = malloc(sizeof(double) * d * d);
    if (!G) return ORACLE_ENOMEM;
    gramian(H, n_items, d, G); /* G^I, Eq. 4 */
    const int st = oracle_foldin_g(H, G, n_items, d, b, alpha0, lambda, nu, sweeps, items, y, alpha, n, w_out);
    free(G);
    return st;
}

int oracle_foldin_g(const double *H, const double *G, int32_t n_items, int32_t d, int32_t b, double alpha0,
                    double lambda, double nu, int32_t sweeps, const int32_t *items, const double *y,
                    const double *alpha, int32_t n, double *w_out) {
    if (d <= 0 || b <= 0 || n < 0) return ORACLE_EINVAL;
    for (int32_t s = 0; s < n; ++s)
        if (items[s] < 0 || items[s] >= n_items) return ORACLE_EINVAL;
    const int bmax = b < d ? b : d;
    double *yhat = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *A = malloc(sizeof(double) * (bmax * bmax + bmax));
    if (!yhat || !A) { free(yhat); free(A); return ORACLE_ENOMEM; }
    double *g = A + bmax * bmax;
    const double lam = lambda * (1.0 + nu * (double)n);
    int status = ORACLE_OK;
    for (int f = 0; f < d; ++f) w_out[f] = 0.0;
    for (int32_t s = 0; s < n; ++s) yhat[s] = 0.0;
    const int nb = (d + b - 1) / b;
    for (int sw = 0; sw < sweeps; ++sw) {
        for (int k = 0; k < nb; ++k) {
            const int p0 = k * b, bs = (d - p0 < b) ? d - p0 : b;
            for (int f = 0; f < bs; ++f) {
                double t = 0.0;
                for (int q = 0; q < d; ++q) t += w_out[q] * G[q * d + p0 + f];
                g[f] = alpha0 * t + lam * w_out[p0 + f];
                for (int q = 0; q < bs; ++q)
                    A[f * bs + q] = alpha0 * G[(p0 + f) * d + p0 + q] + (f == q ? lam : 0.0);
            }
            for (int32_t s = 0; s < n; ++s) {
                const double *h = H + (int64_t)items[s] * d + p0;
                const double a = alpha ? alpha[s] : 1.0, yy = y ? y[s] : 1.0;
                for (int f = 0; f < bs; ++f) {
                    g[f] += a * (yhat[s] - yy) * h[f];
                    for (int q = 0; q < bs; ++q) A[f * bs + q] += a * h[f] * h[q];
                }
            }
            if (cholesky_solve(A, g, bs)) { status = ORACLE_ENOTPD; continue; }
            for (int f = 0; f < bs; ++f) w_out[p0 + f] -= g[f];
            for (int32_t s = 0; s < n; ++s) {
                const double *h = H + (int64_t)items[s] * d + p0;
                double t = 0.0;
                for (int f = 0; f < bs; ++f) t += g[f] * h[f];
                yhat[s] -= t;
            }
        }
    }
    free(yhat);
    free(A);
    return status;
}
