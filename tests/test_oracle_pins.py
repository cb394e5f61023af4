"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value comes from
an independent computation (brute force over all |U| x |I| pairs, a dense
weighted least-squares solve through numpy's SVD-based lstsq, central finite
differences of the brute-force loss, hand derivations in tests/golden), or
from an identity between two different algorithms of the paper (Algorithm 3
with b = d is Algorithm 1; with b = 1 it is Algorithm 2).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2110_14044_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_derived.json")


# ----------------------------------------------------------------- helpers

def tiny(n_users=7, n_items=5, d=6, density=0.45, seed=1, weighted=True):
    """A small random problem with general labels y and weights alpha."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n_users, n_items)) < density
    mask[0, :] = False          # a user with an empty history
    mask[1, :] = True           # a user with every item
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    nnz = data.nnz
    y = rng.uniform(0.5, 2.0, nnz) if weighted else None
    alpha = rng.uniform(0.5, 3.0, nnz) if weighted else None
    W = rng.normal(0, 0.4, (n_users, d))
    H = rng.normal(0, 0.4, (n_items, d))
    return data, y, alpha, W, H


def dense_weights(data, y, alpha):
    """Dense per-pair label Y and weight A (zero where (u,i) is not in S)."""
    Y = np.zeros((data.n_users, data.n_items))
    A = np.zeros((data.n_users, data.n_items))
    for u in range(data.n_users):
        for s in range(data.u_indptr[u], data.u_indptr[u + 1]):
            i = data.u_items[s]
            Y[u, i] = 1.0 if y is None else y[s]
            A[u, i] = 1.0 if alpha is None else alpha[s]
    return Y, A


def brute_loss(data, y, alpha, W, H, alpha0, lam, nu):
    """Eq. 2 term by term over every (u, i) pair, with per-row lambda."""
    Y, A = dense_weights(data, y, alpha)
    total = 0.0
    for u in range(data.n_users):
        for i in range(data.n_items):
            yh = float(np.dot(W[u], H[i]))
            if A[u, i] > 0:
                total += A[u, i] * (yh - Y[u, i]) ** 2
            total += alpha0 * yh * yh
    nu_len = np.diff(data.u_indptr)
    ni_len = np.diff(data.i_indptr)
    for u in range(data.n_users):
        total += lam * (1 + nu * nu_len[u]) * float(np.dot(W[u], W[u]))
    for i in range(data.n_items):
        total += lam * (1 + nu * ni_len[i]) * float(np.dot(H[i], H[i]))
    return total


def lstsq_user(data, y, alpha, H, u, alpha0, lam, nu):
    """argmin_w of the user-u part of Eq. 2, as a stacked weighted LS problem.

    alpha (yh - y)^2 + alpha0 yh^2 = (alpha + alpha0) (yh - alpha y / (alpha + alpha0))^2
    + const, so each item contributes one row sqrt(c_i) h_i with target
    sqrt(c_i) p_i; the L2 term contributes sqrt(lambda_u) I with target 0.
    """
    Y, A = dense_weights(data, y, alpha)
    n_u = data.u_indptr[u + 1] - data.u_indptr[u]
    c = alpha0 + A[u]
    p = np.where(A[u] > 0, A[u] * Y[u] / c, 0.0)
    d = H.shape[1]
    M = np.vstack([np.sqrt(c)[:, None] * H, np.sqrt(lam * (1 + nu * n_u)) * np.eye(d)])
    t = np.concatenate([np.sqrt(c) * p, np.zeros(d)])
    return np.linalg.lstsq(M, t, rcond=None)[0]


def transpose_problem(data, y, alpha):
    """Swap the roles of users and items (for the item-side LS check)."""
    users = np.repeat(np.arange(data.n_users), np.diff(data.u_indptr))
    items = data.u_items
    t = synth.from_pairs(data.n_items, data.n_users, items, users)
    # entries of t are in (item, user) order; carry y/alpha along
    order = np.lexsort((users, items))
    ty = None if y is None else np.asarray(y)[order]
    ta = None if alpha is None else np.asarray(alpha)[order]
    return t, ty, ta


def fd_grad(f, x, idx, eps=1e-4):
    """Central differences (exact for a quadratic up to rounding)."""
    g = []
    for k in idx:
        xp = x.copy(); xp[k] += eps
        xm = x.copy(); xm[k] -= eps
        g.append((f(xp) - f(xm)) / (2 * eps))
    return np.array(g)


def make(data, y, alpha, d, b, alpha0, lam, nu):
    return oracle.Problem.from_data(data, d, b, alpha0, lam, nu, y=y, alpha=alpha, n_threads=2)


# ------------------------------------------------------------------- pins

def test_golden_hand_derived():
    cases = json.load(open(GOLDEN))["cases"]
    for c in cases:
        if c["name"] == "foldin_d2":
            w, st = oracle.foldin(np.array(c["H"]), c["d"], c["b"], c["alpha0"], c["lambda"],
                                  c["nu"], c["sweeps"], c["items"], y=c["y"])
            assert st == 0
            np.testing.assert_allclose(w, c["w"], rtol=1e-14, atol=1e-15)
            continue
        u, i = zip(*c["pairs"])
        data = synth.from_pairs(c["n_users"], c["n_items"], u, i)
        P = oracle.Problem.from_data(data, c["d"], c["b"], c["alpha0"], c["lambda"], c["nu"])
        W, H = P.factors(c["W"], c["H"])
        if "objective" in c:
            assert abs(oracle.objective(P, W, H) - c["objective"]) < 1e-14
        if "W_after_user_step" in c:
            yhat = oracle.predict(P, W, H)
            for k in range(-(-c["d"] // c["b"])):
                assert oracle.halfstep(P, 0, k, W, H, yhat) == 0
            np.testing.assert_allclose(W, c["W_after_user_step"], rtol=1e-14, atol=1e-15)
            if c["b"] == 1:  # the same user pass through the scalar iCD code path
                W2, H2 = P.factors(c["W"], c["H"])
                yh2 = oracle.predict(P, W2, H2)
                for f in range(c["d"]):
                    oracle.halfstep(P, 0, f, W2, H2, yh2)
                np.testing.assert_allclose(W2, c["W_after_user_step"], rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("nu", [0.0, 0.7])
def test_objective_equals_brute_force(nu):
    data, y, alpha, W, H = tiny()
    P = make(data, y, alpha, 6, 2, 0.3, 0.05, nu)
    want = brute_loss(data, y, alpha, W, H, 0.3, 0.05, nu)
    assert abs(oracle.objective(P, W, H) - want) <= 1e-12 * abs(want)


def test_gramian_identity_all_pairs():
    # sum_u sum_i yhat^2 = <W^T W, H^T H>_F: isolate the alpha0 term.
    data, y, alpha, W, H = tiny(seed=3)
    P0 = make(data, y, alpha, 6, 2, 0.0, 0.0, 0.0)
    P1 = make(data, y, alpha, 6, 2, 1.0, 0.0, 0.0)
    allpairs = float(((W @ H.T) ** 2).sum())
    got = oracle.objective(P1, W, H) - oracle.objective(P0, W, H)
    assert abs(got - allpairs) <= 1e-12 * allpairs


def test_predict_is_dot_product():
    data, y, alpha, W, H = tiny(seed=4)
    P = make(data, y, alpha, 6, 3, 0.1, 0.1, 0.0)
    yh = oracle.predict(P, W, H)
    users = np.repeat(np.arange(data.n_users), np.diff(data.u_indptr))
    np.testing.assert_allclose(yh, (W @ H.T)[users, data.u_items], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("nu", [0.0, 0.5])
def test_user_step_b_eq_d_is_dense_least_squares(nu):
    data, y, alpha, W, H = tiny(seed=5)
    d = W.shape[1]
    P = make(data, y, alpha, d, d, 0.25, 0.08, nu)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    assert oracle.halfstep(P, 0, 0, W1, H1, yhat) == 0
    for u in range(data.n_users):
        want = lstsq_user(data, y, alpha, H, u, 0.25, 0.08, nu)
        np.testing.assert_allclose(W1[u], want, rtol=1e-9, atol=1e-11)


def test_item_step_b_eq_d_is_dense_least_squares():
    data, y, alpha, W, H = tiny(seed=6)
    d = W.shape[1]
    P = make(data, y, alpha, d, d, 0.25, 0.08, 0.3)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    assert oracle.halfstep(P, 1, 0, W1, H1, yhat) == 0
    t, ty, ta = transpose_problem(data, y, alpha)
    for i in range(data.n_items):
        want = lstsq_user(t, ty, ta, W, i, 0.25, 0.08, 0.3)
        np.testing.assert_allclose(H1[i], want, rtol=1e-9, atol=1e-11)


@pytest.mark.parametrize("b", [1, 2, 4, 6])
def test_every_block_step_is_exact_block_minimiser(b):
    """After a block-side step the brute-force gradient on that block is zero.

    Catches a wrong Gramian slice, a stale cache, a wrong lambda_r or a sign
    error: any of them leaves a nonzero partial derivative.  b=4 with d=6 has
    a ragged last block.
    """
    data, y, alpha, W, H = tiny(seed=7)
    d = W.shape[1]
    a0, lam, nu = 0.3, 0.05, 0.4
    P = make(data, y, alpha, d, b, a0, lam, nu)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    nb = -(-d // b)
    for k in range(nb):
        cols = list(range(k * b, min(d, (k + 1) * b)))
        for side in (0, 1):
            assert oracle.halfstep(P, side, k, W1, H1, yhat) == 0
            M = W1 if side == 0 else H1
            for r in range(M.shape[0]):
                def f(v, r=r):
                    Wt, Ht = W1.copy(), H1.copy()
                    (Wt if side == 0 else Ht)[r] = v
                    return brute_loss(data, y, alpha, Wt, Ht, a0, lam, nu)
                g = fd_grad(f, M[r].copy(), cols)
                assert np.max(np.abs(g)) < 1e-6, (side, k, r, g)
            # the maintained cache still equals the model's predictions
            np.testing.assert_allclose(yhat, oracle.predict(P, W1, H1), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("b", [1, 3, 8, 16])
def test_objective_never_increases(b):
    prob = synth.preset("parity_2k", n_users=300, n_items=150, nnz=4000, len_max=150)
    data = prob.data
    P = oracle.Problem.from_data(data, 16, b, 0.1, 1e-3, 0.5, n_threads=4)
    L0 = oracle.objective(P, prob.W0, prob.H0)
    _, _, _, trace, st = oracle.ialspp(P, 3, prob.W0, prob.H0, trace=True)
    assert st == 0
    seq = np.concatenate([[L0], trace])
    assert np.all(np.diff(seq) <= 1e-12 * seq[:-1]), np.diff(seq).max()
    assert seq[-1] < 0.99 * seq[0]


def test_b_eq_d_is_algorithm_1():
    data, y, alpha, W, H = tiny(n_users=30, n_items=20, d=5, seed=8)
    P = make(data, y, alpha, 5, 5, 0.2, 0.03, 0.6)
    Wa, Ha, _, _, st = oracle.ialspp(P, 3, W, H)
    Wb, Hb, st2 = oracle.ials(P, 3, W, H)
    assert st == 0 and st2 == 0
    np.testing.assert_allclose(Wa, Wb, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Ha, Hb, rtol=1e-9, atol=1e-12)


def test_algorithm_1_is_dense_least_squares():
    data, y, alpha, W, H = tiny(seed=9)
    d = W.shape[1]
    P = make(data, y, alpha, d, d, 0.15, 0.07, 0.2)
    W1, H1, st = oracle.ials(P, 1, W, H)
    assert st == 0
    Wexp = np.stack([lstsq_user(data, y, alpha, H, u, 0.15, 0.07, 0.2)
                     for u in range(data.n_users)])
    np.testing.assert_allclose(W1, Wexp, rtol=1e-9, atol=1e-11)
    t, ty, ta = transpose_problem(data, y, alpha)
    Hexp = np.stack([lstsq_user(t, ty, ta, Wexp, i, 0.15, 0.07, 0.2)
                     for i in range(data.n_items)])
    np.testing.assert_allclose(H1, Hexp, rtol=1e-8, atol=1e-10)


def test_b_eq_1_is_algorithm_2():
    data, y, alpha, W, H = tiny(n_users=30, n_items=20, d=5, seed=10)
    P = make(data, y, alpha, 5, 1, 0.2, 0.03, 0.6)
    Wa, Ha, ya, _, st = oracle.ialspp(P, 3, W, H)
    Wb, Hb, yb, st2 = oracle.icd(P, 3, W, H)
    assert st == 0 and st2 == 0
    np.testing.assert_allclose(Wa, Wb, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(Ha, Hb, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(ya, yb, rtol=1e-10, atol=1e-13)


def test_user_block_sweeps_converge_to_closed_form():
    """Block CD on the strictly convex user subproblem reaches the LS solution."""
    data, y, alpha, W, H = tiny(seed=11)
    d = W.shape[1]
    P = make(data, y, alpha, d, 2, 0.25, 0.08, 0.0)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    for _ in range(300):
        for k in range(3):
            oracle.halfstep(P, 0, k, W1, H1, yhat)
    for u in range(data.n_users):
        np.testing.assert_allclose(W1[u], lstsq_user(data, y, alpha, H, u, 0.25, 0.08, 0.0),
                                   rtol=1e-7, atol=1e-9)


def test_row_step_matches_half_step():
    data, y, alpha, W, H = tiny(n_users=20, n_items=12, d=6, seed=12)
    P = make(data, y, alpha, 6, 4, 0.2, 0.05, 0.3)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    for side in (0, 1):
        for k in (0, 1):
            n_rows = data.n_users if side == 0 else data.n_items
            rows = {r: oracle.row_step(P, side, k, W1, H1, yhat, r) for r in range(n_rows)}
            oracle.halfstep(P, side, k, W1, H1, yhat)
            M = W1 if side == 0 else H1
            for r, (st, w) in rows.items():
                assert st == 0
                np.testing.assert_array_equal(M[r, k * 4:k * 4 + w.size], w)


def test_foldin_one_sweep_b_eq_d_is_least_squares():
    rng = np.random.default_rng(13)
    H = rng.normal(0, 0.5, (9, 5))
    items = np.array([0, 2, 3, 7])
    yy = rng.uniform(0.5, 2, 4)
    aa = rng.uniform(0.5, 2, 4)
    one = synth.from_pairs(1, 9, [0, 0, 0, 0], items)
    want = lstsq_user(one, yy, aa, H, 0, 0.3, 0.1, 0.5)
    w, st = oracle.foldin(H, 5, 5, 0.3, 0.1, 0.5, 1, items, y=yy, alpha=aa)
    assert st == 0
    np.testing.assert_allclose(w, want, rtol=1e-10, atol=1e-12)
    w2, st = oracle.foldin(H, 5, 2, 0.3, 0.1, 0.5, 400, items, y=yy, alpha=aa)
    np.testing.assert_allclose(w2, want, rtol=1e-7, atol=1e-9)
    w0, st = oracle.foldin(H, 5, 2, 0.3, 0.1, 0.5, 4, [], None)
    assert st == 0 and np.all(w0 == 0.0)


def test_foldin_equals_training_user_step():
    """Fold-in of an existing user's history = that user's rows in a user-only pass from w=0."""
    data, y, alpha, W, H = tiny(seed=14)
    d = W.shape[1]
    P = make(data, y, alpha, d, 3, 0.2, 0.05, 0.4)
    W1, H1 = P.factors(np.zeros_like(W), H)
    yhat = oracle.predict(P, W1, H1)
    for _ in range(2):
        for k in range(2):
            oracle.halfstep(P, 0, k, W1, H1, yhat)
    for u in range(data.n_users):
        lo, hi = data.u_indptr[u], data.u_indptr[u + 1]
        w, st = oracle.foldin(H, d, 3, 0.2, 0.05, 0.4, 2, data.u_items[lo:hi],
                              y=y[lo:hi], alpha=alpha[lo:hi])
        np.testing.assert_allclose(w, W1[u], rtol=1e-11, atol=1e-13)


def test_not_positive_definite_is_reported():
    # lambda = 0, alpha0 = 0 and an empty history: the Hessian is the zero matrix.
    data, y, alpha, W, H = tiny(seed=15)
    P = make(data, y, alpha, 6, 2, 0.0, 0.0, 0.0)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    before = W1[0].copy()
    assert oracle.halfstep(P, 0, 0, W1, H1, yhat) == oracle.ENOTPD
    np.testing.assert_array_equal(W1[0], before)


def test_bad_transpose_is_rejected():
    data, *_ = tiny(seed=16)
    bad = data.i_users.copy()
    bad[0] = (bad[0] + 1) % data.n_users
    with pytest.raises(ValueError):
        oracle.Problem(data.n_users, data.n_items, data.u_indptr, data.u_items, data.i_indptr,
                       bad, 6, 2, 0.1, 0.1)


def test_rows_step_matches_row_step():
    data, y, alpha, W, H = tiny(n_users=20, n_items=12, d=6, seed=17)
    P = make(data, y, alpha, 6, 2, 0.2, 0.05, 0.3)
    W1, H1 = P.factors(W, H)
    yhat = oracle.predict(P, W1, H1)
    rows = np.array([3, 0, 11, 5])
    st, out = oracle.rows_step(P, 1, 2, W1, H1, yhat, rows)
    for k, r in enumerate(rows):
        s1, w1 = oracle.row_step(P, 1, 2, W1, H1, yhat, r)
        assert st[k] == s1 == 0
        np.testing.assert_array_equal(out[k], w1)


@pytest.mark.parametrize("b", [1, 2, 4])
def test_epochs_reach_a_stationary_point_of_the_loss(b):
    """Iterated to convergence, Algorithm 3 stops where the whole brute-force
    gradient of Eq. 2 vanishes (every coordinate of W and H, not only the
    block just solved), from b = 1 (iCD) through b = d (iALS)."""
    data, y, alpha, W, H = tiny(seed=21, d=4)
    a0, lam, nu = 0.2, 0.1, 0.3
    P = make(data, y, alpha, 4, b, a0, lam, nu)
    W1, H1, _, trace, st = oracle.ialspp(P, 400, W, H, trace=True)
    assert st == 0
    gW = fd_grad(lambda v: brute_loss(data, y, alpha, v.reshape(W1.shape), H1, a0, lam, nu),
                 W1.ravel().copy(), range(W1.size))
    gH = fd_grad(lambda v: brute_loss(data, y, alpha, W1, v.reshape(H1.shape), a0, lam, nu),
                 H1.ravel().copy(), range(H1.size))
    assert max(np.abs(gW).max(), np.abs(gH).max()) < 1e-8
    assert abs(trace[-1] - brute_loss(data, y, alpha, W1, H1, a0, lam, nu)) < 1e-10 * trace[-1]


def test_foldin_with_precomputed_gramian_is_the_same_computation():
    """oracle.foldin with G^I from oracle.gramian (formed once for many requests)
    gives bitwise the result of forming it inside the call, and G^I is H^T H."""
    rng = np.random.default_rng(77)
    H = rng.normal(0, 0.1, (60, 12))
    G = oracle.gramian(H)
    np.testing.assert_allclose(G, H.T @ H, rtol=1e-12, atol=1e-14)
    items = rng.choice(60, 17, replace=False).astype(np.int32)
    y = rng.uniform(0.5, 2.0, 17)
    w1, s1 = oracle.foldin(H, 12, 4, 0.1, 1e-2, 0.5, 3, items, y=y)
    w2, s2 = oracle.foldin(H, 12, 4, 0.1, 1e-2, 0.5, 3, items, y=y, G=G)
    assert s1 == s2 == 0
    assert np.array_equal(w1, w2)


@pytest.mark.parametrize("algo", ["ialspp", "ials", "icd"])
def test_relabelling_users_and_items_permutes_the_iterates(algo):
    """Rows of one side are solved independently (Section 3.2), so renaming users
    and items only renames the result, for Algorithms 1-3 alike: a mix-up of user
    and item ids, or of the item-major to user-major position map, breaks this."""
    data, y, alpha, W, H = tiny(n_users=25, n_items=18, d=6, seed=31)
    rng = np.random.default_rng(32)
    pu, pi = rng.permutation(data.n_users), rng.permutation(data.n_items)
    users = np.repeat(np.arange(data.n_users), np.diff(data.u_indptr))
    nu_, ni_ = pu[users], pi[np.asarray(data.u_items)]
    order = np.lexsort((ni_, nu_))  # the relabelled problem's user-major order
    data2 = synth.from_pairs(data.n_users, data.n_items, nu_, ni_)
    y2, a2 = np.asarray(y)[order], np.asarray(alpha)[order]
    W2, H2 = np.empty_like(W), np.empty_like(H)
    W2[pu], H2[pi] = W, H
    b = {"ialspp": 2, "ials": 6, "icd": 1}[algo]

    def run(dat, yy, aa, W0, H0):
        P = make(dat, yy, aa, 6, b, 0.2, 0.04, 0.5)
        out = getattr(oracle, algo)(P, 2, W0, H0)
        return out[0], out[1], out[-1]

    Wa, Ha, st = run(data, y, alpha, W, H)
    Wb, Hb, st2 = run(data2, y2, a2, W2, H2)
    assert st == 0 and st2 == 0
    np.testing.assert_allclose(Wb[pu], Wa, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(Hb[pi], Ha, rtol=1e-9, atol=1e-12)


def test_scaling_every_weight_leaves_the_iterates_unchanged():
    """Every term of Eq. 2 carries one of alpha_s, alpha0 or lambda_r, so scaling all
    three by c scales the loss by c and leaves every Newton step (Eq. 9: g and A of
    Eqs. 11-12 both scale by c) and so every iterate unchanged.  A term that misses
    its weight in the gradient or the Hessian breaks this."""
    data, y, alpha, W, H = tiny(n_users=25, n_items=18, d=6, seed=33)
    c = 3.7
    Pa = make(data, y, alpha, 6, 3, 0.2, 0.04, 0.5)
    Pb = make(data, y, np.asarray(alpha) * c, 6, 3, 0.2 * c, 0.04 * c, 0.5)
    Wa, Ha, _, _, st = oracle.ialspp(Pa, 2, W, H)
    Wb, Hb, _, _, st2 = oracle.ialspp(Pb, 2, W, H)
    assert st == 0 and st2 == 0
    np.testing.assert_allclose(Wb, Wa, rtol=1e-10, atol=1e-13)
    np.testing.assert_allclose(Hb, Ha, rtol=1e-10, atol=1e-13)
    assert abs(oracle.objective(Pb, Wb, Hb) - c * oracle.objective(Pa, Wa, Ha)) <= 1e-10 * c * oracle.objective(Pa, Wa, Ha)


def test_foldin_does_not_depend_on_item_names_or_history_order():
    """Fold-in (Section 5.1.1: a new user's embedding against frozen item factors)
    sums over the request's history, so renaming the items (with H's rows) or
    listing the history in another order changes nothing but rounding."""
    rng = np.random.default_rng(34)
    n_items, d = 40, 6
    H = rng.normal(0, 0.5, (n_items, d))
    items = rng.choice(n_items, 15, replace=False)
    yy, aa = rng.uniform(0.5, 2, 15), rng.uniform(0.5, 2, 15)
    w, st = oracle.foldin(H, d, 2, 0.2, 0.05, 0.5, 3, items, y=yy, alpha=aa)
    assert st == 0
    pi = rng.permutation(n_items)
    H2 = np.empty_like(H)
    H2[pi] = H
    order = rng.permutation(15)
    w2, st2 = oracle.foldin(H2, d, 2, 0.2, 0.05, 0.5, 3, pi[items][order], y=yy[order], alpha=aa[order])
    assert st2 == 0
    np.testing.assert_allclose(w2, w, rtol=1e-10, atol=1e-12)
