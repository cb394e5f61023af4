"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the plain FP32 path must match the oracle to 1e-5 relative
objective per epoch and 1e-3 maximum relative embedding error, where the
relative error of a row is |x_r - x*_r| / max(|x*_r|, 1e-6 median_r |x*_r|).
Single block-side steps are held to 1e-4 (a handful of FP32 roundings).
"""
import numpy as np
import pytest

import oracle
from paper_2110_14044_gb300 import _abi, synth

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-5
EMB_TOL = 1e-3
STEP_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14044_gb300 import build
    build.build()
    oracle.build()


def Model(*a, **k):
    import paper_2110_14044_gb300 as ials
    return ials.Model(*a, **k)


def rel_embed_err(X, Xref):
    X = np.asarray(X, np.float64)
    Xref = np.asarray(Xref, np.float64)
    nref = np.linalg.norm(Xref, axis=1)
    floor = max(1e-6 * np.median(nref), 1e-30)
    return float(np.max(np.linalg.norm(X - Xref, axis=1) / np.maximum(nref, floor)))


def small(n_users=300, n_items=200, nnz=6000, seed=0, d=32, len_max=200):
    prob = synth.preset("parity_2k", seed=seed, n_users=n_users, n_items=n_items, nnz=nnz,
                        len_max=len_max, d=d)
    return prob


def weights(nnz, seed):
    rng = np.random.default_rng(seed)
    return (rng.uniform(0.5, 2.0, nnz).astype(np.float32),
            rng.uniform(0.5, 3.0, nnz).astype(np.float32))


# --------------------------------------------------------- full parity workload

def test_parity_workload_five_epochs():
    """2,000 x 1,000, 50k positives, d=16, b=8, alpha0=0.1, lambda=1e-3, 5 epochs."""
    prob = synth.preset("parity_2k", seed=0)
    data = prob.data
    m = Model(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, W0=prob.W0, H0=prob.H0)
    objs = []
    for _ in range(prob.epochs):
        o, st = m.epoch(1, objective=True)
        assert st == 0
        objs.append(o)
    W, H = m.factors()
    P = oracle.Problem.from_data(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu)
    Wr, Hr, _, trace, st = oracle.ialspp(P, prob.epochs, prob.W0, prob.H0, trace=True)
    assert st == 0
    per_epoch = trace.reshape(prob.epochs, -1)[:, -1]
    rel = np.abs(np.array(objs) - per_epoch) / np.abs(per_epoch)
    assert rel.max() <= OBJ_TOL, rel
    assert rel_embed_err(W, Wr) <= EMB_TOL
    assert rel_embed_err(H, Hr) <= EMB_TOL


# --------------------------------------------------------- step-level parity

@pytest.mark.parametrize("b", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("weighted", [False, True])
def test_block_steps_match_oracle(b, weighted):
    d = 32
    prob = small(d=d, seed=b)
    data = prob.data
    y, a = weights(data.nnz, b) if weighted else (None, None)
    nu = 0.5 if weighted else 0.0
    m = Model(data, d, b, 0.1, 2e-3, nu, W0=prob.W0, H0=prob.H0, y=y, alpha=a)
    P = oracle.Problem.from_data(data, d, b, 0.1, 2e-3, nu, y=y, alpha=a)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    m.recompute_residuals()
    yref = 1.0 if y is None else y.astype(np.float64)
    np.testing.assert_allclose(m.residuals(), yhat - yref, rtol=1e-5, atol=1e-6)
    nb = d // b
    for k in range(min(nb, 3)):
        for side in (0, 1):
            assert m.block_step(side, k) == 0
            assert oracle.halfstep(P, side, k, W, H, yhat) == 0
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= STEP_TOL, (k, side)
            assert rel_embed_err(Hg, H) <= STEP_TOL, (k, side)
    e = m.residuals().astype(np.float64)
    scale = np.abs(yhat - yref).max()
    assert np.abs(e - (yhat - yref)).max() <= STEP_TOL * scale


def test_long_rows_are_split_and_still_exact():
    """A user with every item and an item with every user exceed the split length."""
    n_users, n_items, d, b = 700, 600, 16, 8
    rng = np.random.default_rng(3)
    mask = rng.random((n_users, n_items)) < 0.02
    mask[5, :] = True
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.05, 3)
    m = Model(data, d, b, 0.1, 1e-3, 0.2, W0=W0, H0=H0)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 0.2)
    Wr, Hr, _, _, st = oracle.ialspp(P, 2, W0, H0)
    W, H = m.factors()
    assert abs(o - oracle.objective(P, Wr, Hr)) <= OBJ_TOL * abs(o)
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL


def test_b_equals_d_is_closed_form_ials():
    prob = small(d=16, seed=4)
    m = Model(prob.data, 16, 16, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0)
    m.epoch(1)
    W, H = m.factors()
    P = oracle.Problem.from_data(prob.data, 16, 16, 0.1, 1e-3, 0.0)
    Wr, Hr, st = oracle.ials(P, 1, prob.W0, prob.H0)
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL


def test_b_equals_1_is_icd():
    prob = small(d=8, seed=5)
    m = Model(prob.data, 8, 1, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0)
    m.epoch(2)
    W, H = m.factors()
    P = oracle.Problem.from_data(prob.data, 8, 1, 0.1, 1e-3, 0.0)
    Wr, Hr, _, st = oracle.icd(P, 2, prob.W0, prob.H0)
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL


def test_objective_matches_oracle():
    prob = small(d=64, seed=6)
    y, a = weights(prob.data.nnz, 6)
    m = Model(prob.data, 64, 16, 0.3, 0.01, 0.7, y=y, alpha=a)
    rng = np.random.default_rng(6)
    W = rng.normal(0, 0.2, (prob.data.n_users, 64)).astype(np.float32)
    H = rng.normal(0, 0.2, (prob.data.n_items, 64)).astype(np.float32)
    m.set_factors(W, H)
    P = oracle.Problem.from_data(prob.data, 64, 16, 0.3, 0.01, 0.7, y=y, alpha=a)
    ref = oracle.objective(P, W, H)
    assert abs(m.objective() - ref) <= 1e-6 * abs(ref)


def test_residual_cache_stays_consistent():
    prob = small(d=32, seed=7)
    m = Model(prob.data, 32, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    m.epoch(2)
    e_kept = m.residuals()
    m.recompute_residuals()
    e_new = m.residuals()
    assert np.abs(e_kept - e_new).max() <= 1e-5 * max(1.0, np.abs(e_new).max())


def test_fp64_retry_path_gives_the_same_answer():
    prob = small(d=16, seed=8)
    data = prob.data
    a = Model(data, 16, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    b = Model(data, 16, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0, force_fp64=True)
    a.epoch(1)
    _, st = b.epoch(1)
    assert st == 0
    retries, not_pd = b.stats()
    assert retries == (data.n_users + data.n_items) * 2 and not_pd == 0
    assert a.stats() == (0, 0)
    Wa, Ha = a.factors()
    Wb, Hb = b.factors()
    assert rel_embed_err(Wb, Wa) <= STEP_TOL and rel_embed_err(Hb, Ha) <= STEP_TOL
    P = oracle.Problem.from_data(data, 16, 8, 0.1, 1e-3)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 1, prob.W0, prob.H0)
    assert rel_embed_err(Wb, Wr) <= EMB_TOL


def test_singular_rows_are_reported_and_left_unchanged():
    # lambda = alpha0 = 0: a user with no interactions has the zero Hessian.
    n_users, n_items, d, b = 50, 40, 8, 4
    rng = np.random.default_rng(9)
    mask = rng.random((n_users, n_items)) < 0.3
    mask[0, :] = False
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1, 9)
    m = Model(data, d, b, 0.0, 0.0, 0.0, W0=W0, H0=H0)
    st = m.block_step(0, 0)
    assert st == _abi.ENOTPD
    W, _ = m.factors()
    np.testing.assert_array_equal(W[0], W0[0])
    assert m.stats()[1] >= 1


def test_empty_interaction_set():
    n_users, n_items, d, b = 5, 4, 8, 4
    data = synth.from_pairs(n_users, n_items, [], [])
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.3, 10)
    m = Model(data, d, b, 0.2, 0.05, W0=W0, H0=H0)
    o, st = m.epoch(1, objective=True)
    assert st == 0
    P = oracle.Problem.from_data(data, d, b, 0.2, 0.05)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 1, W0, H0)
    W, H = m.factors()
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
    assert abs(o - oracle.objective(P, Wr, Hr)) <= OBJ_TOL * abs(o)


def test_deterministic_and_graph_replay_bitwise():
    prob = small(d=32, seed=11)
    runs = []
    for graph in (False, False, True):
        m = Model(prob.data, 32, 32, 0.1, 1e-3, 1.0, W0=prob.W0, H0=prob.H0, graph=graph)
        m.epoch(2)
        runs.append(m.factors())
        m.close()
    for W, H in runs[1:]:
        np.testing.assert_array_equal(W, runs[0][0])
        np.testing.assert_array_equal(H, runs[0][1])


def test_checkpoint_resume_is_bitwise():
    prob = small(d=16, seed=12)
    a = Model(prob.data, 16, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    a.epoch(3)
    b = Model(prob.data, 16, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    b.epoch(1)
    W1, H1 = b.factors()
    b.close()
    c = Model(prob.data, 16, 8, 0.1, 1e-3, W0=W1, H0=H1)
    c.epoch(2)
    for x, y in zip(a.factors(), c.factors()):
        np.testing.assert_array_equal(x, y)


def test_partial_gramian_entry_point():
    import torch
    rng = np.random.default_rng(13)
    for n, d, p0, bs in [(1, 4, 0, 4), (1000, 16, 8, 8), (20011, 128, 32, 32), (5000, 256, 0, 64)]:
        X = rng.normal(0, 1, (n, d)).astype(np.float32)
        Xt = torch.from_numpy(X).cuda()
        G = torch.empty((d, bs), dtype=torch.float32, device="cuda")
        _abi.ials_partial_gramian(Xt, n, d, p0, bs, G)
        ref = X.astype(np.float64).T @ X[:, p0:p0 + bs].astype(np.float64)
        err = np.abs(G.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-5, (n, d, err)


def test_bad_inputs_rejected():
    prob = small(d=16, seed=14)
    data = prob.data
    bad = data.u_items.copy()
    bad[1] = bad[0] if data.u_indptr[1] > 1 else data.n_items  # repeat or out of range
    with pytest.raises(_abi.IalsError) as ei:
        _abi.ials_create(_abi.make_params(16, 8, 0.1, 1e-3), data.n_users, data.n_items,
                         data.u_indptr, bad)
    assert ei.value.status == _abi.EINVAL
    wrong_t = data.i_users.copy()
    wrong_t[0] = (wrong_t[0] + 1) % data.n_users
    with pytest.raises(_abi.IalsError) as ei:
        _abi.ials_create(_abi.make_params(16, 8, 0.1, 1e-3), data.n_users, data.n_items,
                         data.u_indptr, data.u_items, data.i_indptr, wrong_t)
    assert ei.value.status == _abi.EINVAL


# --------------------------------------------------------- full-size sampled parity

@pytest.fixture(scope="module")
def ml20m():
    return synth.preset("ml20m_136k", seed=0)


def test_full_size_sampled_rows(ml20m):
    """136k x 20k, 10M positives, d=128, b=32: one user step and one item step.

    The oracle recomputes sampled rows (including the longest, split ones) one by
    one from the same pre-step state; the whole step is also checked through the
    maintained residual cache.
    """
    prob = ml20m
    data = prob.data
    m = Model(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, W0=prob.W0, H0=prob.H0)
    P = oracle.Problem.from_data(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu)
    rng = np.random.default_rng(0)
    for side, block in ((0, 0), (1, 0), (0, 3), (1, 3)):
        W, H = m.factors()
        # the oracle's predictions come from the factors alone (Eq. 1); the GPU's
        # maintained cache (y = 1, so residual = yhat - 1) is checked against them
        # separately rather than fed to the reference
        yhat = oracle.predict(P, W, H)
        e = m.residuals().astype(np.float64)
        assert np.abs(e - (yhat - 1.0)).max() <= 1e-4, (side, block)
        ptr = data.u_indptr if side == 0 else data.i_indptr
        lens = np.diff(ptr)
        n_rows = lens.size
        rows = np.unique(np.concatenate([np.argsort(-lens)[:6], rng.integers(0, n_rows, 120)]))
        st, ref = oracle.rows_step(P, side, block, W, H, yhat, rows)
        assert np.all(st == 0)
        assert m.block_step(side, block) == 0
        W2, H2 = m.factors()
        got = (W2 if side == 0 else H2)[rows, block * prob.b:(block + 1) * prob.b]
        err = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-12)
        assert err.max() <= EMB_TOL, (side, block, err.max())
    # the maintained cache still matches the model after four steps
    e_kept = m.residuals()
    m.recompute_residuals()
    assert np.abs(e_kept - m.residuals()).max() <= 1e-4


def test_full_size_objective_never_increases(ml20m):
    prob = ml20m
    m = Model(prob.data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, W0=prob.W0, H0=prob.H0,
              graph=True)
    prev = m.objective()
    for _ in range(2):
        o, st = m.epoch(1, objective=True)
        assert st == 0
        assert o <= prev * (1 + 1e-6)
        prev = o


def test_set_factors_refreshes_residual_cache():
    prob = small(d=16, seed=15)
    m = Model(prob.data, 16, 8, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    e = m.residuals()
    P = oracle.Problem.from_data(prob.data, 16, 8, 0.1, 1e-3)
    np.testing.assert_allclose(e, oracle.predict(P, prob.W0, prob.H0) - 1.0, rtol=1e-5, atol=1e-6)


def test_block_step_right_after_set_factors():
    """Replacing the factors marks the residual cache stale; a block step issued
    next (no epoch, no explicit recompute) must rebuild it from the new factors."""
    d, b = 16, 8
    prob = small(d=d, seed=16)
    m = Model(prob.data, d, b, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    assert m.block_step(0, 0) == 0
    rng = np.random.default_rng(17)
    W1 = (0.1 * rng.standard_normal(prob.W0.shape)).astype(np.float32)
    H1 = (0.1 * rng.standard_normal(prob.H0.shape)).astype(np.float32)
    m.set_factors(W1, H1)
    P = oracle.Problem.from_data(prob.data, d, b, 0.1, 1e-3)
    W, H = P.factors(W1, H1)
    yhat = oracle.predict(P, W, H)
    for side in (0, 1):
        assert m.block_step(side, 1) == 0
        assert oracle.halfstep(P, side, 1, W, H, yhat) == 0
        Wg, Hg = m.factors()
        assert rel_embed_err(Wg, W) <= STEP_TOL, side
        assert rel_embed_err(Hg, H) <= STEP_TOL, side
    e = m.residuals().astype(np.float64)
    assert np.abs(e - (yhat - 1.0)).max() <= STEP_TOL * np.abs(yhat - 1.0).max()


@pytest.mark.parametrize("d,b", [(4, 4), (20, 4), (48, 16), (100, 4), (1024, 32)])
def test_unusual_dimensions(d, b):
    prob = small(d=d, seed=16)
    m = Model(prob.data, d, b, 0.1, 1e-3, 0.3, W0=prob.W0, H0=prob.H0)
    P = oracle.Problem.from_data(prob.data, d, b, 0.1, 1e-3, 0.3)
    np.testing.assert_allclose(m.residuals(), oracle.predict(P, prob.W0, prob.H0) - 1.0,
                               rtol=1e-5, atol=1e-6)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    for side in (0, 1):
        assert m.block_step(side, d // b - 1) == 0
        oracle.halfstep(P, side, d // b - 1, W, H, yhat)
    Wg, Hg = m.factors()
    assert rel_embed_err(Wg, W) <= STEP_TOL and rel_embed_err(Hg, H) <= STEP_TOL


# --------------------------------------------------------- block sizes 64 and 128 (one CTA per row)

@pytest.mark.parametrize("b", [64, 128])
@pytest.mark.parametrize("weighted", [False, True])
def test_large_blocks_match_oracle(b, weighted):
    d = 128
    prob = small(d=d, seed=30 + b)
    data = prob.data
    y, a = weights(data.nnz, b) if weighted else (None, None)
    nu = 0.5 if weighted else 0.0
    m = Model(data, d, b, 0.1, 2e-3, nu, W0=prob.W0, H0=prob.H0, y=y, alpha=a)
    P = oracle.Problem.from_data(data, d, b, 0.1, 2e-3, nu, y=y, alpha=a)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    yref = 1.0 if y is None else y.astype(np.float64)
    for k in range(d // b):
        for side in (0, 1):
            assert m.block_step(side, k) == 0
            assert oracle.halfstep(P, side, k, W, H, yhat) == 0
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= STEP_TOL, (k, side)
            assert rel_embed_err(Hg, H) <= STEP_TOL, (k, side)
    e = m.residuals().astype(np.float64)
    assert np.abs(e - (yhat - yref)).max() <= STEP_TOL * np.abs(yhat - yref).max()


@pytest.mark.parametrize("b", [64, 128])
def test_large_blocks_long_rows_and_epochs(b):
    n_users, n_items, d = 700, 600, 128
    rng = np.random.default_rng(40 + b)
    mask = rng.random((n_users, n_items)) < 0.03
    mask[5, :] = True
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 4)
    m = Model(data, d, b, 0.1, 1e-3, 0.2, W0=W0, H0=H0)
    objs = [m.epoch(1, objective=True)[0] for _ in range(2)]
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 0.2)
    Wr, Hr, _, trace, st = oracle.ialspp(P, 2, W0, H0, trace=True)
    assert st == 0
    ref = trace.reshape(2, -1)[:, -1]
    assert np.max(np.abs(np.array(objs) - ref) / ref) <= OBJ_TOL
    W, H = m.factors()
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL


def test_large_block_fp64_retry_path():
    prob = small(d=128, seed=50)
    data = prob.data
    a = Model(data, 128, 64, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    b = Model(data, 128, 64, 0.1, 1e-3, W0=prob.W0, H0=prob.H0, force_fp64=True)
    a.epoch(1)
    _, st = b.epoch(1)
    assert st == 0
    retries, not_pd = b.stats()
    assert retries == (data.n_users + data.n_items) * 2 and not_pd == 0
    Wa, Ha = a.factors()
    Wb, Hb = b.factors()
    assert rel_embed_err(Wb, Wa) <= STEP_TOL and rel_embed_err(Hb, Ha) <= STEP_TOL


def test_autotuner_returns_the_fastest_admissible_block():
    from paper_2110_14044_gb300 import autotune
    prob = small(d=64, seed=60)
    best, table = autotune.autotune_block_size(prob.data, 64, 0.1, 1e-3, 0.0, epochs=1,
                                               W0=prob.W0, H0=prob.H0)
    assert set(table) == {1, 2, 4, 8, 16, 32, 64}
    assert best == min(table, key=table.get) and all(v > 0 for v in table.values())
    best16, t16 = autotune.autotune_block_size(prob.data, 64, 0.1, 1e-3, 0.0, epochs=1,
                                               precision=_abi.PREC_BF16, W0=prob.W0, H0=prob.H0)
    assert set(t16) == {16, 32, 64}


def test_autotuner_tunes_the_split_length_at_the_chosen_block():
    from paper_2110_14044_gb300 import autotune
    prob = synth.preset("skewed_136k", seed=61, n_users=3000, n_items=600, nnz=90_000, d=64)
    res = autotune.autotune(prob.data, 64, 0.1, 1e-3, 1.0, candidates=(16, 32),
                            split_candidates=(0, 64, 256), epochs=1, W0=prob.W0, H0=prob.H0)
    assert res["b"] in (16, 32) and res["b"] == min(res["epoch_s_by_b"], key=res["epoch_s_by_b"].get)
    assert set(res["epoch_s_by_split_len"]) == {0, 64, 256}
    assert res["split_len"] == min(res["epoch_s_by_split_len"], key=res["epoch_s_by_split_len"].get)
    assert res["epoch_s"] == res["epoch_s_by_split_len"][res["split_len"]]


@pytest.mark.parametrize("split_len,precision,d,b", [(32, _abi.PREC_FP32, 64, 32), (96, _abi.PREC_FP32, 64, 32),
                                                     (64, _abi.PREC_BF16, 64, 32), (64, _abi.PREC_FP32, 128, 64),
                                                     (96, _abi.PREC_BF16, 128, 64)])
def test_short_split_length_matches_oracle(split_len, precision, d, b):
    """A split length far below the default cuts most rows into many chunks (and
    the longest into hundreds): the chunk-order sums still give the oracle's epoch
    (b = 32: warp kernels; b = 64: the warp-pair kernels and their split-row solve)."""
    prob = synth.preset("skewed_136k", seed=62, n_users=2000, n_items=500, nnz=60_000, d=d)
    data = prob.data
    m = Model(data, d, b, 0.1, 1e-3, 1.0, precision=precision, W0=prob.W0, H0=prob.H0,
              split_len=split_len)
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 1.0)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, prob.W0, prob.H0)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    ref = oracle.objective(P, Wr, Hr)
    W, H = m.factors()
    tol_obj, tol_emb = (OBJ_TOL, EMB_TOL) if precision == _abi.PREC_FP32 else (1e-3, 5e-2)
    assert abs(o - ref) / ref <= tol_obj
    assert rel_embed_err(W, Wr) <= tol_emb and rel_embed_err(H, Hr) <= tol_emb


@pytest.mark.parametrize("precision,d,b", [(_abi.PREC_FP32, 64, 8), (_abi.PREC_FP32, 64, 32),
                                           (_abi.PREC_BF16, 64, 32), (_abi.PREC_FP32, 128, 64),
                                           (_abi.PREC_BF16, 128, 64), (_abi.PREC_FP32, 256, 128),
                                           (_abi.PREC_BF16, 256, 128)])
def test_split_item_rows_update_residuals_in_user_order(precision, d, b):
    """Item rows cut into chunks that hold most interactions update their residuals
    in one user-major scan.  Users without interactions sit between active ones,
    at both ends and in a run of 40 (more than the 32 user boundaries a warp reads
    at a time).  The residual cache after the epoch equals the residuals
    recomputed from the factors, and the epoch matches the oracle."""
    rng = np.random.default_rng(70 + b)
    n_users, n_items = 1500, 300
    active = np.ones(n_users, bool)
    active[rng.choice(n_users, 150, replace=False)] = False
    active[600:640] = False
    active[0] = active[-1] = False
    mask = (rng.random((n_users, n_items)) < 0.08) & active[:, None]
    mask[active, 3] = True  # one item held by every active user
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    assert np.diff(data.i_indptr).min() > 32  # every item row is split at split_len = 32
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 80 + b)
    m = Model(data, d, b, 0.1, 1e-3, 1.0, precision=precision, W0=W0, H0=H0, split_len=32)
    o, st = m.epoch(1, objective=True)
    assert st == 0
    W, H = m.factors()
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 1.0)
    e = m.residuals().astype(np.float64)
    ref_e = oracle.predict(P, W, H) - 1.0
    res_tol = 1e-4 if precision == _abi.PREC_FP32 else 1e-3
    assert np.abs(e - ref_e).max() <= res_tol * max(1.0, np.abs(ref_e).max())
    Wr, Hr, _, _, _ = oracle.ialspp(P, 1, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    tol_obj, tol_emb = (OBJ_TOL, EMB_TOL) if precision == _abi.PREC_FP32 else (1e-3, 5e-2)
    print(f"d={d} b={b} prec={precision}: rel objective {abs(o - ref) / ref:.2e}, "
          f"residual cache {np.abs(e - ref_e).max():.2e}")
    assert abs(o - ref) / ref <= tol_obj
    assert rel_embed_err(W, Wr) <= tol_emb and rel_embed_err(H, Hr) <= tol_emb


@pytest.mark.parametrize("precision", [_abi.PREC_FP32, _abi.PREC_BF16])
def test_relabelled_problem_gives_the_relabelled_result(precision):
    """Renaming users and items only renames the result (rows of a side are solved
    independently): the task order, the chunks of long rows, the position map and the
    user-major residual scan all change with the names, the factors only by rounding.
    Users without interactions included; every item row is cut into chunks."""
    d, b = 64, 32
    rng = np.random.default_rng(90)
    n_users, n_items = 1500, 300
    active = np.ones(n_users, bool)
    active[rng.choice(n_users, 150, replace=False)] = False
    active[600:640] = False
    active[0] = active[-1] = False
    mask = (rng.random((n_users, n_items)) < 0.08) & active[:, None]
    mask[active, 3] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 90)
    pu, pi = rng.permutation(n_users), rng.permutation(n_items)
    users = np.repeat(np.arange(n_users), np.diff(data.u_indptr))
    data2 = synth.from_pairs(n_users, n_items, pu[users], pi[np.asarray(data.u_items)])
    W2, H2 = np.empty_like(W0), np.empty_like(H0)
    W2[pu], H2[pi] = W0, H0
    m1 = Model(data, d, b, 0.1, 1e-3, 1.0, precision=precision, W0=W0, H0=H0, split_len=32)
    m2 = Model(data2, d, b, 0.1, 1e-3, 1.0, precision=precision, W0=W2, H0=H2, split_len=32)
    o1, st1 = m1.epoch(2, objective=True)
    o2, st2 = m2.epoch(2, objective=True)
    assert st1 == 0 and st2 == 0
    Wa, Ha = m1.factors()
    Wb, Hb = m2.factors()
    tol = 1e-4 if precision == _abi.PREC_FP32 else 1e-3  # measured 4e-6 / 3e-5: rounding order only
    print(f"prec={precision}: relabelled W {rel_embed_err(Wb[pu], Wa):.2e} H {rel_embed_err(Hb[pi], Ha):.2e}, "
          f"objective {abs(o1 - o2) / o1:.2e}")
    assert rel_embed_err(Wb[pu], Wa) <= tol and rel_embed_err(Hb[pi], Ha) <= tol
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 1.0)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    obj_tol = OBJ_TOL if precision == _abi.PREC_FP32 else 1e-3
    assert abs(o1 - ref) <= obj_tol * ref and abs(o2 - ref) <= obj_tol * ref


@pytest.mark.parametrize("b,precision", [(16, _abi.PREC_FP32), (64, _abi.PREC_FP32), (32, _abi.PREC_BF16)])
def test_skewed_user_activity_epochs(b, precision):
    """Zipf(1.3) user activity with rows capped at the whole catalogue (the skewed
    workload's shape, scaled down): every row length class in one launch."""
    d = 64
    prob = synth.preset("skewed_136k", seed=9, n_users=3000, n_items=600, nnz=90_000, d=d)
    data = prob.data
    assert np.diff(data.u_indptr).max() == data.n_items
    m = Model(data, d, b, 0.1, 1e-3, 1.0, precision=precision, graph=True, W0=prob.W0, H0=prob.H0)
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 1.0)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, prob.W0, prob.H0)
    ref = oracle.objective(P, Wr, Hr)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    W, H = m.factors()
    tol_obj, tol_emb = (OBJ_TOL, EMB_TOL) if precision == _abi.PREC_FP32 else (1e-3, 5e-2)
    assert abs(o - ref) / ref <= tol_obj
    assert rel_embed_err(W, Wr) <= tol_emb and rel_embed_err(H, Hr) <= tol_emb


def test_profile_and_work_model_hooks():
    """bench.py's measurement hooks: per-kernel event times cover the profiled epochs,
    launch counts follow the block structure, and with no split rows the sparse step's
    algorithmic bytes are the per-interaction figure (column id, b-slice, residual read
    and write, plus the position map on the item side) and the per-row terms."""
    n_users, n_items, d, b = 400, 300, 32, 8
    rng = np.random.default_rng(71)
    u, i = np.nonzero(rng.random((n_users, n_items)) < 0.05)   # short rows only: no splits
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 71)
    m = Model(data, d, b, 0.1, 1e-3, 0.5, W0=W0, H0=H0)
    epochs, nb = 2, d // b
    kern, total, st = _abi.ials_profile_epochs(m.ctx, epochs)
    assert st == 0 and total > 0
    ms = sum(v[0] for v in kern.values())
    assert 0.3 * total <= ms <= 1.05 * total
    assert kern["residual"][1] == epochs
    assert kern["sparse"][1] == epochs * nb * 2
    assert kern["split_solve"][1] == 0 and kern["split_resid"][1] == 0
    work = _abi.ials_work_model(m.ctx)
    nnz, rows = data.nnz, n_users + n_items
    per_nz = (4 + 4 * b + 4 + 4) + (4 + 4 * b + 4 + 4 + 4)      # user side + item side
    per_row = 4 * b + 8 * b + 16 + 24                           # R read, x read/write, ptr, task
    assert work["sparse"][0] == pytest.approx(nb * (nnz * per_nz + rows * per_row), rel=1e-12)
    # Gramian FLOPs: 2 |fixed| d b per half-step (Eq. 10)
    assert work["gram"][1] == pytest.approx(nb * 2 * (n_items + n_users) * d * b, rel=1e-12)


# --------------------------------------------------------- block size 256 (FP32)

@pytest.mark.parametrize("weighted", [False, True])
def test_block_size_256_steps_and_epochs(weighted):
    """b = 256 (d = 512): single block steps against the oracle, then an epoch with
    rows long enough to be cut into chunks (split-row path) against the oracle."""
    d, b = 512, 256
    n_users, n_items = 1200, 1000  # more rows than d on both sides: well-conditioned Gramians
    rng = np.random.default_rng(70 + weighted)
    mask = rng.random((n_users, n_items)) < 0.02
    mask[5, :] = True   # longer than the chunk length on both sides
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 7)
    y, a = weights(data.nnz, 71) if weighted else (None, None)
    m = Model(data, d, b, 0.1, 2e-3, 0.5, W0=W0, H0=H0, y=y, alpha=a)
    P = oracle.Problem.from_data(data, d, b, 0.1, 2e-3, 0.5, y=y, alpha=a)
    W, H = P.factors(W0, H0)
    yhat = oracle.predict(P, W, H)
    for k in range(d // b):
        for side in (0, 1):
            assert m.block_step(side, k) == 0
            assert oracle.halfstep(P, side, k, W, H, yhat) == 0
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= STEP_TOL and rel_embed_err(Hg, H) <= STEP_TOL, (k, side)
    o, st = m.epoch(1, objective=True)
    assert st == 0
    Wr, Hr, _, _, _ = oracle.ialspp(P, 1, W, H)
    assert abs(o - oracle.objective(P, Wr, Hr)) <= OBJ_TOL * abs(o)


def test_block_size_256_fp64_retry_and_ials_path():
    """Every FP32 pivot treated as failed at b = 256: the FP64 re-solve (its systems
    in global memory above b = 128) gives the same step; b = d = 256 runs the
    iALS path (Algorithm 1) and matches the oracle's closed form."""
    d = 256
    # more users and items than d, so that the Gramians (and the row systems) are
    # well conditioned enough for an FP32 comparison
    prob = small(n_users=1500, n_items=1200, nnz=30000, seed=72, d=d, len_max=400)
    data = prob.data
    a = Model(data, d, 256, 0.1, 1e-3, W0=prob.W0, H0=prob.H0, general=True)
    f = Model(data, d, 256, 0.1, 1e-3, W0=prob.W0, H0=prob.H0, general=True, force_fp64=True)
    assert a.block_step(0, 0) == 0 and f.block_step(0, 0) == 0
    retries, not_pd = f.stats()
    assert retries == data.n_users and not_pd == 0
    assert rel_embed_err(f.factors()[0], a.factors()[0]) <= STEP_TOL
    # both half-steps of the general path at b = d against the oracle.  A row with
    # no interactions has the exact solution 0 here (its row term is its Hessian
    # times the old row), so the rounding left in it scales with the old row:
    # errors are measured against the larger of the old and the new row norms.
    P = oracle.Problem.from_data(data, d, 256, 0.1, 1e-3, 0.0)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    for side in (0, 1):
        if side == 1:
            assert a.block_step(1, 0) == 0
        old = (W if side == 0 else H).copy()
        assert oracle.halfstep(P, side, 0, W, H, yhat) == 0
        got, ref = a.factors()[side].astype(np.float64), (W if side == 0 else H)
        scale = np.maximum(np.linalg.norm(ref, axis=1), np.linalg.norm(old, axis=1))
        assert np.max(np.linalg.norm(got - ref, axis=1) / scale) <= STEP_TOL, side
    e = a.residuals().astype(np.float64)
    assert np.abs(e - (yhat - 1.0)).max() <= STEP_TOL * np.abs(yhat - 1.0).max()
    m = Model(data, d, d, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0)
    m.epoch(1)
    W, H = m.factors()
    P = oracle.Problem.from_data(data, d, d, 0.1, 1e-3, 0.0)
    Wr, Hr, st = oracle.ials(P, 1, prob.W0, prob.H0)
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
