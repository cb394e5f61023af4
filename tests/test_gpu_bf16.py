"""The BF16 tensor-core path (precision IALS_PREC_BF16) against the FP64 oracle.

The BF16 form must stay within 1e-3 relative objective of the oracle per epoch.
Each product keeps about 16 bits (hi*hi + hi*lo + lo*hi), so block steps are
held to 1e-3 relative embedding error and whole runs are reported.
"""
import numpy as np
import pytest

import oracle
from paper_2110_14044_gb300 import _abi, synth

pytestmark = pytest.mark.gpu

BF16_OBJ_TOL = 1e-3


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
    return ials.Model(*a, precision=_abi.PREC_BF16, **k)


def rel_embed_err(X, Xref):
    X = np.asarray(X, np.float64)
    Xref = np.asarray(Xref, np.float64)
    nref = np.linalg.norm(Xref, axis=1)
    floor = max(1e-6 * np.median(nref), 1e-30)
    return float(np.max(np.linalg.norm(X - Xref, axis=1) / np.maximum(nref, floor)))


@pytest.mark.parametrize("d,b", [(32, 16), (32, 32), (128, 32)])
def test_bf16_epochs_within_objective_tolerance(d, b):
    prob = synth.preset("parity_2k", seed=3, d=d, b=b)
    data = prob.data
    m = Model(data, d, b, prob.alpha0, prob.lam, 0.5, W0=prob.W0, H0=prob.H0)
    objs = []
    for _ in range(prob.epochs):
        o, st = m.epoch(1, objective=True)
        assert st == 0
        objs.append(o)
    P = oracle.Problem.from_data(data, d, b, prob.alpha0, prob.lam, 0.5)
    Wr, Hr, _, trace, st = oracle.ialspp(P, prob.epochs, prob.W0, prob.H0, trace=True)
    ref = trace.reshape(prob.epochs, -1)[:, -1]
    rel = np.abs(np.array(objs) - ref) / ref
    W, H = m.factors()
    print(f"bf16 d={d} b={b}: max rel objective {rel.max():.2e}, "
          f"embedding W {rel_embed_err(W, Wr):.2e} H {rel_embed_err(H, Hr):.2e}")
    assert rel.max() <= BF16_OBJ_TOL
    assert rel_embed_err(W, Wr) <= 5e-2 and rel_embed_err(H, Hr) <= 5e-2


@pytest.mark.parametrize("b", [16, 32, 64, 128])
def test_bf16_block_steps(b):
    d = 64 if b <= 32 else 128
    prob = synth.preset("parity_2k", seed=b, n_users=300, n_items=200, nnz=6000, len_max=200, d=d)
    data = prob.data
    m = Model(data, d, b, 0.1, 2e-3, 0.3, W0=prob.W0, H0=prob.H0)
    P = oracle.Problem.from_data(data, d, b, 0.1, 2e-3, 0.3)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    for k in range(min(2, d // b)):
        for side in (0, 1):
            assert m.block_step(side, k) == 0
            oracle.halfstep(P, side, k, W, H, yhat)
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= 1e-3 and rel_embed_err(Hg, H) <= 1e-3, (k, side)
    e = m.residuals().astype(np.float64)
    assert np.abs(e - (yhat - 1.0)).max() <= 1e-3 * np.abs(yhat - 1.0).max()


def test_bf16_long_rows_and_determinism():
    n_users, n_items, d, b = 700, 600, 32, 32
    rng = np.random.default_rng(5)
    mask = rng.random((n_users, n_items)) < 0.03
    mask[5, :] = True
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 5)
    runs = []
    for graph in (False, True):
        m = Model(data, d, b, 0.1, 1e-3, 0.2, W0=W0, H0=H0, graph=graph)
        o, st = m.epoch(2, objective=True)
        assert st == 0
        runs.append((o, *m.factors()))
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 0.2)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    assert abs(runs[0][0] - ref) / ref <= BF16_OBJ_TOL


@pytest.mark.parametrize("b", [64, 128])
def test_bf16_large_blocks_long_rows_and_epochs(b):
    """CTA kernels (b = 64, 128): rows cut into chunks, graph replay, objective vs the oracle."""
    n_users, n_items, d = 500, 400, 128
    rng = np.random.default_rng(b)
    mask = rng.random((n_users, n_items)) < 0.04
    mask[3, :] = True        # a long user row
    mask[:, 11] = True       # a long item row
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), b)
    runs = []
    for graph in (False, True):
        m = Model(data, d, b, 0.1, 1e-3, 0.3, W0=W0, H0=H0, graph=graph)
        o, st = m.epoch(2, objective=True)
        assert st == 0
        runs.append((o, *m.factors()))
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    np.testing.assert_array_equal(runs[0][2], runs[1][2])
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 0.3)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    print(f"b={b}: objective rel err {abs(runs[0][0] - ref) / ref:.2e}, "
          f"embedding W {rel_embed_err(runs[0][1], Wr):.2e} H {rel_embed_err(runs[0][2], Hr):.2e}")
    assert abs(runs[0][0] - ref) / ref <= BF16_OBJ_TOL
    assert rel_embed_err(runs[0][1], Wr) <= 5e-2 and rel_embed_err(runs[0][2], Hr) <= 5e-2


def test_bf16_fp64_retry_updates_shadows():
    prob = synth.preset("parity_2k", seed=7, n_users=300, n_items=200, nnz=6000, len_max=200, d=32, b=16)
    a = Model(prob.data, 32, 16, 0.1, 1e-3, W0=prob.W0, H0=prob.H0)
    b = Model(prob.data, 32, 16, 0.1, 1e-3, W0=prob.W0, H0=prob.H0, force_fp64=True)
    oa, _ = a.epoch(2, objective=True)
    ob, st = b.epoch(2, objective=True)
    assert st == 0 and b.stats()[0] > 0
    assert abs(oa - ob) / oa <= 1e-4


def test_bf16_rejects_unsupported_inputs():
    prob = synth.preset("parity_2k", seed=8, n_users=50, n_items=40, nnz=500, len_max=40, d=32, b=8)
    with pytest.raises(_abi.IalsError):
        Model(prob.data, 32, 8, 0.1, 1e-3)   # b = 8
    with pytest.raises(_abi.IalsError):
        Model(prob.data, 36, 4, 0.1, 1e-3)   # b = 4, d % 8 != 0
    # weighted data is supported on this path (test_bf16_weighted_*)
    Model(prob.data, 32, 16, 0.1, 1e-3, alpha=np.ones(prob.data.nnz, np.float32)).close()


@pytest.mark.parametrize("n,d,p0,bs", [(1, 8, 0, 16), (64, 128, 32, 32), (1000, 64, 48, 16),
                                       (20011, 128, 96, 32), (136000, 128, 0, 32), (5000, 256, 224, 32),
                                       (3000, 1024, 512, 32), (5000, 256, 64, 64), (20011, 128, 0, 128),
                                       (3000, 1024, 896, 128)])
def test_tcgen05_gramian(n, d, p0, bs):
    """tcgen05 Gramian (BF16 hi/lo, FP32 accumulate) against FP64 numpy."""
    import torch
    if d < p0 + bs:
        pytest.skip("block outside d")
    rng = np.random.default_rng(n)
    X = rng.normal(0, 0.3, (n, d)).astype(np.float32)
    G = torch.full((d, bs), float("nan"), dtype=torch.float32, device="cuda")
    _abi.ials_partial_gramian_bf16(torch.from_numpy(X).cuda(), n, d, p0, bs, G)
    ref = X.astype(np.float64).T @ X[:, p0:p0 + bs].astype(np.float64)
    got = G.cpu().numpy()
    err = np.abs(got - ref).max() / max(np.abs(ref).max(), 1e-30)
    assert err <= 1e-4, err


def test_msd_shaped_subsample_bf16_b128_sampled_rows():
    """The d = 1024 configuration (BF16 pattern, b = 128) on its 1% user subsample
    (5,700 users x 41,000 items, 340,000 positives; a whole oracle epoch there takes
    minutes of FP64 Cholesky): after one GPU epoch, one user and one item block step
    are checked row by row against the oracle evaluated from the same state, on the
    longest rows and a random sample."""
    prob = synth.preset("msd_570k", seed=0, n_users=5700, nnz=340_000)
    assert prob.d == 1024 and prob.b == 128
    data = prob.data
    m = Model(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu, W0=prob.W0, H0=prob.H0)
    assert m.epoch(1)[1] == 0
    P = oracle.Problem.from_data(data, prob.d, prob.b, prob.alpha0, prob.lam, prob.nu)
    rng = np.random.default_rng(3)
    for side, block in ((0, 2), (1, 2)):
        W, H = m.factors()
        yhat = oracle.predict(P, W, H)  # from the factors (Eq. 1), not from the GPU's cache
        assert np.abs(m.residuals() - (yhat - 1.0)).max() <= 1e-4, side
        lens = np.diff(data.u_indptr if side == 0 else data.i_indptr)
        rows = np.unique(np.concatenate([np.argsort(-lens)[:4], rng.integers(0, lens.size, 40)]))
        st, ref = oracle.rows_step(P, side, block, W, H, yhat, rows)
        assert np.all(st == 0)
        assert m.block_step(side, block) == 0
        W2, H2 = m.factors()
        got = (W2 if side == 0 else H2)[rows, block * prob.b:(block + 1) * prob.b]
        err = np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-12)
        print(f"side {side}: max row rel err {err.max():.2e}")
        assert err.max() <= 1e-3, (side, err.max())


@pytest.mark.parametrize("b", [16, 32, 64, 128])
def test_bf16_weighted_block_steps(b):
    """General (y, alpha) data on the BF16 pattern: rows scaled by sqrt(alpha) before
    the compensated products; single block steps against the oracle."""
    d = 64 if b <= 32 else 128
    prob = synth.preset("parity_2k", seed=50 + b, n_users=300, n_items=200, nnz=6000, len_max=200, d=d)
    data = prob.data
    rng = np.random.default_rng(b)
    y = rng.uniform(0.5, 2.0, data.nnz).astype(np.float32)
    al = rng.uniform(0.5, 3.0, data.nnz).astype(np.float32)
    m = Model(data, d, b, 0.1, 2e-3, 0.3, W0=prob.W0, H0=prob.H0, y=y, alpha=al)
    P = oracle.Problem.from_data(data, d, b, 0.1, 2e-3, 0.3, y=y, alpha=al)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    for k in range(min(2, d // b)):
        for side in (0, 1):
            assert m.block_step(side, k) == 0
            oracle.halfstep(P, side, k, W, H, yhat)
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= 1e-3 and rel_embed_err(Hg, H) <= 1e-3, (k, side)
    e = m.residuals().astype(np.float64)
    ref_e = yhat - y.astype(np.float64)
    assert np.abs(e - ref_e).max() <= 1e-3 * np.abs(ref_e).max()


@pytest.mark.parametrize("d,b", [(32, 32), (128, 64), (128, 128)])
def test_bf16_weighted_epochs_with_long_rows(d, b):
    """Weighted epochs with rows long enough to be cut into chunks, against the
    oracle's objective (1e-3) and embeddings."""
    n_users, n_items = 700, 600
    rng = np.random.default_rng(60 + b)
    mask = rng.random((n_users, n_items)) < 0.03
    mask[5, :] = True
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), 6)
    y = rng.uniform(0.5, 2.0, data.nnz).astype(np.float32)
    al = rng.uniform(0.5, 3.0, data.nnz).astype(np.float32)
    m = Model(data, d, b, 0.1, 1e-3, 0.2, W0=W0, H0=H0, y=y, alpha=al, graph=True)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    P = oracle.Problem.from_data(data, d, b, 0.1, 1e-3, 0.2, y=y, alpha=al)
    Wr, Hr, _, _, _ = oracle.ialspp(P, 2, W0, H0) if b < d else (*oracle.ials(P, 2, W0, H0)[:2], None, None, None)
    ref = oracle.objective(P, Wr, Hr)
    W, H = m.factors()
    print(f"bf16 weighted d={d} b={b}: rel objective {abs(o - ref) / ref:.2e}, "
          f"embedding W {rel_embed_err(W, Wr):.2e} H {rel_embed_err(H, Hr):.2e}")
    assert abs(o - ref) <= BF16_OBJ_TOL * ref
    assert rel_embed_err(W, Wr) <= 5e-2 and rel_embed_err(H, Hr) <= 5e-2
