"""The end points of the block size through their own GPU paths: b = 1 runs
iCD (Algorithm 2, Eqs. 5-7: one coordinate per pass, Gramian columns formed
on the way) and b = d in {64, 128} runs iALS (Algorithm 1, Eq. 3: rows solved
for directly, no residual cache).  Each is checked against the FP64 oracle's
own Algorithm 2 / Algorithm 1 routines, and against the library's general
block path (IALS_FLAG_GENERAL), on weighted data and with long rows cut into
chunks."""
import numpy as np
import pytest

import oracle
from paper_2110_14044_gb300 import _abi, synth

pytestmark = pytest.mark.gpu

OBJ_TOL = 1e-5
EMB_TOL = 1e-3
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
    return ials.Model(*a, **k)


def rel_embed_err(X, Xref):
    X = np.asarray(X, np.float64)
    Xref = np.asarray(Xref, np.float64)
    nref = np.linalg.norm(Xref, axis=1)
    floor = max(1e-6 * np.median(nref), 1e-30)
    return float(np.max(np.linalg.norm(X - Xref, axis=1) / np.maximum(nref, floor)))


def long_row_problem(d, seed, n_users=700, n_items=600, density=0.03):
    """Random pattern plus one user holding every item and one item held by every
    user (both longer than the chunk length, so both sides cut rows into chunks)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n_users, n_items)) < density
    mask[5, :] = True
    mask[:, 7] = True
    u, i = np.nonzero(mask)
    data = synth.from_pairs(n_users, n_items, u, i)
    W0, H0 = synth.init_factors(n_users, n_items, d, 0.1 / np.sqrt(d), seed)
    y = rng.uniform(0.5, 2.0, data.nnz).astype(np.float32)
    a = rng.uniform(0.5, 3.0, data.nnz).astype(np.float32)
    return data, W0, H0, y, a


@pytest.mark.parametrize("weighted", [False, True])
def test_icd_path_matches_oracle_algorithm_2(weighted):
    d = 16
    data, W0, H0, y, a = long_row_problem(d, 11)
    if not weighted:
        y = a = None
    m = Model(data, d, 1, 0.1, 1e-3, 0.5, W0=W0, H0=H0, y=y, alpha=a)
    objs = []
    for _ in range(3):
        o, st = m.epoch(1, objective=True)
        assert st == 0
        objs.append(o)
    W, H = m.factors()
    P = oracle.Problem.from_data(data, d, 1, 0.1, 1e-3, 0.5, y=y, alpha=a)
    Wr, Hr, _, st = oracle.icd(P, 3, W0, H0)
    assert st == 0
    ref = oracle.objective(P, Wr, Hr)
    print(f"iCD weighted={weighted}: rel objective {abs(objs[-1] - ref) / ref:.2e}, "
          f"embedding W {rel_embed_err(W, Wr):.2e} H {rel_embed_err(H, Hr):.2e}")
    assert abs(objs[-1] - ref) <= OBJ_TOL * ref
    assert objs[0] >= objs[1] >= objs[2]
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
    # the general block path at b = 1 computes the same iteration
    g = Model(data, d, 1, 0.1, 1e-3, 0.5, W0=W0, H0=H0, y=y, alpha=a, general=True)
    g.epoch(3)
    Wg, Hg = g.factors()
    assert rel_embed_err(W, Wg) <= EMB_TOL and rel_embed_err(H, Hg) <= EMB_TOL


def test_icd_path_single_coordinate_steps_and_graph():
    """ials_block_step at b = 1 is one coordinate of iCD on one side; a CUDA-graph
    epoch gives bitwise the same factors as an eager one."""
    d = 8
    prob = synth.preset("parity_2k", seed=12, n_users=300, n_items=200, nnz=6000, len_max=200, d=d)
    data = prob.data
    m = Model(data, d, 1, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0)
    P = oracle.Problem.from_data(data, d, 1, 0.1, 1e-3, 0.0)
    W, H = P.factors(prob.W0, prob.H0)
    yhat = oracle.predict(P, W, H)
    for f in (0, 5):
        for side in (0, 1):
            assert m.block_step(side, f) == 0
            assert oracle.halfstep(P, side, f, W, H, yhat) == 0
            Wg, Hg = m.factors()
            assert rel_embed_err(Wg, W) <= 1e-4 and rel_embed_err(Hg, H) <= 1e-4, (f, side)
    e = m.residuals().astype(np.float64)
    assert np.abs(e - (yhat - 1.0)).max() <= 1e-4 * np.abs(yhat - 1.0).max()
    a = Model(data, d, 1, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0)
    b = Model(data, d, 1, 0.1, 1e-3, 0.0, W0=prob.W0, H0=prob.H0, graph=True)
    a.epoch(2)
    b.epoch(2)
    for x, z in zip(a.factors(), b.factors()):
        assert np.array_equal(x, z)


@pytest.mark.parametrize("d", [64, 128])
@pytest.mark.parametrize("weighted", [False, True])
def test_ials_path_matches_oracle_algorithm_1(d, weighted):
    data, W0, H0, y, a = long_row_problem(d, 20 + d)
    if not weighted:
        y = a = None
    m = Model(data, d, d, 0.1, 1e-3, 0.5, W0=W0, H0=H0, y=y, alpha=a)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    W, H = m.factors()
    P = oracle.Problem.from_data(data, d, d, 0.1, 1e-3, 0.5, y=y, alpha=a)
    Wr, Hr, st = oracle.ials(P, 2, W0, H0)
    assert st == 0
    ref = oracle.objective(P, Wr, Hr)
    print(f"iALS d={d} weighted={weighted}: rel objective {abs(o - ref) / ref:.2e}, "
          f"embedding W {rel_embed_err(W, Wr):.2e} H {rel_embed_err(H, Hr):.2e}")
    assert abs(o - ref) <= OBJ_TOL * ref
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
    # after an iALS epoch the residual cache is rebuilt on demand from the factors
    e = m.residuals().astype(np.float64)
    ref_e = oracle.predict(P, W, H) - (1.0 if y is None else y.astype(np.float64))
    assert np.abs(e - ref_e).max() <= 1e-4 * max(1.0, np.abs(ref_e).max())


@pytest.mark.parametrize("d", [64, 128])
def test_ials_path_bf16_and_fp64_retry(d):
    data, W0, H0, _, _ = long_row_problem(d, 30 + d)
    P = oracle.Problem.from_data(data, d, d, 0.1, 1e-3, 0.5)
    Wr, Hr, st = oracle.ials(P, 2, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    m = Model(data, d, d, 0.1, 1e-3, 0.5, W0=W0, H0=H0, precision=_abi.PREC_BF16, graph=True)
    o, st = m.epoch(2, objective=True)
    assert st == 0
    print(f"iALS BF16 d={d}: rel objective {abs(o - ref) / ref:.2e}")
    assert abs(o - ref) <= BF16_OBJ_TOL * ref
    # every FP32 pivot treated as failed: all rows re-solved in FP64, same answer
    f = Model(data, d, d, 0.1, 1e-3, 0.5, W0=W0, H0=H0, force_fp64=True)
    o64, st = f.epoch(2, objective=True)
    assert st == 0
    n_retry, n_notpd = f.stats()
    assert n_retry == 2 * (data.n_users + data.n_items) and n_notpd == 0  # two epochs
    W, H = f.factors()
    assert abs(o64 - ref) <= OBJ_TOL * ref
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL


@pytest.mark.parametrize("weighted", [False, True])
def test_ials_above_b_256_matches_oracle_algorithm_1(weighted):
    """b = d = 320: the row systems no longer fit on chip and live in a global
    workspace (5 x 5 tiles of 64); long rows are taken whole by one block."""
    d = 320
    data, W0, H0, y, a = long_row_problem(d, 40 + weighted)
    if not weighted:
        y = a = None
    m = Model(data, d, d, 0.1, 1e-3, 0.5, W0=W0, H0=H0, y=y, alpha=a, graph=True)
    o, st = m.epoch(2, objective=True)
    assert st == 0 and m.stats() == (0, 0)
    W, H = m.factors()
    P = oracle.Problem.from_data(data, d, d, 0.1, 1e-3, 0.5, y=y, alpha=a)
    Wr, Hr, st = oracle.ials(P, 2, W0, H0)
    assert st == 0
    ref = oracle.objective(P, Wr, Hr)
    print(f"iALS d={d} weighted={weighted}: rel objective {abs(o - ref) / ref:.2e}, "
          f"embedding W {rel_embed_err(W, Wr):.2e} H {rel_embed_err(H, Hr):.2e}")
    assert abs(o - ref) <= OBJ_TOL * ref
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
    with pytest.raises(_abi.IalsError):  # no general block step above b = 256
        m.block_step(0, 0)


def test_ials_above_b_256_fp64_retry():
    """Every FP32 pivot treated as failed: every row re-solved by the FP64 form of the
    same kernel, with the oracle's answer."""
    d = 320
    data, W0, H0, _, _ = long_row_problem(d, 50, n_users=400, n_items=500)
    P = oracle.Problem.from_data(data, d, d, 0.1, 1e-3, 0.5)
    Wr, Hr, st = oracle.ials(P, 1, W0, H0)
    ref = oracle.objective(P, Wr, Hr)
    f = Model(data, d, d, 0.1, 1e-3, 0.5, W0=W0, H0=H0, force_fp64=True)
    o64, st = f.epoch(1, objective=True)
    assert st == 0
    assert f.stats() == (data.n_users + data.n_items, 0)
    W, H = f.factors()
    assert abs(o64 - ref) <= OBJ_TOL * ref
    assert rel_embed_err(W, Wr) <= EMB_TOL and rel_embed_err(H, Hr) <= EMB_TOL
