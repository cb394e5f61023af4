"""Fold-in serving (ials_foldin_*) against the FP64 oracle, and its batching behaviour."""
import threading

import numpy as np
import pytest

import oracle
from paper_2110_14044_gb300 import _abi

pytestmark = pytest.mark.gpu

TOL = 1e-4  # FP32 solve of well-conditioned b x b systems, a few sweeps


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14044_gb300 import build
    build.build()
    oracle.build()


def server(*a, **k):
    import paper_2110_14044_gb300 as ials
    return ials.FoldinServer(*a, **k)


def requests(n_items, count, seed, max_len=300):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(np.exp(rng.uniform(0, np.log(max_len)))) if k % 7 else 0
        items = rng.choice(n_items, size=min(n, n_items), replace=False).astype(np.int32)
        y = rng.uniform(0.5, 1.5, items.size).astype(np.float32) if k % 3 == 1 else None
        out.append((items, y))
    return out


def rel(w, ref):
    return np.linalg.norm(w - ref) / max(np.linalg.norm(ref), 1e-12)


@pytest.mark.parametrize("d,b,sweeps", [(64, 16, 4), (64, 32, 1), (128, 64, 4), (256, 64, 4), (128, 128, 2)])
def test_foldin_matches_oracle(d, b, sweeps):
    rng = np.random.default_rng(d + b)
    n_items = 700
    H = rng.normal(0, 0.05, (n_items, d)).astype(np.float32)
    srv = server(H, d, b, 0.1, 1e-2, 0.5, sweeps=sweeps, workspace_bytes=256 << 20)
    reqs = requests(n_items, 25, d)
    tickets = [srv.submit(it, y) for it, y in reqs]
    for (items, y), t in zip(reqs, tickets):
        w = srv.result(t)
        ref, st = oracle.foldin(H, d, b, 0.1, 1e-2, 0.5, sweeps, items, y=y)
        assert st == 0
        assert rel(w, ref) <= TOL, (items.size, rel(w, ref))
    srv.close()


def test_foldin_one_sweep_b_eq_d_is_closed_form():
    rng = np.random.default_rng(1)
    d = 64
    H = rng.normal(0, 0.2, (300, d)).astype(np.float32)
    items = rng.choice(300, 40, replace=False).astype(np.int32)
    srv = server(H, d, d, 0.2, 0.05, 0.0, sweeps=1, workspace_bytes=64 << 20)
    w = srv.result(srv.submit(items))
    Hd = H.astype(np.float64)
    A = Hd[items].T @ Hd[items] + 0.2 * Hd.T @ Hd + 0.05 * np.eye(d)   # Eq. 3 with y = alpha = 1
    ref = np.linalg.solve(A, Hd[items].sum(axis=0))
    assert rel(w, ref) <= TOL
    srv.close()


def test_foldin_result_does_not_depend_on_the_batch():
    rng = np.random.default_rng(2)
    d, b = 128, 32
    H = rng.normal(0, 0.05, (2000, d)).astype(np.float32)
    srv = server(H, d, b, 0.1, 1e-2, 1.0, sweeps=4, workspace_bytes=512 << 20)
    probe = rng.choice(2000, 500, replace=False).astype(np.int32)
    alone = srv.result(srv.submit(probe))
    others = requests(2000, 400, 3, max_len=2000)

    def flood(part):
        for it, y in part:
            srv.submit(it, y)

    shared = False
    for attempt in range(5):  # until the probe is seen to share its batch with others
        threads = [threading.Thread(target=flood, args=(others[k::4],)) for k in range(4)]
        for t in threads:
            t.start()
        mixed_ticket = srv.submit(probe)
        for t in threads:
            t.join()
        mixed, info = srv.result_info(mixed_ticket)
        np.testing.assert_array_equal(alone, mixed)
        assert info["cluster"]  # 500 interactions: split over a CTA cluster
        if info["batch_size"] > 1:
            shared = True
            break
    assert shared, "the probe never landed in a batch with other requests"
    srv.close()


@pytest.mark.parametrize("n", [1, 384, 385, 3000])
def test_foldin_long_requests_on_clusters_match_oracle(n):
    """Requests above the one-CTA limit run on a cluster of CTAs that share the
    interactions; the result still matches the oracle, and a short request in the
    same batch is unaffected."""
    rng = np.random.default_rng(10 + n)
    d, b, n_items = 256, 64, 5000
    H = rng.normal(0, 0.05, (n_items, d)).astype(np.float32)
    srv = server(H, d, b, 0.1, 1e-3, 1.0, sweeps=4, workspace_bytes=1 << 30)
    items = rng.choice(n_items, n, replace=False).astype(np.int32)
    y = rng.uniform(0.5, 2.0, n).astype(np.float32)
    short = rng.choice(n_items, 50, replace=False).astype(np.int32)
    t1, t2 = srv.submit(items, y), srv.submit(short)
    w, info = srv.result_info(t1)
    w2, info2 = srv.result_info(t2)
    assert info["cluster"] == (n > 384) and not info2["cluster"]
    ref, st = oracle.foldin(H, d, b, 0.1, 1e-3, 1.0, 4, items, y=y)
    assert st == 0
    assert rel(w, ref) <= TOL, rel(w, ref)
    ref2, _ = oracle.foldin(H, d, b, 0.1, 1e-3, 1.0, 4, short)
    assert rel(w2, ref2) <= TOL
    srv.close()


def test_foldin_memory_admission_and_poll_semantics():
    rng = np.random.default_rng(4)
    d, b = 64, 32
    H = rng.normal(0, 0.05, (1000, d)).astype(np.float32)
    # room for only a few requests at a time: the rest must wait for memory
    srv = server(H, d, b, 0.1, 1e-2, 0.0, sweeps=2, workspace_bytes=200 << 10)
    reqs = requests(1000, 60, 5, max_len=400)
    tickets = [srv.submit(it, y) for it, y in reqs]
    for (items, y), t in zip(reqs, tickets):
        w = srv.result(t, timeout_s=60)
        ref, _ = oracle.foldin(H, d, b, 0.1, 1e-2, 0.0, 2, items, y=y)
        assert rel(w, ref) <= TOL
    with pytest.raises(_abi.IalsError) as ei:
        srv.poll(tickets[0])  # already collected
    assert ei.value.status == _abi.ENOTFOUND
    with pytest.raises(_abi.IalsError) as ei:
        srv.submit(np.arange(1000, dtype=np.int32) % 1000 + 1000)  # ids out of range
    assert ei.value.status == _abi.EINVAL
    with pytest.raises(_abi.IalsError):
        srv.submit(np.zeros(60000, np.int32))  # can never fit 200 KB
    srv.close()
