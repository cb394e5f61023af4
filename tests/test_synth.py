"""The seeded input generator (no method arithmetic): shapes the benchmarks rely on."""
import numpy as np

from paper_2110_14044_gb300 import synth


def _check_csr(data):
    ul = np.diff(data.u_indptr)
    assert ul.sum() == data.nnz == data.u_items.size
    for u in range(data.n_users):   # sorted, distinct items per row
        row = data.u_items[data.u_indptr[u]:data.u_indptr[u + 1]]
        assert np.all(np.diff(row) > 0)
    # the item view is the exact transpose
    t_ptr, t_idx = synth.transpose_csr(data.n_users, data.n_items, data.u_indptr, data.u_items)
    np.testing.assert_array_equal(t_ptr, data.i_indptr)
    np.testing.assert_array_equal(t_idx, data.i_users)


def test_lognormal_lengths_hit_nnz_and_clip():
    d = synth.make_interactions(1500, 400, 30_000, 1.0, 2.5, 1.0, 2, 300, seed=3)
    ul = np.diff(d.u_indptr)
    assert d.nnz == 30_000 and ul.min() >= 2 and ul.max() <= 300
    _check_csr(d)


def test_zipf_user_activity_is_skewed_and_capped_at_the_catalogue():
    n_users, n_items, nnz = 2000, 500, 60_000
    d = synth.make_interactions(n_users, n_items, nnz, 1.05, 0.0, 0.0, 5, 200_000, seed=4,
                                user_zipf=1.3)
    ul = np.diff(d.u_indptr)
    assert d.nnz == nnz and ul.min() >= 5
    assert ul.max() == n_items                      # the heaviest users hold the whole catalogue
    assert np.median(ul) < 0.3 * ul.mean()          # and most users very little (lognormal(2.5, 1): 0.61)
    _check_csr(d)
    # same seed, same data
    d2 = synth.make_interactions(n_users, n_items, nnz, 1.05, 0.0, 0.0, 5, 200_000, seed=4,
                                 user_zipf=1.3)
    np.testing.assert_array_equal(d.u_items, d2.u_items)


def test_stored_oracle_trace_matches_the_generator():
    """tests/golden/msd_subsample_trace.json was computed on the generator's 1% MSD-shaped
    subsample; a change to the generator that alters those inputs must come with a new
    trace (make_oracle_trace.py), else the GPU comparison would only skip."""
    import hashlib
    import json
    import os
    rec = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "msd_subsample_trace.json")))
    prob = synth.preset("msd_570k", seed=0, n_users=5700, nnz=340_000)
    h = hashlib.sha256()
    for a in (prob.data.u_indptr, prob.data.u_items, prob.W0, prob.H0):
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest()[:16] == rec["inputs_sha256_16"]
    assert (prob.data.n_users, prob.data.n_items, prob.data.nnz, prob.d, prob.b) == (
        rec["problem"]["n_users"], rec["problem"]["n_items"], rec["problem"]["nnz"],
        rec["problem"]["d"], rec["problem"]["b"])
