"""Seeded synthetic interaction data shaped like the iALS++ benchmarks.

This module only draws inputs: interaction sets S (as CSR index arrays) and
initial factor matrices.  It holds none of the solver's arithmetic, so both the
FP64 oracle and the CUDA path can be fed from it.

The paper's own workloads (Table 2: ML20M, 136,677 x 20,108 with 10.0M
interactions, and MSD, 571,355 x 41,140 with 33.6M) are not available here;
the presets below stand in for them with the same shape:

* item popularity follows a Zipf law over a random permutation of item ids,
* per-user history lengths are lognormal (or Zipf over the users), clipped,
  then rescaled so that the total hits |S| exactly,
* within a user row items are drawn without replacement (successive sampling
  from the Zipf weights), so every (u, i) pair occurs at most once,
* y = alpha = 1 (binary implicit feedback, Section 2: "in most cases
  alpha = y = 1").

Random numbers come from numpy's Philox counter-based generator.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Interactions",
    "Problem",
    "make_interactions",
    "transpose_csr",
    "init_factors",
    "preset",
    "PRESETS",
]


@dataclasses.dataclass
class Interactions:
    """User-major and item-major CSR views of one interaction set S."""

    n_users: int
    n_items: int
    u_indptr: np.ndarray  # int64, n_users + 1
    u_items: np.ndarray   # int32, nnz, sorted within each row
    i_indptr: np.ndarray  # int64, n_items + 1
    i_users: np.ndarray   # int32, nnz, sorted within each row

    @property
    def nnz(self) -> int:
        return int(self.u_indptr[-1])


@dataclasses.dataclass
class Problem:
    """One seeded workload: data, hyperparameters and initial factors."""

    name: str
    data: Interactions
    d: int
    b: int
    alpha0: float
    lam: float
    nu: float
    epochs: int
    W0: np.ndarray  # float32, n_users x d
    H0: np.ndarray  # float32, n_items x d


def _rng(seed: int, stream: int) -> np.random.Generator:
    # Philox with a per-purpose stream key keeps draws independent of each other.
    return np.random.Generator(np.random.Philox(key=[seed, stream]))


def _lengths(rng, n_users, nnz, mu, sigma, lo, hi, user_zipf=None):
    """Lengths clipped to [lo, hi], rescaled to sum to nnz exactly: lognormal(mu,
    sigma) draws, or (user_zipf = s) Zipf(s) activity over a random permutation of
    the users (rank r gets weight r^-s)."""
    if user_zipf is None:
        raw = rng.lognormal(mean=mu, sigma=sigma, size=n_users)
    else:
        raw = np.empty(n_users)
        raw[rng.permutation(n_users)] = np.arange(1, n_users + 1, dtype=np.float64) ** (-user_zipf)
    if not (lo * n_users <= nnz <= hi * n_users):
        raise ValueError("nnz is not reachable with the given clip range")

    def total(scale):
        return int(np.clip(np.rint(raw * scale), lo, hi).sum())

    a, b = 0.0, 1.0
    while total(b) < nnz:
        b *= 2.0
    for _ in range(200):
        m = 0.5 * (a + b)
        if total(m) < nnz:
            a = m
        else:
            b = m
    lens = np.clip(np.rint(raw * b), lo, hi).astype(np.int64)
    # Correct the remainder one unit at a time, starting from the largest rows.
    diff = nnz - int(lens.sum())
    order = np.argsort(-lens, kind="stable")
    k = 0
    while diff != 0:
        j = order[k % n_users]
        if diff > 0 and lens[j] < hi:
            lens[j] += 1
            diff -= 1
        elif diff < 0 and lens[j] > lo:
            lens[j] -= 1
            diff += 1
        k += 1
    return lens


def _zipf_weights(rng, n_items, s):
    ranks = np.arange(1, n_items + 1, dtype=np.float64)
    w = ranks ** (-s)
    w /= w.sum()
    perm = rng.permutation(n_items)  # popularity rank r -> item id perm[r]
    p = np.empty(n_items)
    p[perm] = w
    return p


def _sample_rows(rng, lens, p, batch_users=65536):
    """For each user draw lens[u] distinct items, successive sampling from p.

    Returns (owner, item) pairs, grouped by nothing in particular.
    """
    n_users = lens.shape[0]
    n_items = p.shape[0]
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    out_u, out_i = [], []
    dense_cut = n_items // 3  # heavy rows: exponential-key sampling instead
    heavy = np.nonzero(lens > dense_cut)[0]
    light = np.nonzero(lens <= dense_cut)[0]
    logp = np.log(np.maximum(p, 1e-300))
    for u in heavy:
        # Successive sampling without replacement == ordering by E_i / p_i.
        keys = np.log(rng.exponential(size=n_items)) - logp
        sel = np.argpartition(keys, lens[u] - 1)[: lens[u]]
        out_u.append(np.full(sel.size, u, dtype=np.int64))
        out_i.append(sel.astype(np.int64))
    pending = light
    factor = 1.3
    while pending.size:
        nxt = []
        for start in range(0, pending.size, batch_users):
            us = pending[start:start + batch_users]
            need = lens[us]
            draws = np.ceil(need * factor).astype(np.int64) + 4
            tot = int(draws.sum())
            items = np.searchsorted(cdf, rng.random(tot), side="right")
            items = np.minimum(items, n_items - 1)
            owner = np.repeat(np.arange(us.size), draws)
            key = owner.astype(np.int64) * n_items + items
            _, first = np.unique(key, return_index=True)
            first.sort()  # distinct (user, item) pairs in draw order
            own = owner[first]
            cnt = np.bincount(own, minlength=us.size)
            starts = np.concatenate([[0], np.cumsum(cnt)])
            rank = np.arange(first.size) - starts[own]
            ok = cnt >= need
            keep = (rank < need[own]) & ok[own]
            out_u.append(us[own[keep]].astype(np.int64))
            out_i.append(items[first[keep]].astype(np.int64))
            nxt.append(us[~ok])
        pending = np.concatenate(nxt) if nxt else np.array([], dtype=np.int64)
        factor *= 2.0
    return np.concatenate(out_u), np.concatenate(out_i)


def transpose_csr(n_rows, n_cols, indptr, indices):
    """Column-major view of a CSR pattern (rows of the result sorted ascending)."""
    nnz = int(indptr[-1])
    row_of = np.repeat(np.arange(n_rows, dtype=np.int32), np.diff(indptr))
    order = np.argsort(indices, kind="stable")
    t_indices = row_of[order].astype(np.int32)
    counts = np.bincount(indices, minlength=n_cols)
    t_indptr = np.zeros(n_cols + 1, dtype=np.int64)
    np.cumsum(counts, out=t_indptr[1:])
    assert t_indptr[-1] == nnz
    return t_indptr, t_indices


def make_interactions(n_users, n_items, nnz, zipf_s, ln_mu, ln_sigma,
                      len_min, len_max, seed, user_zipf=None) -> Interactions:
    """Draw a binary interaction set with Zipf items and lognormal (or, with
    user_zipf, Zipf) user lengths; a row holds at most n_items distinct items."""
    len_max = min(len_max, n_items)
    lens = _lengths(_rng(seed, 1), n_users, nnz, ln_mu, ln_sigma, len_min, len_max, user_zipf)
    rng = _rng(seed, 2)
    p = _zipf_weights(rng, n_items, zipf_s)
    owner, items = _sample_rows(rng, lens, p)
    order = np.lexsort((items, owner))
    u_indptr = np.zeros(n_users + 1, dtype=np.int64)
    np.cumsum(lens, out=u_indptr[1:])
    u_items = items[order].astype(np.int32)
    assert u_items.size == nnz
    i_indptr, i_users = transpose_csr(n_users, n_items, u_indptr, u_items)
    return Interactions(n_users, n_items, u_indptr, u_items, i_indptr, i_users)


def from_pairs(n_users, n_items, users, items) -> Interactions:
    """Build both CSR views from explicit (u, i) pairs (duplicates rejected)."""
    users = np.asarray(users, dtype=np.int64)
    items = np.asarray(items, dtype=np.int64)
    key = users * n_items + items
    if np.unique(key).size != key.size:
        raise ValueError("duplicate (u, i) pair")
    order = np.lexsort((items, users))
    users, items = users[order], items[order]
    u_indptr = np.zeros(n_users + 1, dtype=np.int64)
    np.cumsum(np.bincount(users, minlength=n_users), out=u_indptr[1:])
    u_items = items.astype(np.int32)
    i_indptr, i_users = transpose_csr(n_users, n_items, u_indptr, u_items)
    return Interactions(n_users, n_items, u_indptr, u_items, i_indptr, i_users)


def init_factors(n_users, n_items, d, std, seed, std_items=None):
    """W then H, each N(0, std^2) in float32 (std given as a standard deviation)."""
    rng = _rng(seed, 3)
    W = rng.normal(0.0, std, size=(n_users, d)).astype(np.float32)
    H = rng.normal(0.0, std if std_items is None else std_items,
                   size=(n_items, d)).astype(np.float32)
    return W, H


# Workload presets.  Sizes and distributions follow the benchmark configurations;
# hyperparameters for the MSD-shaped case come from Table 2 (alpha0 = 0.02,
# lambda = 0.002).
PRESETS = {
    # Parity workload: full problem in the oracle within seconds.
    "parity_2k": dict(n_users=2000, n_items=1000, nnz=50_000, zipf_s=1.0, ln_mu=2.5,
                      ln_sigma=1.0, len_min=1, len_max=500, d=16, b=8, alpha0=0.1,
                      lam=1e-3, nu=0.0, epochs=5),
    # ML20M-shaped mid-scale workload.
    "ml20m_136k": dict(n_users=136_000, n_items=20_000, nnz=10_000_000, zipf_s=1.05,
                       ln_mu=3.7, ln_sigma=1.1, len_min=5, len_max=8000, d=128, b=32,
                       alpha0=0.1, lam=1e-3, nu=1.0, epochs=16),
    # ML20M shape with extremely skewed user activity: Zipf(1.3) users; "at most
    # 200,000 items per row" cannot hold with 20,000 items, so rows are capped at
    # the whole catalogue.  Swept over d with the block size autotuned.
    "skewed_136k": dict(n_users=136_000, n_items=20_000, nnz=10_000_000, zipf_s=1.05,
                        ln_mu=0.0, ln_sigma=0.0, user_zipf=1.3, len_min=5, len_max=200_000,
                        d=128, b=32, alpha0=0.1, lam=1e-3, nu=1.0, epochs=16),
    # MSD-shaped large workload.
    "msd_570k": dict(n_users=570_000, n_items=41_000, nnz=34_000_000, zipf_s=0.9,
                     ln_mu=3.5, ln_sigma=1.2, len_min=1, len_max=50_000, d=1024, b=128,
                     alpha0=0.02, lam=2e-3, nu=1.0, epochs=8),
}


def preset(name: str, seed: int = 0, **overrides) -> Problem:
    """Materialise a preset (optionally with overridden fields) for one seed."""
    cfg = dict(PRESETS[name])
    cfg.update(overrides)
    data = make_interactions(cfg["n_users"], cfg["n_items"], cfg["nnz"], cfg["zipf_s"],
                             cfg["ln_mu"], cfg["ln_sigma"], cfg["len_min"], cfg["len_max"],
                             seed, cfg.get("user_zipf"))
    d = cfg["d"]
    std = 0.1 / math.sqrt(d)
    W0, H0 = init_factors(data.n_users, data.n_items, d, std, seed)
    return Problem(name, data, d, cfg["b"], cfg["alpha0"], cfg["lam"], cfg["nu"],
                   cfg["epochs"], W0, H0)
