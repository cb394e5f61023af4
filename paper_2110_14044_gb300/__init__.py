"""GB300 (sm_103a) iALS++: subspace coordinate descent for implicit matrix factorisation.

The compute path is libials.so (hand-written CUDA kernels behind the C ABI in
include/ials.h); ``_abi`` is its ctypes binding and ``Model`` a small
convenience wrapper that only marshals arguments.  ``synth`` draws seeded
synthetic workloads.  Importing this package does not load the library; the
first call does, and fails loudly if it has not been built.
"""
from __future__ import annotations

import numpy as np

from . import _abi
from ._abi import (IalsError, ials_block_step, ials_create, ials_destroy, ials_epoch,
                   ials_get_factors, ials_get_residuals, ials_last_error, ials_last_stats,
                   ials_objective, ials_partial_gramian, ials_recompute_residuals,
                   ials_set_factors, make_params)

__all__ = [
    "Model", "IalsError", "make_params", "ials_create", "ials_destroy", "ials_epoch",
    "ials_objective", "ials_get_factors", "ials_set_factors", "ials_recompute_residuals",
    "ials_block_step", "ials_get_residuals", "ials_last_stats", "ials_partial_gramian",
    "ials_last_error",
]


class Model:
    """One training context on the current CUDA device.

    ``data`` is anything with n_users, n_items, u_indptr, u_items, i_indptr,
    i_users (e.g. ``synth.Interactions``).  Factors are returned as float32
    numpy arrays.
    """

    def __init__(self, data, d, b, alpha0, lam, nu=0.0, init_std=None, seed=0,
                 precision=_abi.PREC_FP32, graph=False, force_fp64=False, y=None, alpha=None,
                 stream=None, W0=None, H0=None):
        flags = (_abi.FLAG_GRAPH if graph else 0) | (_abi.FLAG_FORCE_FP64 if force_fp64 else 0)
        if init_std is None:
            init_std = 0.1 / np.sqrt(d)
        self.params = make_params(d, b, alpha0, lam, nu, init_std, seed, precision, flags)
        self.n_users, self.n_items, self.d, self.b = data.n_users, data.n_items, d, b
        self.nnz = int(data.u_indptr[-1])
        keep = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt)
        self._y, self._alpha = keep(y, np.float32), keep(alpha, np.float32)
        self.ctx = ials_create(self.params, data.n_users, data.n_items,
                               keep(data.u_indptr, np.int64), keep(data.u_items, np.int32),
                               keep(data.i_indptr, np.int64), keep(data.i_users, np.int32),
                               self._y, self._alpha, stream)
        if W0 is not None or H0 is not None:
            self.set_factors(W0, H0)

    def close(self):
        if self.ctx is not None:
            ials_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def epoch(self, n=1, objective=False):
        return ials_epoch(self.ctx, n, objective)

    def objective(self):
        return ials_objective(self.ctx)

    def factors(self):
        W = np.empty((self.n_users, self.d), np.float32)
        H = np.empty((self.n_items, self.d), np.float32)
        ials_get_factors(self.ctx, W, H)
        return W, H

    def set_factors(self, W=None, H=None):
        W = None if W is None else np.ascontiguousarray(W, dtype=np.float32)
        H = None if H is None else np.ascontiguousarray(H, dtype=np.float32)
        ials_set_factors(self.ctx, W, H)

    def residuals(self):
        e = np.empty(self.nnz, np.float32)
        ials_get_residuals(self.ctx, e)
        return e

    def recompute_residuals(self):
        ials_recompute_residuals(self.ctx)

    def block_step(self, side, block):
        return ials_block_step(self.ctx, side, block)

    def stats(self):
        return ials_last_stats(self.ctx)
