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
                   ials_foldin_close, ials_foldin_open, ials_foldin_poll, ials_foldin_submit,
                   ials_get_factors, ials_get_residuals, ials_last_error, ials_last_stats,
                   ials_objective, ials_partial_gramian, ials_recompute_residuals,
                   ials_set_factors, make_params)

__all__ = [
    "Model", "FoldinServer", "IalsError", "make_params", "ials_create", "ials_destroy", "ials_epoch",
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
                 stream=None, W0=None, H0=None, general=False, split_len=0):
        flags = ((_abi.FLAG_GRAPH if graph else 0) | (_abi.FLAG_FORCE_FP64 if force_fp64 else 0)
                 | (_abi.FLAG_GENERAL if general else 0))
        if init_std is None:
            init_std = 0.1 / np.sqrt(d)
        self.params = make_params(d, b, alpha0, lam, nu, init_std, seed, precision, flags, split_len)
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


class FoldinServer:
    """Fold-in of new users against frozen item factors (continuous batching).

    ``submit`` queues a request and returns a ticket; ``result`` waits for it.
    """

    def __init__(self, H, d, b, alpha0, lam, nu=0.0, sweeps=4, workspace_bytes=1 << 30,
                 stream=None):
        H = np.ascontiguousarray(H, dtype=np.float32)
        self.d = d
        self.params = make_params(d, b, alpha0, lam, nu)
        self.srv = ials_foldin_open(H, H.shape[0], self.params, workspace_bytes, sweeps, stream)

    def submit(self, items, y=None):
        return ials_foldin_submit(self.srv, items, y)

    def poll(self, ticket, timeout_us=0):
        """(status, w): status 0 with the embedding, or EAGAIN / ETIMEDOUT with None."""
        w = np.empty(self.d, np.float32)
        st = ials_foldin_poll(self.srv, ticket, w, timeout_us)
        return st, (w if st in (_abi.OK, _abi.ENOTPD) else None)

    def result(self, ticket, timeout_s=60.0):
        st, w = self.poll(ticket, int(timeout_s * 1e6))
        if st != _abi.OK:
            raise IalsError(st, ials_last_error())
        return w

    def result_info(self, ticket, timeout_s=60.0):
        """(embedding, info): info gives latency_us, batch, batch_size and cluster."""
        w = np.empty(self.d, np.float32)
        st, info = _abi.ials_foldin_poll_info(self.srv, ticket, w, int(timeout_s * 1e6))
        if st != _abi.OK:
            raise IalsError(st, ials_last_error())
        return w, info

    def close(self):
        if getattr(self, "srv", None) is not None:
            ials_foldin_close(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
