"""ctypes front end of the FP64 iALS++ oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it.

The C source is ``ials_oracle.c`` beside this file; :func:`build` compiles it
with gcc into ``libials_oracle.so`` (in-tree, git-ignored).  Every function
here converts its arguments to contiguous float64 / int64 / int32 arrays and
calls the C routine of the same name; no arithmetic happens in Python.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ials_oracle.c")
_LIB = os.path.join(_HERE, "libials_oracle.so")
_lib = None

OK, EINVAL, ENOMEM, ENOTPD = 0, 1, 2, 4


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n_users", C.c_int32), ("n_items", C.c_int32), ("nnz", C.c_int64),
        ("u_ptr", C.c_void_p), ("u_idx", C.c_void_p),
        ("i_ptr", C.c_void_p), ("i_idx", C.c_void_p), ("i_pos", C.c_void_p),
        ("y", C.c_void_p), ("alpha", C.c_void_p),
        ("d", C.c_int32), ("b", C.c_int32),
        ("alpha0", C.c_double), ("lam", C.c_double), ("nu", C.c_double),
        ("n_threads", C.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER(_Problem)
        vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        lib.oracle_build_pos.argtypes = [i32, i32, vp, vp, vp, vp, vp]
        lib.oracle_build_pos.restype = C.c_int
        lib.oracle_predict.argtypes = [P, vp, vp, vp]
        lib.oracle_predict.restype = None
        lib.oracle_objective.argtypes = [P, vp, vp]
        lib.oracle_objective.restype = f64
        lib.oracle_halfstep.argtypes = [P, C.c_int, C.c_int, vp, vp, vp]
        lib.oracle_halfstep.restype = C.c_int
        lib.oracle_row_step.argtypes = [P, C.c_int, C.c_int, vp, vp, vp, i64, vp]
        lib.oracle_row_step.restype = C.c_int
        lib.oracle_rows_step.argtypes = [P, C.c_int, C.c_int, vp, vp, vp, vp, i64, vp, vp]
        lib.oracle_rows_step.restype = C.c_int
        lib.oracle_ialspp.argtypes = [P, C.c_int, vp, vp, vp, vp]
        lib.oracle_ialspp.restype = C.c_int
        lib.oracle_ials.argtypes = [P, C.c_int, vp, vp]
        lib.oracle_ials.restype = C.c_int
        lib.oracle_icd.argtypes = [P, C.c_int, vp, vp, vp]
        lib.oracle_icd.restype = C.c_int
        lib.oracle_foldin.argtypes = [vp, i32, i32, i32, f64, f64, f64, i32, vp, vp, vp, i32, vp]
        lib.oracle_foldin.restype = C.c_int
        lib.oracle_foldin_g.argtypes = [vp, vp, i32, i32, i32, f64, f64, f64, i32, vp, vp, vp, i32, vp]
        lib.oracle_foldin_g.restype = C.c_int
        lib.oracle_gramian.argtypes = [vp, i32, i32, vp]
        lib.oracle_gramian.restype = None
        _lib = lib
    return _lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Problem:
    """An interaction set plus hyperparameters, in the oracle's layout."""

    def __init__(self, n_users, n_items, u_indptr, u_items, i_indptr, i_users, d, b,
                 alpha0, lam, nu=0.0, y=None, alpha=None, n_threads=None):
        lib = _load()
        self.n_users, self.n_items, self.d, self.b = int(n_users), int(n_items), int(d), int(b)
        self.u_ptr = _c(u_indptr, np.int64)
        self.u_idx = _c(u_items, np.int32)
        self.i_ptr = _c(i_indptr, np.int64)
        self.i_idx = _c(i_users, np.int32)
        self.nnz = int(self.u_ptr[-1])
        self.y = None if y is None else _c(y, np.float64)
        self.alpha = None if alpha is None else _c(alpha, np.float64)
        self.i_pos = np.empty(self.nnz, dtype=np.int64)
        st = lib.oracle_build_pos(self.n_users, self.n_items, _ptr(self.u_ptr), _ptr(self.u_idx),
                                  _ptr(self.i_ptr), _ptr(self.i_idx), _ptr(self.i_pos))
        if st != OK:
            raise ValueError("item-major CSR is not the transpose of the user-major CSR")
        self.alpha0, self.lam, self.nu = float(alpha0), float(lam), float(nu)
        self.n_threads = int(n_threads or os.cpu_count() or 1)
        self._s = _Problem(self.n_users, self.n_items, self.nnz, _ptr(self.u_ptr),
                           _ptr(self.u_idx), _ptr(self.i_ptr), _ptr(self.i_idx),
                           _ptr(self.i_pos), _ptr(self.y), _ptr(self.alpha), self.d, self.b,
                           self.alpha0, self.lam, self.nu, self.n_threads)

    @classmethod
    def from_data(cls, data, d, b, alpha0, lam, nu=0.0, **kw):
        return cls(data.n_users, data.n_items, data.u_indptr, data.u_items, data.i_indptr,
                   data.i_users, d, b, alpha0, lam, nu, **kw)

    def with_block(self, b):
        """The same problem with another block size."""
        return Problem(self.n_users, self.n_items, self.u_ptr, self.u_idx, self.i_ptr,
                       self.i_idx, self.d, b, self.alpha0, self.lam, self.nu, self.y,
                       self.alpha, self.n_threads)

    @property
    def ref(self):
        return C.byref(self._s)

    def factors(self, W, H):
        W = np.array(W, dtype=np.float64, order="C", copy=True)
        H = np.array(H, dtype=np.float64, order="C", copy=True)
        assert W.shape == (self.n_users, self.d) and H.shape == (self.n_items, self.d)
        return W, H


def predict(P: Problem, W, H):
    """Eq. 1 over S, user-major order."""
    W, H = P.factors(W, H)
    out = np.empty(P.nnz)
    _load().oracle_predict(P.ref, _ptr(W), _ptr(H), _ptr(out))
    return out


def objective(P: Problem, W, H) -> float:
    """Eq. 2 (with per-row lambda), FP64."""
    W, H = P.factors(W, H)
    return float(_load().oracle_objective(P.ref, _ptr(W), _ptr(H)))


def halfstep(P: Problem, side: int, block: int, W, H, yhat):
    """One block-side step of Algorithm 3, in place on float64 W, H, yhat."""
    for a in (W, H, yhat):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    return _load().oracle_halfstep(P.ref, side, block, _ptr(W), _ptr(H), _ptr(yhat))


def row_step(P: Problem, side: int, block: int, W, H, yhat, r: int):
    """New w_{r,pi} (or h_{r,pi}) that a half-step would produce for row r."""
    for a in (W, H, yhat):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    bs = min(P.b, P.d - block * P.b)
    out = np.empty(bs)
    st = _load().oracle_row_step(P.ref, side, block, _ptr(W), _ptr(H), _ptr(yhat), int(r),
                                 _ptr(out))
    return st, out


def rows_step(P: Problem, side: int, block: int, W, H, yhat, rows):
    """row_step for many rows at once; returns (status per row, n_rows x bs values)."""
    W = _c(W, np.float64)
    H = _c(H, np.float64)
    yhat = _c(yhat, np.float64)
    rows = _c(rows, np.int64)
    bs = min(P.b, P.d - block * P.b)
    out = np.empty((rows.size, bs))
    st = np.empty(rows.size, dtype=np.int32)
    rc = _load().oracle_rows_step(P.ref, side, block, _ptr(W), _ptr(H), _ptr(yhat), _ptr(rows),
                                  rows.size, _ptr(out), _ptr(st))
    if rc != OK:
        raise ValueError("oracle_rows_step failed: %d" % rc)
    return st, out


def ialspp(P: Problem, epochs: int, W, H, trace: bool = False):
    """T epochs of Algorithm 3; returns (W, H, yhat, trace or None, status)."""
    W, H = P.factors(W, H)
    yhat = np.empty(P.nnz)
    nb = -(-P.d // P.b)
    tr = np.empty(max(1, epochs * 2 * nb)) if trace else None
    st = _load().oracle_ialspp(P.ref, epochs, _ptr(W), _ptr(H), _ptr(yhat), _ptr(tr))
    return W, H, yhat, (tr[: epochs * 2 * nb] if trace else None), st


def ials(P: Problem, epochs: int, W, H):
    """T epochs of Algorithm 1 (closed form, Eq. 3); returns (W, H, status)."""
    W, H = P.factors(W, H)
    st = _load().oracle_ials(P.ref, epochs, _ptr(W), _ptr(H))
    return W, H, st


def icd(P: Problem, epochs: int, W, H):
    """T epochs of Algorithm 2 (iCD); returns (W, H, yhat, status)."""
    W, H = P.factors(W, H)
    yhat = np.empty(P.nnz)
    st = _load().oracle_icd(P.ref, epochs, _ptr(W), _ptr(H), _ptr(yhat))
    return W, H, yhat, st


def gramian(H):
    """G^I = H^T H (Eq. 4) in FP64, for repeated fold-ins against the same H."""
    H = _c(H, np.float64)
    G = np.empty((H.shape[1], H.shape[1]))
    _load().oracle_gramian(_ptr(H), H.shape[0], H.shape[1], _ptr(G))
    return G


def foldin(H, d, b, alpha0, lam, nu, sweeps, items, y=None, alpha=None, G=None):
    """Embedding of a new user against frozen H; returns (w, status).  With G (from
    gramian(H)) the Gramian is not formed again."""
    H = _c(H, np.float64)
    assert H.ndim == 2 and H.shape[1] == d
    items = _c(items, np.int32)
    y = None if y is None else _c(y, np.float64)
    alpha = None if alpha is None else _c(alpha, np.float64)
    w = np.empty(d)
    if G is None:
        st = _load().oracle_foldin(_ptr(H), H.shape[0], d, b, alpha0, lam, nu, sweeps, _ptr(items),
                                   _ptr(y), _ptr(alpha), items.size, _ptr(w))
    else:
        G = _c(G, np.float64)
        assert G.shape == (d, d)
        st = _load().oracle_foldin_g(_ptr(H), _ptr(G), H.shape[0], d, b, alpha0, lam, nu, sweeps,
                                     _ptr(items), _ptr(y), _ptr(alpha), items.size, _ptr(w))
    return w, st
