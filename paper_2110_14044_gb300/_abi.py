"""ctypes binding of libials.so (argument marshalling only).

Every function here has the name of the C entry point it calls (see
include/ials.h), converts Python / numpy / torch arguments to pointers and
sizes, and turns a non-zero status into an ``IalsError``.  No arithmetic of
the method happens in Python.  If the shared library is missing the first call
raises ``RuntimeError``; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libials.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTPD, EAGAIN, ETIMEDOUT, ENOTFOUND = range(8)
PREC_FP32, PREC_BF16 = 0, 1
FLAG_GRAPH, FLAG_FORCE_FP64, FLAG_GENERAL = 1, 2, 4

_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTPD", 5: "EAGAIN",
           6: "ETIMEDOUT", 7: "ENOTFOUND"}

# Every symbol include/ials.h declares (checked by the CPU test suite).
EXPORTS = (
    "ials_create", "ials_destroy", "ials_epoch", "ials_objective", "ials_get_factors",
    "ials_set_factors", "ials_recompute_residuals", "ials_block_step", "ials_get_residuals",
    "ials_last_stats", "ials_partial_gramian", "ials_last_error", "ials_profile_epochs",
    "ials_work_model", "ials_partial_gramian_noalloc", "ials_partial_gramian_bf16",
    "ials_foldin_open", "ials_foldin_submit", "ials_foldin_poll", "ials_foldin_close",
    "ials_foldin_poll_timed", "ials_foldin_poll_info",
)

KERNEL_KINDS = ("residual", "gram", "rowterm", "sparse", "split_solve", "split_resid", "retry",
                "objective")


class IalsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class ials_foldin_info(C.Structure):
    _fields_ = [("latency_us", C.c_double), ("batch", C.c_uint64), ("batch_size", C.c_int32),
                ("cluster", C.c_int32)]


class ials_params(C.Structure):
    _fields_ = [("d", C.c_int32), ("b", C.c_int32), ("alpha0", C.c_double),
                ("lambda_", C.c_double), ("nu", C.c_double), ("init_std", C.c_double),
                ("seed", C.c_uint64), ("precision", C.c_int32), ("flags", C.c_int32),
                ("split_len", C.c_int32), ("reserved", C.c_int32)]


_lib = None


def lib():
    """Load libials.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2110_14044_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        st = C.c_int
        P = C.POINTER(ials_params)
        sig = {
            "ials_create": ([P, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, C.POINTER(vp)], st),
            "ials_destroy": ([vp], st),
            "ials_epoch": ([vp, i32, C.POINTER(C.c_double)], st),
            "ials_objective": ([vp, C.POINTER(C.c_double)], st),
            "ials_get_factors": ([vp, vp, vp], st),
            "ials_set_factors": ([vp, vp, vp], st),
            "ials_recompute_residuals": ([vp], st),
            "ials_block_step": ([vp, i32, i32], st),
            "ials_get_residuals": ([vp, vp], st),
            "ials_last_stats": ([vp, C.POINTER(i64), C.POINTER(i64)], st),
            "ials_partial_gramian": ([vp, i64, i32, i32, i32, vp, vp], st),
            "ials_last_error": ([], C.c_char_p),
            "ials_profile_epochs": ([vp, i32, vp, vp, i32, C.POINTER(C.c_double)], st),
            "ials_work_model": ([vp, vp, vp, i32], st),
            "ials_partial_gramian_noalloc": ([vp, i64, i32, i32, i32, vp, vp], st),
            "ials_partial_gramian_bf16": ([vp, i64, i32, i32, i32, vp, vp], st),
            "ials_foldin_open": ([vp, i32, P, C.c_size_t, i32, vp, C.POINTER(vp)], st),
            "ials_foldin_submit": ([vp, vp, vp, i32, C.POINTER(C.c_uint64)], st),
            "ials_foldin_poll": ([vp, C.c_uint64, vp, i32], st),
            "ials_foldin_close": ([vp], st),
            "ials_foldin_poll_timed": ([vp, C.c_uint64, vp, i32, C.POINTER(C.c_double)], st),
            "ials_foldin_poll_info": ([vp, C.c_uint64, vp, i32, C.POINTER(ials_foldin_info)], st),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise IalsError(status, lib().ials_last_error().decode())
    return status


def _ptr(a):
    """Pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def make_params(d, b, alpha0, lam, nu=0.0, init_std=0.01, seed=0, precision=PREC_FP32, flags=0,
                split_len=0):
    return ials_params(int(d), int(b), float(alpha0), float(lam), float(nu), float(init_std),
                       int(seed), int(precision), int(flags), int(split_len), 0)


def ials_create(params, n_users, n_items, u_indptr, u_items, i_indptr=None, i_users=None,
                y=None, alpha=None, stream=None):
    """Create a context; CSR arrays may be numpy (host) or torch (host or device)."""
    nnz = int(u_indptr[-1])
    out = C.c_void_p()
    _check(lib().ials_create(C.byref(params), int(n_users), int(n_items), nnz, _ptr(u_indptr),
                             _ptr(u_items), _ptr(i_indptr), _ptr(i_users), _ptr(y), _ptr(alpha),
                             _stream(stream), C.byref(out)))
    return out


def ials_destroy(ctx):
    return _check(lib().ials_destroy(ctx))


def ials_epoch(ctx, n_epochs=1, want_objective=False):
    obj = C.c_double(0.0)
    status = lib().ials_epoch(ctx, int(n_epochs), C.byref(obj) if want_objective else None)
    if status not in (OK, ENOTPD):
        _check(status)
    return (obj.value if want_objective else None), status


def ials_objective(ctx):
    obj = C.c_double(0.0)
    _check(lib().ials_objective(ctx, C.byref(obj)))
    return obj.value


def ials_get_factors(ctx, W=None, H=None):
    return _check(lib().ials_get_factors(ctx, _ptr(W), _ptr(H)))


def ials_set_factors(ctx, W=None, H=None):
    return _check(lib().ials_set_factors(ctx, _ptr(W), _ptr(H)))


def ials_recompute_residuals(ctx):
    return _check(lib().ials_recompute_residuals(ctx))


def ials_block_step(ctx, side, block):
    status = lib().ials_block_step(ctx, int(side), int(block))
    if status not in (OK, ENOTPD):
        _check(status)
    return status


def ials_get_residuals(ctx, e):
    return _check(lib().ials_get_residuals(ctx, _ptr(e)))


def ials_last_stats(ctx):
    a, b = C.c_int64(0), C.c_int64(0)
    _check(lib().ials_last_stats(ctx, C.byref(a), C.byref(b)))
    return a.value, b.value


def ials_partial_gramian(X, n, d, p0, bs, G, stream=None):
    return _check(lib().ials_partial_gramian(_ptr(X), int(n), int(d), int(p0), int(bs), _ptr(G),
                                             _stream(stream)))


def ials_last_error():
    return lib().ials_last_error().decode()


def ials_profile_epochs(ctx, n_epochs=1):
    """Per-kernel-kind device time (ms) and launch counts over n_epochs eager epochs."""
    n = len(KERNEL_KINDS)
    ms = np.zeros(n, np.float64)
    cnt = np.zeros(n, np.int64)
    total = C.c_double(0.0)
    status = lib().ials_profile_epochs(ctx, int(n_epochs), ms.ctypes.data, cnt.ctypes.data, n,
                                       C.byref(total))
    if status not in (OK, ENOTPD):
        _check(status)
    return ({k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_KINDS)},
            total.value, status)


def ials_work_model(ctx):
    """Algorithmic bytes and FLOPs of one epoch per kernel kind."""
    n = len(KERNEL_KINDS)
    b = np.zeros(n, np.float64)
    f = np.zeros(n, np.float64)
    _check(lib().ials_work_model(ctx, b.ctypes.data, f.ctypes.data, n))
    return {k: (float(b[i]), float(f[i])) for i, k in enumerate(KERNEL_KINDS)}


def ials_partial_gramian_noalloc(X, n, d, p0, bs, G, stream=None):
    """Partial Gramian that allocates nothing (fixed 8 MiB device scratch; enqueue only)."""
    return _check(lib().ials_partial_gramian_noalloc(_ptr(X), int(n), int(d), int(p0), int(bs),
                                                     _ptr(G), _stream(stream)))


def ials_partial_gramian_bf16(X, n, d, p0, bs, G, stream=None):
    """Partial Gramian on tcgen05 tensor cores (BF16 hi/lo compensated, FP32 accumulate)."""
    return _check(lib().ials_partial_gramian_bf16(_ptr(X), int(n), int(d), int(p0), int(bs), _ptr(G),
                                                  _stream(stream)))


def ials_foldin_open(H, n_items, params, workspace_bytes, sweeps, stream=None):
    out = C.c_void_p()
    _check(lib().ials_foldin_open(_ptr(H), int(n_items), C.byref(params), int(workspace_bytes),
                                  int(sweeps), _stream(stream), C.byref(out)))
    return out


def ials_foldin_submit(srv, items, y=None):
    """Queue one request (numpy int32 items, optional float32 y); returns a ticket."""
    items = np.ascontiguousarray(items, dtype=np.int32)
    y = None if y is None else np.ascontiguousarray(y, dtype=np.float32)
    t = C.c_uint64(0)
    _check(lib().ials_foldin_submit(srv, _ptr(items), _ptr(y), int(items.size), C.byref(t)))
    return t.value


def ials_foldin_poll(srv, ticket, w_out, timeout_us=0):
    """Status of one request; on OK w_out (float32 numpy, d) holds the embedding."""
    status = lib().ials_foldin_poll(srv, C.c_uint64(ticket), _ptr(w_out), int(timeout_us))
    if status not in (OK, EAGAIN, ETIMEDOUT, ENOTPD):
        _check(status)
    return status


def ials_foldin_close(srv):
    return _check(lib().ials_foldin_close(srv))


def ials_foldin_poll_timed(srv, ticket, w_out, timeout_us=0):
    """(status, latency in microseconds from submit to result, or None)."""
    lat = C.c_double(-1.0)
    status = lib().ials_foldin_poll_timed(srv, C.c_uint64(ticket), _ptr(w_out), int(timeout_us),
                                          C.byref(lat))
    if status not in (OK, EAGAIN, ETIMEDOUT, ENOTPD):
        _check(status)
    return status, (lat.value if status in (OK, ENOTPD) else None)


def ials_foldin_poll_info(srv, ticket, w_out, timeout_us=0):
    """(status, info dict or None): how a finished request was served (latency, batch,
    batch size, whether it ran on a CTA cluster)."""
    info = ials_foldin_info()
    status = lib().ials_foldin_poll_info(srv, C.c_uint64(ticket), _ptr(w_out), int(timeout_us),
                                         C.byref(info))
    if status not in (OK, EAGAIN, ETIMEDOUT, ENOTPD):
        _check(status)
    if status not in (OK, ENOTPD):
        return status, None
    return status, {"latency_us": info.latency_us, "batch": info.batch, "batch_size": info.batch_size,
                    "cluster": bool(info.cluster)}
