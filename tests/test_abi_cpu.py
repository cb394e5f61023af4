"""CPU checks of the C ABI: the library builds, loads and exports what include/ials.h declares.

No compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

from paper_2110_14044_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ials_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(_abi.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("ials_create", "ials_epoch", "ials_objective", "ials_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in sorted(declared_symbols()):
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    assert set(_abi.EXPORTS) == declared_symbols()


def test_params_struct_layout():
    # d, b, alpha0, lambda, nu, init_std, seed, precision, flags (C layout with padding)
    assert ctypes.sizeof(_abi.ials_params) == 4 + 4 + 8 * 4 + 8 + 4 + 4


def test_last_error_is_callable_without_gpu(lib):
    lib.ials_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ials_last_error(), bytes)


def test_create_fails_loudly_without_device_or_with_bad_args():
    import numpy as np
    p = _abi.make_params(16, 3, 0.1, 0.01)  # b = 3 is not allowed
    with pytest.raises(_abi.IalsError) as ei:
        _abi.ials_create(p, 2, 2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32))
    assert ei.value.status == _abi.EINVAL
