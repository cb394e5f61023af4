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
    assert ctypes.sizeof(_abi.ials_params) == 4 + 4 + 8 * 4 + 8 + 4 + 4 + 4 + 4


def test_last_error_is_callable_without_gpu(lib):
    lib.ials_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.ials_last_error(), bytes)


def test_create_fails_loudly_without_device_or_with_bad_args():
    import numpy as np
    p = _abi.make_params(16, 3, 0.1, 0.01)  # b = 3 is not allowed
    with pytest.raises(_abi.IalsError) as ei:
        _abi.ials_create(p, 2, 2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32))
    assert ei.value.status == _abi.EINVAL


def _create(p, n_users, n_items, uptr, uidx, **kw):
    import numpy as np
    return _abi.ials_create(p, n_users, n_items, np.asarray(uptr, np.int64), np.asarray(uidx, np.int32), **kw)


@pytest.mark.parametrize("case", ["d", "b_not_dividing", "bf16_b", "alpha0",
                                  "indptr_end", "indptr_order", "item_range", "repeat",
                                  "transpose_len", "transpose_pairs", "alpha_zero", "y_nan",
                                  "split_len_small", "split_len_large", "reserved", "big_b_not_d",
                                  "big_too_large", "big_bf16", "big_general"])
def test_create_validates_on_the_host(case):
    """Every argument check runs on the host before any device work, so a bad
    input is rejected with IALS_EINVAL and a message, GPU or not."""
    import numpy as np
    fp32, bf16 = _abi.PREC_FP32, _abi.PREC_BF16
    good = dict(p=_abi.make_params(16, 8, 0.1, 0.01), n_users=3, n_items=4,
                uptr=[0, 2, 3, 5], uidx=[0, 1, 3, 1, 2])
    kw = {}
    if case == "d":
        good["p"] = _abi.make_params(18, 2, 0.1, 0.01)
    elif case == "b_not_dividing":
        good["p"] = _abi.make_params(16, 32, 0.1, 0.01)
    elif case == "bf16_b":
        good["p"] = _abi.make_params(16, 8, 0.1, 0.01, precision=bf16)
    elif case == "alpha0":
        good["p"] = _abi.make_params(16, 8, -0.1, 0.01)
    elif case == "indptr_end":
        good["uptr"] = [1, 2, 3, 5]  # must start at 0
    elif case == "indptr_order":
        good["uptr"] = [0, 3, 2, 5]
    elif case == "item_range":
        good["uidx"] = [0, 1, 4, 1, 2]
    elif case == "repeat":
        good["uidx"] = [1, 1, 3, 1, 2]
    elif case == "transpose_len":
        kw["i_indptr"] = np.array([0, 1, 2, 4, 5], np.int64)
        kw["i_users"] = np.array([0, 0, 1, 2, 0], np.int32)
    elif case == "transpose_pairs":
        # item-major view of the same lengths but a wrong user for item 3
        kw["i_indptr"] = np.array([0, 1, 3, 4, 5], np.int64)
        kw["i_users"] = np.array([0, 0, 1, 2, 1], np.int32)
    elif case == "alpha_zero":
        kw["alpha"] = np.array([1, 1, 0, 1, 1], np.float32)
    elif case == "y_nan":
        kw["y"] = np.array([1, np.nan, 1, 1, 1], np.float32)
    elif case == "split_len_small":
        good["p"] = _abi.make_params(16, 8, 0.1, 0.01, split_len=31)
    elif case == "split_len_large":
        good["p"] = _abi.make_params(16, 8, 0.1, 0.01, split_len=(1 << 24) + 1)
    elif case == "reserved":
        good["p"] = _abi.make_params(16, 8, 0.1, 0.01)
        good["p"].reserved = 1
    elif case == "big_b_not_d":      # above 256 only b = d (iALS) exists
        good["p"] = _abi.make_params(1024, 512, 0.1, 0.01)
    elif case == "big_too_large":
        good["p"] = _abi.make_params(1088, 1088, 0.1, 0.01)
    elif case == "big_bf16":
        good["p"] = _abi.make_params(512, 512, 0.1, 0.01, precision=_abi.PREC_BF16)
    elif case == "big_general":      # the general block step stops at b = 256
        good["p"] = _abi.make_params(512, 512, 0.1, 0.01, flags=_abi.FLAG_GENERAL)
    with pytest.raises(_abi.IalsError) as ei:
        _create(**good, **kw)
    assert ei.value.status == _abi.EINVAL, (case, str(ei.value))


def test_create_accepts_valid_input_up_to_the_device_check():
    """The same (valid) arguments pass every host check; without an sm_103a
    device the call then fails with IALS_ECUDA, never silently on the CPU."""
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    for p in (_abi.make_params(16, 8, 0.1, 0.01),
              _abi.make_params(32, 16, 0.1, 0.01, precision=_abi.PREC_BF16),  # weights in BF16 too
              _abi.make_params(320, 320, 0.1, 0.01)):                         # iALS above b = 256
        with pytest.raises(_abi.IalsError) as ei:
            _create(p, 3, 4, [0, 2, 3, 5], [0, 1, 3, 1, 2],
                    i_indptr=np.array([0, 1, 3, 4, 5], np.int64), i_users=np.array([0, 2, 0, 2, 1], np.int32),
                    y=np.ones(5, np.float32), alpha=np.full(5, 2.0, np.float32))
        assert ei.value.status == _abi.ECUDA, str(ei.value)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every call raises; nothing falls back to the CPU."""
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "libials.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _abi.ials_last_error()
    with pytest.raises(RuntimeError, match="missing"):
        _abi.ials_create(_abi.make_params(16, 8, 0.1, 0.01), 1, 1, [0, 0], [])
