"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/amqft.h declares; argument checks work without a GPU (no kernels run)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(amqft_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1404_1810_gb300 import build

    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("amqft_plan", "amqft_exec_fwd", "amqft_exec_inv", "amqft_destroy", "amqft_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_argument_checks_need_no_gpu(lib):
    lib.amqft_plan.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                               ctypes.c_int]
    lib.amqft_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p(1)
    assert lib.amqft_plan(ctypes.byref(h), 10, 0, 1, 0) == -2
    assert h.value is None
    assert b"variant" in lib.amqft_last_error()
    assert lib.amqft_plan(ctypes.byref(h), 40, 4, 1, 0) == -1
    assert lib.amqft_plan(ctypes.byref(h), 10, 4, -1, 0) == -8
    assert lib.amqft_plan(ctypes.byref(h), 10, 4, 1, 9) == -3
    assert lib.amqft_plan(None, 10, 4, 1, 0) == -8
    lib.amqft_destroy.argtypes = [ctypes.c_void_p]
    assert lib.amqft_destroy(None) == 0
    lib.amqft_exec_fwd.argtypes = [ctypes.c_void_p] * 5
    assert lib.amqft_exec_fwd(None, None, None, None, None) == -8
    lib.amqft_plan_launches.argtypes = [ctypes.c_void_p]
    lib.amqft_plan_launches.restype = ctypes.c_int64
    assert lib.amqft_plan_launches(None) == -8
    lib.amqft_plan_set_constants.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert lib.amqft_plan_set_constants(None, 1) == -8
    lib.amqft_plan_get_constants.argtypes = [ctypes.c_void_p]
    assert lib.amqft_plan_get_constants(None) == -8


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1404_1810_gb300.amqft as b

    with pytest.raises(RuntimeError):
        _fresh_load(b, str(tmp_path / "missing.so"))


def _fresh_load(mod, path):
    saved = mod._lib
    mod._lib = None
    try:
        return mod.load(path)
    finally:
        mod._lib = saved
