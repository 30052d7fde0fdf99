"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, exports every function include/pbe.h declares, and rejects
bad arguments before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2411_00742_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_header_functions_exported(lib):
    names = _lib.header_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} has no ctypes signature"


def test_version(lib):
    assert lib.pbe_version() >= 100


def test_bad_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    nc = (ctypes.c_int64 * 2)(10, 10)
    lm = (ctypes.c_double * 2)(1.0, 1.0)
    assert lib.pbe_create_grid(ctypes.byref(h), 3, nc, lm) == _lib.PBE_EINVAL
    assert b"ndim" in lib.pbe_last_error()
    nc0 = (ctypes.c_int64 * 2)(0, 10)
    assert lib.pbe_create_grid(ctypes.byref(h), 1, nc0, lm) == _lib.PBE_EINVAL
    lm0 = (ctypes.c_double * 2)(-1.0, 1.0)
    assert lib.pbe_create_grid(ctypes.byref(h), 1, nc, lm0) == _lib.PBE_EINVAL
    assert lib.pbe_create_grid(None, 1, nc, lm) == _lib.PBE_EINVAL
    assert lib.pbe_set_path(None, 0) == _lib.PBE_EINVAL
    assert lib.pbe_solve(None, None, 0, None, 0, None) == _lib.PBE_EINVAL
    assert lib.pbe_destroy_grid(None) == _lib.PBE_OK


def test_no_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_2411_00742_gb300 as P
    with pytest.raises(P.PbeError) as e:
        P.Grid(1, (10,), (1.0,))
    assert e.value.status == _lib.PBE_ECUDA


def _imports(path):
    src = open(path).read()
    return set(re.findall(r"^\s*(?:from|import)\s+([A-Za-z_][\w.]*)", src, flags=re.M))


def test_product_and_oracle_are_independent():
    pkg = os.path.join(ROOT, "paper_2411_00742_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            p = os.path.join(dirpath, f)
            if f.endswith(".py"):
                assert not any(m.split(".")[0] in ("oracle", "pbe_inputs") for m in _imports(p)), p
            if f.endswith((".cu", ".cuh", ".h", ".c")):
                assert "pbe_oracle" not in open(p).read(), p
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        p = os.path.join(ROOT, "oracle", f)
        if f.endswith(".py"):
            assert not any(m.split(".")[0] == "paper_2411_00742_gb300" for m in _imports(p)), p
        if f.endswith((".c", ".h")):
            assert "pbe.h" not in open(p).read() and "pbe_device" not in open(p).read(), p
