"""ctypes declarations of the C ABI in include/pbe.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

PBE_OK, PBE_EINVAL, PBE_ENOMEM, PBE_ECUDA, PBE_ENONFINITE, PBE_ETIMEOUT, PBE_ESTATE = range(7)
PBE_MEM_HOST, PBE_MEM_DEVICE = 0, 1
PBE_KINETICS_POWER_LAW, PBE_KINETICS_FIXED, PBE_KINETICS_MLP = 0, 1, 2
PBE_PATH_PLAIN, PBE_PATH_FUSED, PBE_PATH_AUTO = 0, 1, 2

STATUS_NAMES = {0: "PBE_OK", 1: "PBE_EINVAL", 2: "PBE_ENOMEM", 3: "PBE_ECUDA", 4: "PBE_ENONFINITE",
                5: "PBE_ETIMEOUT", 6: "PBE_ESTATE"}


class PbeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Kinetics(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("kg", ctypes.c_double * 2), ("g", ctypes.c_double * 2),
                ("kb", ctypes.c_double), ("b", ctypes.c_double), ("csat", ctypes.c_double * 3),
                ("T0", ctypes.c_double), ("T1", ctypes.c_double), ("t_cool", ctypes.c_double),
                ("kappa", ctypes.c_double), ("cfl", ctypes.c_double),
                ("scheme", ctypes.c_int), ("growth_form", ctypes.c_int), ("solubility_form", ctypes.c_int),
                ("ea", ctypes.c_double * 2)]


class Instance(ctypes.Structure):
    _fields_ = [("ncells", ctypes.c_int64), ("lmax", ctypes.c_double), ("kin", Kinetics),
                ("C0", ctypes.c_double), ("t0", ctypes.c_double)]


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)

# name -> argtypes (restype is pbe_status = int unless listed in _RESTYPES)
SIGNATURES = {
    "pbe_create_grid": [ctypes.POINTER(_P), _I, _PI64, _PD],
    "pbe_destroy_grid": [_P],
    "pbe_set_stream": [_P, _P],
    "pbe_set_path": [_P, _I],
    "pbe_set_kinetics": [_P, ctypes.POINTER(Kinetics)],
    "pbe_set_state": [_P, _P, _D, _D, _I],
    "pbe_init_seed_gaussian": [_P, _PD, _PD, _D, _D, _D],
    "pbe_init_seed_gaussian_mass": [_P, _PD, _PD, _D, _D, _D, _D],
    "pbe_get_state": [_P, _P, _PD, _PD, _I],
    "pbe_step": [_P, _D, _PD],
    "pbe_solve": [_P, _PD, _I, _P, _I, _PI64],
    "pbe_moments": [_P, _P, _I],
    "pbe_set_max_steps": [_P, _I64],
    "pbe_set_growth_poly": [_P, _PD, _I],
    "pbe_set_closure_box": [_P, _PD, _PD],
    "pbe_closure_grad": [ctypes.POINTER(_P), _I, _PD],
    "pbe_growth_poly_grad": [_P, _PD, _I],
    "pbe_set_wait_limit": [_P, _D],
    "pbe_set_block_limit": [_P, _I],
    "pbe_set_window": [_P, _I],
    "pbe_set_timing": [_P, _I],
    "pbe_kernel_time": [_P, _PD],
    "pbe_vjp": [_P, _PD, _I, _P, _I, _I, _PD, _P, _PD, _P, _I, _PD],
    "pbe_set_closure": [_P, ctypes.POINTER(ctypes.c_float), _I],
    "pbe_solve_1d_noalloc": [ctypes.POINTER(Kinetics), _I64, _D, _P, _D, _D, _PD, _I, _P, _PI64, _P],
    "pbe_batch_create": [ctypes.POINTER(_P), ctypes.POINTER(Instance), _I],
    "pbe_batch_destroy": [_P],
    "pbe_batch_set_stream": [_P, _P],
    "pbe_batch_offsets": [_P, _PI64],
    "pbe_batch_set_state": [_P, _P, _I],
    "pbe_batch_get_state": [_P, _P, _P, _P, _I],
    "pbe_batch_solve": [_P, _PD, _I, _P, _I, _PI64],
    "pbe_batch_set_config": [_P, _I],
    "pbe_batch_set_schedule": [_P, _I, _I, _I],
    "pbe_batch_set_closure": [_P, ctypes.POINTER(ctypes.c_float), _I],
    "pbe_batch_set_closure_box": [_P, _P, _P],
    "pbe_batch_set_vjp_schedule": [_P, _I, _I],
    "pbe_batch_get_schedule": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "pbe_batch_vjp": [_P, _PD, _I, _P, _I, _I, _PD, _PD, _P, _I],
    "pbe_batch_steps": [_P, _PI64],
    "pbe_batch_autotune": [_P, _PD, _I, ctypes.POINTER(_I)],
    "pbe_adam_update": [_P, _P, _P, _P, _I, _D, _D, _D, _D, _I, _P],
    "pbe_last_error": [],
    "pbe_version": [],
}
_RESTYPES = {"pbe_last_error": ctypes.c_char_p, "pbe_version": ctypes.c_int}

_lib = None


def header_functions(path: str | None = None) -> list[str]:
    """Names of the functions declared in include/pbe.h."""
    path = path or os.path.join(_build.INCLUDE, "pbe.h")
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pbe_[a-z0-9_]+)\s*\(", src)))


def load(build_if_missing: bool = True):
    """Load libpbe.so; raises if it is missing and cannot be built.  There is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"CUDA extension missing: {_build.LIB} (run __graft_entry__.build())")
    lib = ctypes.CDLL(_build.LIB)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = _RESTYPES.get(name, ctypes.c_int)
    _lib = lib
    return lib


def check(status: int):
    if status != PBE_OK:
        raise PbeError(status, load().pbe_last_error().decode(errors="replace"))
