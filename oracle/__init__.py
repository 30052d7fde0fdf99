"""CPU FP64 oracle of the crystallization PBE step (Sec. 2.1; SI Sec. S1).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2411_00742_gb300``) never imports, links or runs anything here, and
this package never imports the product path.

The oracle is a plain C program (``pbe_oracle.c``) compiled with
``-O2 -ffp-contract=off`` and loaded through ctypes; ``mom.py`` holds the
method-of-moments reference (SI Sec. S1.2), ``exact.py`` an exact-rational
brute force for tiny grids.

Parity status: every function exported here is pinned by a ``-m "not gpu"``
test against closed forms, invariants, exact translation, the method of
moments or exact rational arithmetic (see ``tests/test_oracle_*.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpbe_oracle.so")
_SOURCES = [os.path.join(_HERE, "pbe_oracle.c"), os.path.join(_HERE, "pbe_oracle_core.h"),
]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fp contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [s for s in _SOURCES if os.path.exists(s)]
    if not force and os.path.exists(_LIB_PATH):
        mtime = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= mtime for s in srcs):
            return _LIB_PATH
    cfiles = [s for s in srcs if s.endswith(".c")]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall",
           "-o", tmp] + cfiles + ["-lm"]
    # with OpenMP where the compiler has it (threads only for the timed CPU
    # baseline: the results are the same on any thread count)
    r = subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], cwd=_HERE, capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("lmax1", ctypes.c_double), ("lmax2", ctypes.c_double),
                ("fixed_kinetics", ctypes.c_int),
                ("kg1", ctypes.c_double), ("g1", ctypes.c_double),
                ("kg2", ctypes.c_double), ("g2", ctypes.c_double),
                ("kb", ctypes.c_double), ("b", ctypes.c_double),
                ("cs0", ctypes.c_double), ("cs1", ctypes.c_double), ("cs2", ctypes.c_double),
                ("T0", ctypes.c_double), ("T1", ctypes.c_double), ("t_cool", ctypes.c_double),
                ("kappa", ctypes.c_double), ("cfl", ctypes.c_double),
                ("mlp", ctypes.POINTER(ctypes.c_double)),
                ("scheme", ctypes.c_int), ("growth_form", ctypes.c_int), ("solubility_form", ctypes.c_int),
                ("ea1", ctypes.c_double), ("ea2", ctypes.c_double),
                ("poly", ctypes.POINTER(ctypes.c_double)), ("npoly", ctypes.c_int),
                ("mlp_box", ctypes.c_int), ("mlp_lo", ctypes.c_double * 3), ("mlp_hi", ctypes.c_double * 3)]


_lib = None
_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(Params)
        lib.orc_psi.restype = ctypes.c_double
        lib.orc_psi.argtypes = [ctypes.c_double, ctypes.c_double]
        lib.orc_temperature.restype = ctypes.c_double
        lib.orc_temperature.argtypes = [P, ctypes.c_double]
        lib.orc_kinetics.argtypes = [P, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_kinetics_mlp.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_timestep.restype = ctypes.c_int
        lib.orc_timestep.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, _D]
        lib.orc_rhs.argtypes = [P, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_face_fluxes.argtypes = [P, _D, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.orc_volume.restype = ctypes.c_double
        lib.orc_volume.argtypes = [P, _D]
        lib.orc_moments.argtypes = [P, _D, _D]
        lib.orc_step.argtypes = [P, _D, ctypes.c_double, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_solve.restype = ctypes.c_long
        lib.orc_solve.argtypes = [P, _D, ctypes.c_double, ctypes.c_double, _D, ctypes.c_int, _D, _D]
        lib.orc_solve_cs.restype = ctypes.c_long
        lib.orc_solve_cs.argtypes = [P, ctypes.c_int, ctypes.c_double, _D, ctypes.c_double,
                                     ctypes.c_double, _D, ctypes.c_int, _D, _D]
        lib.orc_set_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads(1)   # one thread unless set_threads says otherwise
        lib.orc_vjp.restype = ctypes.c_long
        lib.orc_vjp.argtypes = [P, _D, ctypes.c_double, ctypes.c_double, _D, ctypes.c_int,
                                _D, _D, _D, _D, _D, _D]
        _lib = lib
    return _lib


MLP_NW = 64 * 3 + 64 + 64 * 64 + 64 + 3 * 64 + 3   # learned closure weight count
_mlp_keep = {}


def set_threads(n: int) -> int:
    """Threads of the oracle's element-wise loops (2-D right-hand side and stage
    updates); returns the count in effect.  Results are identical on any count."""
    return int(_load().orc_set_threads(int(n)))


def _poly(problem) -> np.ndarray:
    """Polynomial growth coefficients of Eq. 6 (growth_form 2): ndim rows of K,
    a_m1 .. a_mK of G_m = sum_k a_mk (S - 1)^k."""
    a = np.ascontiguousarray(getattr(problem, "poly", ()), dtype=np.float64).reshape(-1)
    if getattr(problem, "growth_form", 0) == 2:
        assert a.size > 0 and a.size % problem.ndim == 0, "poly holds ndim x K coefficients"
    return a


def params(problem, mlp=None) -> Params:
    """ctypes parameter block; mlp = flat float64 weights of the learned closure
    (layout W1[64][3], b1, W2[64][64], b2, W3[3][64], b3) or None."""
    p = problem
    n2 = p.ncells[1] if p.ndim == 2 else 1
    l2 = p.lmax[1] if p.ndim == 2 else 1.0
    mp = None
    if mlp is not None:
        arr = np.ascontiguousarray(mlp, dtype=np.float64)
        assert arr.size == MLP_NW
        _mlp_keep[id(arr)] = arr
        mp = arr.ctypes.data_as(_D)
    P = Params(p.ndim, int(p.ncells[0]), int(n2), float(p.lmax[0]), float(l2),
               int(bool(p.fixed_kinetics)),
               float(p.kg[0]), float(p.g[0]), float(p.kg[1]), float(p.g[1]),
               float(p.kb), float(p.b),
               float(p.csat[0]), float(p.csat[1]), float(p.csat[2]),
               float(p.T0), float(p.T1), float(p.t_cool), float(p.kappa), float(p.cfl), mp,
               int(getattr(p, "scheme", 0)), int(getattr(p, "growth_form", 0)), int(getattr(p, "solubility_form", 0)),
               float(getattr(p, "ea", (0.0, 0.0))[0]), float(getattr(p, "ea", (0.0, 0.0))[1]))
    poly = _poly(p)
    if poly.size:
        P.poly = poly.ctypes.data_as(_D)
        P.npoly = poly.size // p.ndim
    box = getattr(p, "mlp_box", ())
    if box:
        P.mlp_box = 1
        for k in range(3):
            P.mlp_lo[k], P.mlp_hi[k] = float(box[0][k]), float(box[1][k])
    P._keep = (arr if mlp is not None else None, poly)
    return P


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def ncols(problem) -> int:
    return 6 if problem.ndim == 1 else 12


def psi(a: float, b: float) -> float:
    return _load().orc_psi(float(a), float(b))


def temperature(problem, t: float) -> float:
    P = params(problem)
    return _load().orc_temperature(ctypes.byref(P), float(t))


def kinetics(problem, C: float, t: float):
    """(G1, G2, B) at concentration C and time t."""
    P = params(problem)
    out = np.zeros(3)
    _load().orc_kinetics(ctypes.byref(P), float(C), float(t), _ptr(out))
    return tuple(out)


def timestep(problem, G1: float, G2: float, t: float, t_next: float):
    """(dt, t_new, clipped)."""
    P = params(problem)
    out = np.zeros(2)
    c = _load().orc_timestep(ctypes.byref(P), float(G1), float(G2), float(t), float(t_next), _ptr(out))
    return out[0], out[1], bool(c)


def rhs(problem, n, G1: float, G2: float, B: float) -> np.ndarray:
    P = params(problem)
    n = np.ascontiguousarray(n, dtype=np.float64)
    L = np.zeros_like(n)
    _load().orc_rhs(ctypes.byref(P), _ptr(n), float(G1), float(G2), float(B), _ptr(L))
    return L


def face_fluxes(problem, n, G1: float, G2: float = 0.0):
    P = params(problem)
    n = np.ascontiguousarray(n, dtype=np.float64)
    if problem.ndim == 1:
        F = np.zeros(problem.ncells[0] + 1)
        _load().orc_face_fluxes(ctypes.byref(P), _ptr(n), float(G1), 0.0, _ptr(F), _ptr(F))
        return F
    N1, N2 = problem.ncells
    F1 = np.zeros((N1 + 1, N2))
    F2 = np.zeros((N1, N2 + 1))
    _load().orc_face_fluxes(ctypes.byref(P), _ptr(n), float(G1), float(G2), _ptr(F1), _ptr(F2))
    return F1, F2


def volume(problem, n) -> float:
    P = params(problem)
    return _load().orc_volume(ctypes.byref(P), _ptr(np.ascontiguousarray(n, dtype=np.float64)))


def moments(problem, n) -> np.ndarray:
    P = params(problem)
    mu = np.zeros(4 if problem.ndim == 1 else 10)
    _load().orc_moments(ctypes.byref(P), _ptr(np.ascontiguousarray(n, dtype=np.float64)), _ptr(mu))
    return mu


def step(problem, n, C: float, t: float, t_next: float):
    """One SSP-RK2 step.  Returns (n_new, dict(dt, C, t, C1, clipped))."""
    P = params(problem)
    n = np.array(n, dtype=np.float64, order="C", copy=True)
    out = np.zeros(5)
    _load().orc_step(ctypes.byref(P), _ptr(n), float(C), float(t), float(t_next), _ptr(out))
    return n, dict(dt=out[0], C=out[1], t=out[2], C1=out[3], clipped=bool(out[4]))


def solve(problem, n0, C0: float, t0: float, t_out, mlp=None):
    """March through the output times.  Returns dict(rows, n, C, t, steps).

    rows[j] = (t, mu0..mu3, C) in 1-D and (t, mu00, mu10, mu01, mu20, mu11,
    mu02, mu30, mu21, mu12, mu03, C) in 2-D."""
    t_out = np.ascontiguousarray(t_out, dtype=np.float64)
    if len(t_out) and (t_out[0] < t0 or np.any(np.diff(t_out) <= 0)):
        raise ValueError("t_out must be increasing and start at or after t0")
    P = params(problem, mlp)
    n = np.array(n0, dtype=np.float64, order="C", copy=True)
    rows = np.zeros((len(t_out), ncols(problem)))
    st = np.zeros(2)
    steps = _load().orc_solve(ctypes.byref(P), _ptr(n), float(C0), float(t0), _ptr(t_out),
                              len(t_out), _ptr(rows), _ptr(st))
    return dict(rows=rows, n=n, C=st[0], t=st[1], steps=int(steps))


def solve_cs(problem, which: int, n0, C0: float, t0: float, t_out, h: float = 1e-30, mlp=None):
    """Complex-step derivative of all output rows w.r.t. kinetic parameter
    ``which`` (0..5 = kg1, g1, kg2, g2, kb, b; 6 + k = closure weight k, or
    polynomial growth coefficient k with growth_form 2).  Returns (rows, drows)."""
    t_out = np.ascontiguousarray(t_out, dtype=np.float64)
    P = params(problem, mlp)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    rows = np.zeros((len(t_out), ncols(problem)))
    drows = np.zeros_like(rows)
    steps = _load().orc_solve_cs(ctypes.byref(P), int(which), float(h), _ptr(n0), float(C0), float(t0),
                                 _ptr(t_out), len(t_out), _ptr(rows), _ptr(drows))
    if steps < 0:
        raise ValueError(f"no differentiable parameter {which}")
    return rows, drows


def solve_instance(inst):
    return solve(inst.problem, inst.n0, inst.C0, inst.t0, inst.t_out)


def vjp(problem, n0, C0: float, t0: float, t_out, drows, mlp=None):
    """Hand-written discrete adjoint: dL/dtheta (kg1, g1, kg2, g2, kb, b), dL/dn0, dL/dC0
    (and dL/dweights of the learned closure when mlp is given, or dL/d(polynomial
    growth coefficients) with growth_form 2, as a fourth result) for seeds
    drows = dL/d(rows) (time column ignored)."""
    t_out = np.ascontiguousarray(t_out, dtype=np.float64)
    drows = np.ascontiguousarray(drows, dtype=np.float64)
    assert drows.shape == (len(t_out), ncols(problem))
    P = params(problem, mlp)
    n0 = np.ascontiguousarray(n0, dtype=np.float64)
    dth = np.zeros(6)
    dn0 = np.zeros_like(n0)
    dC0 = np.zeros(1)
    dW = np.zeros(MLP_NW)
    dA = np.zeros(max(_poly(problem).size, 1))
    steps = _load().orc_vjp(ctypes.byref(P), _ptr(n0), float(C0), float(t0), _ptr(t_out), len(t_out),
                            _ptr(drows), _ptr(dth), _ptr(dn0), _ptr(dC0), _ptr(dW), _ptr(dA))
    if steps < 0:
        raise ValueError("no adjoint for this scheme / kinetics form")
    if mlp is not None:
        return dth, dn0, dC0[0], dW
    if getattr(problem, "growth_form", 0) == 2:
        return dth, dn0, dC0[0], dA
    return dth, dn0, dC0[0]


def kinetics_mlp(problem, mlp, C: float, t: float, ratio: float):
    """(G1, G2, B) of the learned closure at concentration C, time t and moment ratio V/mu0."""
    P = params(problem, mlp)
    out = np.zeros(3)
    _load().orc_kinetics_mlp(ctypes.byref(P), float(C), float(t), float(ratio), _ptr(out))
    return tuple(out)


def relative_loss(rows, target, cols):
    """Sum of squared relative errors of the chosen row columns (the parameter
    estimation objective of Sec. 4.1, Eq. 5, with relative residuals)."""
    r = (rows[:, cols] - target[:, cols]) / target[:, cols]
    return float(np.sum(r * r))


def relative_loss_seeds(rows, target, cols):
    """dL/drows of relative_loss."""
    g = np.zeros_like(rows)
    g[:, cols] = 2.0 * (rows[:, cols] - target[:, cols]) / target[:, cols] ** 2
    return g
