"""GB300 (sm_103a) solver for the crystallization population balance equation.

The explicit high-resolution finite-volume step (Sec. 2.1, Eq. 3 in
semi-discrete form, SI Sec. S1.1) with its coupled solute balance (Eq. 4)
runs entirely in the CUDA kernels of ``libpbe.so``; this package only
marshals arguments to the C ABI declared in ``include/pbe.h``.  PyTorch is
used for device memory and streams.  There is no CPU fallback: every call
raises if the CUDA library or a device is unavailable.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (PBE_KINETICS_FIXED, PBE_KINETICS_MLP, PBE_KINETICS_POWER_LAW, PBE_MEM_DEVICE, PBE_MEM_HOST,
                   PBE_PATH_AUTO, PBE_PATH_FUSED, PBE_PATH_PLAIN, PbeError, Kinetics)

CLOSURE_SIZE = 64 * 3 + 64 + 64 * 64 + 64 + 3 * 64 + 3   # weights of the learned closure

__all__ = ["Grid", "Batch", "PbeError", "kinetics_struct", "ncols", "closure_grad"]

_PATHS = {"plain": PBE_PATH_PLAIN, "fused": PBE_PATH_FUSED, "auto": PBE_PATH_AUTO}


def ncols(ndim: int) -> int:
    return 6 if ndim == 1 else 12


def kinetics_struct(problem, theta=None, closure: bool = False) -> Kinetics:
    """pbe_kinetics from any object with the fields of a problem description
    (kg, g, kb, b, csat, T0, T1, t_cool, kappa, cfl, fixed_kinetics);
    theta = (kg1, g1, kg2, g2, kb, b) overrides the kinetic parameters."""
    k = Kinetics()
    k.kind = PBE_KINETICS_FIXED if getattr(problem, "fixed_kinetics", False) else PBE_KINETICS_POWER_LAW
    if theta is None:
        theta = (problem.kg[0], problem.g[0], problem.kg[1], problem.g[1], problem.kb, problem.b)
    th = [float(v) for v in theta]
    k.kg[0], k.g[0], k.kg[1], k.g[1], k.kb, k.b = th
    if closure:
        k.kind = PBE_KINETICS_MLP
    for i in range(3):
        k.csat[i] = float(problem.csat[i])
    k.T0, k.T1, k.t_cool = float(problem.T0), float(problem.T1), float(problem.t_cool)
    k.kappa, k.cfl = float(problem.kappa), float(problem.cfl)
    k.scheme = int(getattr(problem, "scheme", 0))
    k.growth_form = int(getattr(problem, "growth_form", 0))
    k.solubility_form = int(getattr(problem, "solubility_form", 0))
    ea = getattr(problem, "ea", (0.0, 0.0))
    k.ea[0], k.ea[1] = float(ea[0]), float(ea[1])
    return k


def _buf(x, writable=False):
    """(pointer, mem flag, keepalive) for a float64 contiguous torch tensor or numpy array."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                raise TypeError("expected a contiguous float64 tensor")
            return ctypes.c_void_p(x.data_ptr()), (PBE_MEM_DEVICE if x.is_cuda else PBE_MEM_HOST), x
    except ImportError:  # pragma: no cover
        pass
    a = np.asarray(x)
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        if writable:
            raise TypeError("expected a contiguous float64 array")
        a = np.ascontiguousarray(a, dtype=np.float64)
    return ctypes.c_void_p(a.ctypes.data), PBE_MEM_HOST, a


class Grid:
    """A PBE grid on the current CUDA device (thin wrapper over pbe_grid)."""

    def __init__(self, ndim: int, ncells, lmax, stream=None):
        self.lib = _lib.load()
        self.ndim = int(ndim)
        self.ncells = tuple(int(v) for v in ncells)
        nc = (ctypes.c_int64 * 2)(*(list(self.ncells) + [1] * (2 - len(self.ncells))))
        lm = (ctypes.c_double * 2)(*([float(v) for v in lmax] + [1.0] * (2 - len(lmax))))
        h = ctypes.c_void_p()
        _lib.check(self.lib.pbe_create_grid(ctypes.byref(h), self.ndim, nc, lm))
        self.h = h
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_problem(cls, problem, stream=None, path: str = "plain"):
        g = cls(problem.ndim, problem.ncells, problem.lmax, stream=stream)
        g.set_kinetics(problem)
        g.set_path(path)
        return g

    @property
    def ncell(self) -> int:
        return int(np.prod(self.ncells))

    def close(self):
        if getattr(self, "h", None):
            self.lib.pbe_destroy_grid(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _lib.check(self.lib.pbe_set_stream(self.h, ctypes.c_void_p(int(handle))))

    def set_path(self, path: str):
        """"plain", "fused" or "auto" (the faster path for the configuration: fused,
        which falls back to plain for the paper scheme)."""
        _lib.check(self.lib.pbe_set_path(self.h, _PATHS[path]))

    def set_window(self, mode: int):
        """Plain-path 2-D stage kernel: -1 auto (default), 0 tile kernel, 1 register-window kernel."""
        _lib.check(self.lib.pbe_set_window(self.h, int(mode)))

    def set_wait_limit(self, seconds: float):
        _lib.check(self.lib.pbe_set_wait_limit(self.h, float(seconds)))

    def set_block_limit(self, blocks: int):
        """Most blocks of the fused path's persistent launches (0: one per SM)."""
        _lib.check(self.lib.pbe_set_block_limit(self.h, int(blocks)))

    def set_max_steps(self, n: int):
        _lib.check(self.lib.pbe_set_max_steps(self.h, int(n)))

    def set_timing(self, enable: bool = True):
        """Record CUDA events around the launch that advances the state in every solve."""
        _lib.check(self.lib.pbe_set_timing(self.h, 1 if enable else 0))

    def kernel_time_ms(self) -> float:
        """Device time of that launch in the last solve (ms; -1 when not recorded)."""
        v = ctypes.c_double(-1.0)
        _lib.check(self.lib.pbe_kernel_time(self.h, ctypes.byref(v)))
        return v.value

    def set_closure(self, weights):
        """Weights of the learned kinetics closure (flat float32, layout W1, b1, W2, b2, W3, b3);
        the matrices are stored as bf16."""
        w = np.ascontiguousarray(weights, dtype=np.float32)
        if w.size != CLOSURE_SIZE:
            raise ValueError(f"the closure has {CLOSURE_SIZE} weights")
        _lib.check(self.lib.pbe_set_closure(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size))

    def set_closure_box(self, lo=None, hi=None):
        """Training box of the closure's inputs (None: no box); outside it, and for
        non-finite network rates, the power law of the kinetic parameters is used."""
        if lo is None or hi is None:
            _lib.check(self.lib.pbe_set_closure_box(self.h, None, None))
            return
        lo = (ctypes.c_double * 3)(*[float(v) for v in lo])
        hi = (ctypes.c_double * 3)(*[float(v) for v in hi])
        _lib.check(self.lib.pbe_set_closure_box(self.h, lo, hi))

    def set_kinetics(self, problem, theta=None, closure: bool = False):
        k = kinetics_struct(problem, theta, closure)
        if k.growth_form == 2:
            self.set_growth_poly(problem.poly)
        box = getattr(problem, "mlp_box", ())
        if closure and box:
            self.set_closure_box(box[0], box[1])
        _lib.check(self.lib.pbe_set_kinetics(self.h, ctypes.byref(k)))

    def set_growth_poly(self, a):
        """Coefficients a_mk of the polynomial growth law (Eq. 6), ndim x K (flat, direction-major)."""
        a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
        if a.size == 0 or a.size % self.ndim:
            raise ValueError("the growth polynomial holds ndim x K coefficients")
        _lib.check(self.lib.pbe_set_growth_poly(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                a.size // self.ndim))
        self._npoly = a.size

    def growth_poly_grad(self):
        """dL/da of the polynomial growth law from the last vjp (fused path)."""
        out = np.zeros(getattr(self, "_npoly", 0))
        _lib.check(self.lib.pbe_growth_poly_grad(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 out.size))
        return out

    def set_state(self, n, C: float, t: float):
        p, mem, keep = _buf(n)
        if (keep.numel() if hasattr(keep, "numel") else keep.size) != self.ncell:
            raise ValueError("state has the wrong number of cells")
        _lib.check(self.lib.pbe_set_state(self.h, p, float(C), float(t), mem))

    def init_seed_gaussian(self, mean, sd, corr: float = 0.0, total_number: float | None = None,
                           C0: float = 0.0, seed_mass: float | None = None, rho_kv: float | None = None):
        """Normal seed at the cell centres, scaled to a number of crystals
        (total_number) or to a seed mass (seed_mass with rho_kv); C = C0, t = 0."""
        m = (ctypes.c_double * 2)(*[float(v) for v in list(mean)[:2]] + [0.0] * (2 - len(list(mean)[:2])))
        s = (ctypes.c_double * 2)(*[float(v) for v in list(sd)[:2]] + [1.0] * (2 - len(list(sd)[:2])))
        if (total_number is None) == (seed_mass is None):
            raise ValueError("give exactly one of total_number and seed_mass")
        if seed_mass is None:
            _lib.check(self.lib.pbe_init_seed_gaussian(self.h, m, s, float(corr), float(total_number), float(C0)))
        else:
            if rho_kv is None:
                raise ValueError("seed_mass needs rho_kv")
            _lib.check(self.lib.pbe_init_seed_gaussian_mass(self.h, m, s, float(corr), float(seed_mass),
                                                            float(rho_kv), float(C0)))

    def get_state(self, out=None):
        """Returns (n, C, t); n is written into ``out`` (tensor/array) or a new numpy array."""
        if out is None:
            out = np.zeros(self.ncells)
        p, mem, keep = _buf(out, writable=True)
        C, t = ctypes.c_double(), ctypes.c_double()
        _lib.check(self.lib.pbe_get_state(self.h, p, ctypes.byref(C), ctypes.byref(t), mem))
        return out, C.value, t.value

    def step(self, t_limit: float) -> float:
        dt = ctypes.c_double()
        _lib.check(self.lib.pbe_step(self.h, float(t_limit), ctypes.byref(dt)))
        return dt.value

    def solve(self, t_out, out=None):
        """March through the output times; returns (rows, steps)."""
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        if out is None:
            out = np.zeros((len(t_out), ncols(self.ndim)))
        p, mem, keep = _buf(out, writable=True)
        steps = ctypes.c_int64()
        _lib.check(self.lib.pbe_solve(self.h, t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      len(t_out), p, mem, ctypes.byref(steps)))
        return out, steps.value

    def vjp(self, t_out, seeds, checkpoint_every: int = 64, dn0_out=None, rows_out=None, dweights_out=None):
        """Gradient of a scalar loss of the rows of solve(t_out) from the current
        state, given seeds = dL/drows.  Returns (dL/dtheta[6], dL/dn0 or None, dL/dC0);
        with the learned closure, dweights_out (float64, CLOSURE_SIZE) receives
        dL/dweights."""
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        sp, smem, skeep = _buf(seeds)
        dth = np.zeros(6)
        dC0 = ctypes.c_double()
        mem = PBE_MEM_HOST
        dn_p = None
        if dn0_out is not None:
            dn_p, mem, dkeep = _buf(dn0_out, writable=True)
        rows_p = None
        if rows_out is not None:
            rows_p, rmem, rkeep = _buf(rows_out, writable=True)
            if dn0_out is not None and rmem != mem:
                raise ValueError("dn0_out and rows_out must live in the same memory")
            mem = rmem
        _lib.check(self.lib.pbe_vjp(self.h, t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t_out),
                                    sp, smem, int(checkpoint_every),
                                    dth.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dn_p,
                                    ctypes.byref(dC0), rows_p, mem,
                                    None if dweights_out is None else
                                    np.ascontiguousarray(dweights_out).ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return dth, dn0_out, dC0.value

    def moments(self, out=None):
        if out is None:
            out = np.zeros(4 if self.ndim == 1 else 10)
        p, mem, keep = _buf(out, writable=True)
        _lib.check(self.lib.pbe_moments(self.h, p, mem))
        return out


def closure_grad(grids) -> np.ndarray:
    """Summed dL/dweights of the learned closure over the last (fused-path) vjp of
    every grid: one launch of the tensor-core weight-gradient kernel."""
    grids = list(grids)
    arr = (ctypes.c_void_p * len(grids))(*[g.h.value if hasattr(g.h, "value") else g.h for g in grids])
    out = np.zeros(CLOSURE_SIZE)
    lib = _lib.load()
    _lib.check(lib.pbe_closure_grad(arr, len(grids), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


class Batch:
    """Many independent 1-D instances solved by one persistent launch
    (thin wrapper over pbe_batch)."""

    def __init__(self, problems, C0, t0=None, stream=None, closure=False):
        """closure: the instances' rates come from the learned closure (set its
        weights with set_closure before solving; the power law of each problem
        is the fallback)."""
        self.lib = _lib.load()
        n = len(problems)
        arr = (_lib.Instance * n)()
        for i, p in enumerate(problems):
            if p.ndim != 1:
                raise ValueError("batched solves are 1-D")
            arr[i].ncells = int(p.ncells[0])
            arr[i].lmax = float(p.lmax[0])
            arr[i].kin = kinetics_struct(p, closure=closure)
            arr[i].C0 = float(C0[i])
            arr[i].t0 = 0.0 if t0 is None else float(t0[i])
        h = ctypes.c_void_p()
        _lib.check(self.lib.pbe_batch_create(ctypes.byref(h), arr, n))
        self.h = h
        self.count = n
        off = (ctypes.c_int64 * (n + 1))()
        _lib.check(self.lib.pbe_batch_offsets(self.h, off))
        self.offsets = np.array(off[:], dtype=np.int64)
        if stream is not None:
            self.set_stream(stream)

    @property
    def total_cells(self) -> int:
        return int(self.offsets[-1])

    def close(self):
        if getattr(self, "h", None):
            self.lib.pbe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        handle = getattr(stream, "cuda_stream", stream)
        _lib.check(self.lib.pbe_batch_set_stream(self.h, ctypes.c_void_p(int(handle))))

    def pack(self, states):
        return np.concatenate([np.ascontiguousarray(s, dtype=np.float64).ravel() for s in states])

    def set_state(self, n_packed):
        p, mem, keep = _buf(n_packed)
        _lib.check(self.lib.pbe_batch_set_state(self.h, p, mem))

    def get_state(self):
        n = np.zeros(self.total_cells)
        C = np.zeros(self.count)
        t = np.zeros(self.count)
        _lib.check(self.lib.pbe_batch_get_state(self.h, ctypes.c_void_p(n.ctypes.data), ctypes.c_void_p(C.ctypes.data),
                                                ctypes.c_void_p(t.ctypes.data), PBE_MEM_HOST))
        return [n[self.offsets[i]:self.offsets[i + 1]] for i in range(self.count)], C, t

    def steps(self) -> np.ndarray:
        """Steps each instance took in the last solve."""
        st = (ctypes.c_int64 * self.count)()
        _lib.check(self.lib.pbe_batch_steps(self.h, st))
        return np.array(st[:], dtype=np.int64)

    def cell_steps(self) -> int:
        """Sum over instances of cells x steps of the last solve."""
        return int(np.sum(np.diff(self.offsets) * self.steps()))

    def vjp(self, t_out, seeds, checkpoint_every: int = 64, dn0_out=None):
        """Per-instance gradients: returns (dL/dtheta [count, 6], dL/dC0 [count]);
        dn0_out (CUDA float64 packed state) receives dL/dn0 when given."""
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        sp, smem, skeep = _buf(seeds)
        dth = np.zeros((self.count, 6))
        dC0 = np.zeros(self.count)
        dn_p = None
        if dn0_out is not None:
            dn_p, _, dkeep = _buf(dn0_out, writable=True)
        _lib.check(self.lib.pbe_batch_vjp(self.h, t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t_out),
                                          sp, smem, int(checkpoint_every),
                                          dth.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          dC0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), dn_p, PBE_MEM_DEVICE))
        return dth, dC0

    def set_config(self, warps_per_block: int):
        _lib.check(self.lib.pbe_batch_set_config(self.h, int(warps_per_block)))

    def set_closure(self, weights):
        """Weights of the learned closure for the batch's closure instances
        (flat float32, the layout of Grid.set_closure)."""
        w = np.ascontiguousarray(weights, dtype=np.float32)
        if w.size != CLOSURE_SIZE:
            raise ValueError(f"the closure has {CLOSURE_SIZE} weights")
        _lib.check(self.lib.pbe_batch_set_closure(self.h, w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), w.size))

    def set_closure_box(self, lo=None, hi=None):
        """Training box of the closure's inputs (None: no box), as Grid.set_closure_box."""
        if lo is None or hi is None:
            _lib.check(self.lib.pbe_batch_set_closure_box(self.h, None, None))
            return
        lo = (ctypes.c_double * 3)(*[float(v) for v in lo])
        hi = (ctypes.c_double * 3)(*[float(v) for v in hi])
        _lib.check(self.lib.pbe_batch_set_closure_box(self.h, lo, hi))

    def set_schedule(self, warps_per_block: int, team_instances: int, warp_cells: int = 6144):
        """Warps per block, the number of costliest instances solved by a whole
        block each, and the largest instance solved by one warp (larger ones
        are team instances too): pbe_batch_set_schedule."""
        _lib.check(self.lib.pbe_batch_set_schedule(self.h, int(warps_per_block), int(team_instances),
                                                   int(warp_cells)))

    def set_vjp_schedule(self, warps: int = 0, blocks_per_sm: int = 0):
        """Warps per instance of vjp (1, 2, 4, 8) and resident teams per SM;
        0 = chosen from the batch size (pbe_batch_set_vjp_schedule)."""
        _lib.check(self.lib.pbe_batch_set_vjp_schedule(self.h, int(warps), int(blocks_per_sm)))

    def schedule(self) -> tuple[int, int, int]:
        """(warps per block, team instances, warp cells) of the current schedule."""
        w, t, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _lib.check(self.lib.pbe_batch_get_schedule(self.h, ctypes.byref(w), ctypes.byref(t), ctypes.byref(c)))
        return w.value, t.value, c.value

    def autotune(self, t_out) -> int:
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        w = ctypes.c_int()
        _lib.check(self.lib.pbe_batch_autotune(self.h, t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                               len(t_out), ctypes.byref(w)))
        return w.value

    def solve(self, t_out, out=None):
        """Returns (rows[count, n_out, 6], total_steps)."""
        t_out = np.ascontiguousarray(t_out, dtype=np.float64)
        if out is None:
            out = np.zeros((self.count, len(t_out), 6))
        p, mem, keep = _buf(out, writable=True)
        steps = ctypes.c_int64()
        _lib.check(self.lib.pbe_batch_solve(self.h, t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                            len(t_out), p, mem, ctypes.byref(steps)))
        return out, steps.value
