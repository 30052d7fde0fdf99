"""pbe_solve_1d_noalloc, the entry point for callers that cannot allocate
memory while running (fixed-budget real-time loops, host frameworks whose
allocator owns all device memory).  It must give the same results as the
grid-based pbe_solve (plain path) on consecutive calls, which share the
library's fixed working array.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import pbe_inputs as pi
from gpu_helpers import REL_N, REL_ROWS

pytestmark = pytest.mark.gpu


def _noalloc_solve(lib, kin, inst, n_dev, rows_dev, torch):
    from paper_2411_00742_gb300 import _lib
    t_out = np.ascontiguousarray(inst.t_out, dtype=np.float64)
    steps = ctypes.c_int64()
    st = lib.pbe_solve_1d_noalloc(ctypes.byref(kin), inst.problem.ncells[0], float(inst.problem.lmax[0]),
                                  ctypes.c_void_p(n_dev.data_ptr()), float(inst.C0), float(inst.t0),
                                  t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t_out),
                                  ctypes.c_void_p(rows_dev.data_ptr()), ctypes.byref(steps),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(st)
    return steps.value


@pytest.mark.parametrize("N", [200, 4097])
def test_noalloc_matches_grid_solve_twice(N):
    import torch
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    lib = _lib.load()
    inst = pi.config_1d(N)
    # reference: the grid-based entry point
    g = P.Grid.from_problem(inst.problem, path="plain")
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
    want_rows, want_steps = g.solve(inst.t_out)
    want_n, want_C, _ = g.get_state()
    g.close()
    kin = P.kinetics_struct(inst.problem)
    for call in range(2):
        n_dev = torch.as_tensor(inst.n0).cuda()
        rows_dev = torch.full((len(inst.t_out), 6), float("nan"), dtype=torch.float64, device="cuda")
        steps = _noalloc_solve(lib, kin, inst, n_dev, rows_dev, torch)
        rows = rows_dev.cpu().numpy()
        n = n_dev.cpu().numpy()
        assert steps == want_steps, (call, steps, want_steps)
        np.testing.assert_allclose(rows[:, 0], want_rows[:, 0], rtol=1e-12)
        err = np.abs(rows[:, 1:] - want_rows[:, 1:])
        assert np.all(err <= REL_ROWS * np.abs(want_rows[:, 1:])), (call, err.max())
        assert np.max(np.abs(n - want_n)) <= REL_N * np.max(np.abs(want_n)), call


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    lib = _lib.load()
    inst = pi.config_1d(200)
    kin = P.kinetics_struct(inst.problem)
    n_dev = torch.zeros(65537, dtype=torch.float64, device="cuda")
    rows = torch.zeros((61, 6), dtype=torch.float64, device="cuda")
    t_out = np.ascontiguousarray(inst.t_out)
    st = lib.pbe_solve_1d_noalloc(ctypes.byref(kin), 65537, 1000.0, ctypes.c_void_p(n_dev.data_ptr()), 0.252, 0.0,
                                  t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 61,
                                  ctypes.c_void_p(rows.data_ptr()), None, None)
    assert st == _lib.PBE_EINVAL
    assert b"65536" in lib.pbe_last_error()


def _call(lib, kin, N, n_dev, t_out, rows, C0=0.252, t0=0.0):
    return lib.pbe_solve_1d_noalloc(ctypes.byref(kin), N, 1000.0, ctypes.c_void_p(n_dev.data_ptr()), C0, t0,
                                    t_out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(t_out),
                                    ctypes.c_void_p(rows.data_ptr()), None, None)


def test_noalloc_rejects_bad_kinetics_and_too_many_outputs():
    """The same value checks as pbe_set_kinetics (a NaN end temperature, a
    negative growth prefactor), and the 4096-row limit of the working array."""
    import torch
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    lib = _lib.load()
    inst = pi.config_1d(200)
    n_dev = torch.as_tensor(inst.n0).cuda()
    rows = torch.zeros((4097, 6), dtype=torch.float64, device="cuda")
    t_out = np.ascontiguousarray(inst.t_out)
    kin = P.kinetics_struct(inst.problem)
    kin.T1 = float("nan")
    assert _call(lib, kin, 200, n_dev, t_out, rows) == _lib.PBE_EINVAL
    kin = P.kinetics_struct(inst.problem)
    kin.kg[0] = -0.05
    assert _call(lib, kin, 200, n_dev, t_out, rows) == _lib.PBE_EINVAL
    assert b"negative" in lib.pbe_last_error()
    kin = P.kinetics_struct(inst.problem)
    many = np.linspace(0.0, 3600.0, 4097)
    assert _call(lib, kin, 200, n_dev, many, rows) == _lib.PBE_EINVAL
    assert b"4096" in lib.pbe_last_error()
    # the input distribution is untouched by rejected calls
    assert np.array_equal(n_dev.cpu().numpy(), inst.n0)


def test_noalloc_row_at_start_time_and_nonfinite_state():
    """A first output time equal to t0 gives the moments of n0 and C0 (no
    step); a NaN in n0 ends the call with PBE_ENONFINITE."""
    import torch
    import oracle
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    lib = _lib.load()
    inst = pi.config_1d(200)
    kin = P.kinetics_struct(inst.problem)
    t_out = np.ascontiguousarray([0.0, 60.0])
    n_dev = torch.as_tensor(inst.n0).cuda()
    rows = torch.zeros((2, 6), dtype=torch.float64, device="cuda")
    assert _call(lib, kin, 200, n_dev, t_out, rows, C0=inst.C0, t0=0.0) == _lib.PBE_OK
    r0 = rows.cpu().numpy()[0]
    assert r0[0] == 0.0 and r0[5] == inst.C0
    np.testing.assert_allclose(r0[1:5], oracle.moments(inst.problem, inst.n0), rtol=1e-13)
    bad = inst.n0.copy()
    bad[37] = float("nan")
    n_bad = torch.as_tensor(bad).cuda()
    assert _call(lib, kin, 200, n_bad, t_out, rows, C0=inst.C0, t0=0.0) == _lib.PBE_ENONFINITE
