"""Parity of the plain FP64 CUDA path with the CPU oracle.

Moments mu and concentration C within 1e-10 relative at every output time,
the distribution within 1e-9 * max(n) in L-inf, the same step count."""
import dataclasses

import numpy as np
import pytest

import oracle
import pbe_inputs as pi
from gpu_helpers import REL_ROWS, assert_n_close, assert_rows_close, compare_instance, gpu_solve

pytestmark = pytest.mark.gpu


def test_1d_config_every_output_time():
    compare_instance(pi.config_1d(200))


def test_1d_config_host_buffers():
    compare_instance(pi.config_1d(200), device_buffers=False)


@pytest.mark.parametrize("N", [1, 2, 3, 5, 101, 1023, 1024, 1025, 1999, 2000, 5000])
def test_1d_ragged_sizes(N):
    compare_instance(pi.config_1d(N))


@pytest.mark.parametrize("shape", [(1, 1), (1, 17), (23, 1), (16, 32), (37, 53), (64, 64), (100, 33)])
def test_2d_ragged_sizes(shape):
    compare_instance(pi.config_2d(*shape))


def test_2d_config_full_size():
    compare_instance(pi.config_2d(256))


def _state_at_every_output(inst):
    import paper_2411_00742_gb300 as P
    g = P.Grid.from_problem(inst.problem)
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
    n, C, t = np.array(inst.n0), inst.C0, inst.t0
    for tk in inst.t_out[1:]:
        rows, _ = g.solve([tk])
        ng, Cg, tg = g.get_state()
        r = oracle.solve(inst.problem, n, C, t, [tk])
        n, C, t = r["n"], r["C"], r["t"]
        assert tg == pytest.approx(t, rel=1e-12)
        assert_n_close(ng, n)
        assert abs(Cg - C) <= REL_ROWS * abs(C)
        assert_rows_close(rows, r["rows"])
    g.close()


def test_1d_state_at_every_output_time():
    _state_at_every_output(pi.config_1d(200))


def test_2d_state_at_every_output_time():
    _state_at_every_output(pi.config_2d(48, 40))


@pytest.mark.parametrize("ndim", [1, 2])
def test_single_step_matches_oracle(ndim):
    import paper_2411_00742_gb300 as P
    inst = pi.config_1d(300) if ndim == 1 else pi.config_2d(40, 24)
    g = P.Grid.from_problem(inst.problem)
    n, C, t = np.array(inst.n0), inst.C0, 0.0
    g.set_state(n, C, t)
    for t_lim in [60.0, 120.0, 1000.0, 1500.0, 4000.0]:
        dt = g.step(t_lim)
        n, info = oracle.step(inst.problem, n, C, t, t_lim)
        C, t = info["C"], info["t"]
        ng, Cg, tg = g.get_state()
        assert dt == pytest.approx(info["dt"], rel=1e-12)
        assert tg == pytest.approx(t, rel=1e-12)
        assert_n_close(ng, n)
        assert abs(Cg - C) <= REL_ROWS * abs(C)
    g.close()


def test_moments_readout():
    import paper_2411_00742_gb300 as P
    for inst in (pi.config_1d(777), pi.config_2d(33, 65)):
        g = P.Grid.from_problem(inst.problem)
        g.set_state(inst.n0, inst.C0, 0.0)
        mu = g.moments()
        want = oracle.moments(inst.problem, inst.n0)
        np.testing.assert_allclose(mu, want, rtol=1e-12)
        g.close()


def test_deterministic_bitwise():
    a = gpu_solve(pi.config_2d(96))
    b = gpu_solve(pi.config_2d(96))
    assert np.array_equal(a["rows"], b["rows"]) and np.array_equal(a["n"], b["n"])


def test_fixed_growth_translation():
    p = pi.Problem(ndim=1, ncells=(800,), lmax=(1000.0,), kg=(0.5, 0.0), kb=0.0, cfl=0.45,
                   fixed_kinetics=True)
    n0 = pi.gaussian_seed_1d(800, 1000.0, 300.0, 30.0, 1e6)
    compare_instance(pi.Instance(p, n0, 0.2, 0.0, np.array([0.0, 100.0, 400.0])))
    p2 = pi.Problem(ndim=2, ncells=(70, 90), lmax=(500.0, 500.0), kg=(0.3, 0.2), kb=5.0, cfl=0.4,
                    fixed_kinetics=True)
    n2 = pi.gaussian_seed_2d(70, 90, 500.0, 500.0, (150.0, 100.0), (20.0, 15.0), -0.4, 1e6)
    compare_instance(pi.Instance(p2, n2, 0.2, 0.0, np.array([50.0, 300.0])))


def test_empty_seed_nucleation_only():
    inst = pi.config_1d(200)
    inst.n0 = np.zeros(200)
    compare_instance(inst)
    inst2 = pi.config_2d(40)
    inst2.n0 = np.zeros((40, 40))
    compare_instance(inst2)


def test_no_supersaturation_no_change():
    inst = pi.config_1d(200)
    p = dataclasses.replace(inst.problem, T1=40.0)   # S stays 1: nothing happens
    inst = pi.Instance(p, inst.n0, inst.C0, 0.0, inst.t_out)
    got, _ = compare_instance(inst)
    # unchanged up to the halving of odd subnormals in the tail (n/2 + n/2)
    np.testing.assert_allclose(got["n"], inst.n0, rtol=0, atol=1e-300)
    assert got["rows"][-1, 5] == inst.C0


def test_nonfinite_state_reported():
    import paper_2411_00742_gb300 as P
    inst = pi.config_1d(200)
    g = P.Grid.from_problem(inst.problem)
    n = inst.n0.copy()
    n[50] = np.nan
    g.set_state(n, inst.C0, 0.0)
    with pytest.raises(P.PbeError) as e:
        g.solve(inst.t_out)
    assert e.value.status == 4
    g.close()


def test_step_budget_reported():
    import paper_2411_00742_gb300 as P
    inst = pi.config_1d(200)
    g = P.Grid.from_problem(inst.problem)
    g.set_max_steps(3)
    g.set_state(inst.n0, inst.C0, 0.0)
    with pytest.raises(P.PbeError) as e:
        g.solve(inst.t_out)
    assert e.value.status == 5
    _, _, t = g.get_state()
    assert t == pytest.approx(180.0)
    g.close()


def test_bad_output_times_rejected():
    import paper_2411_00742_gb300 as P
    inst = pi.config_1d(50)
    g = P.Grid.from_problem(inst.problem)
    g.set_state(inst.n0, inst.C0, 100.0)
    with pytest.raises(P.PbeError):
        g.solve([50.0, 200.0])
    with pytest.raises(P.PbeError):
        g.solve([200.0, 150.0])
    g.close()


def test_init_seed_gaussian_matches_the_input_generator():
    """pbe_init_seed_gaussian / _mass reproduce the seeded inputs (normal
    seed at cell centres, scaled by number or by seed mass)."""
    import paper_2411_00742_gb300 as P
    i1 = pi.config_1d(200)
    g = P.Grid.from_problem(i1.problem)
    g.init_seed_gaussian([150.0], [20.0], total_number=1e8, C0=i1.C0)
    n, C, t = g.get_state()
    g.close()
    np.testing.assert_allclose(n, i1.n0, rtol=1e-13, atol=1e-13 * i1.n0.max())
    assert C == i1.C0 and t == 0.0
    i2 = pi.config_2d(48, 40)
    g = P.Grid.from_problem(i2.problem)
    g.init_seed_gaussian([100.0, 60.0], [15.0, 10.0], corr=0.3, total_number=1e8, C0=i2.C0)
    n, _, _ = g.get_state()
    g.close()
    np.testing.assert_allclose(n, i2.n0, rtol=1e-13, atol=1e-13 * i2.n0.max())
    # the paper's base case: seed scaled by its mass (1 g)
    i3 = pi.paper_base_case(120)
    g = P.Grid.from_problem(i3.problem)
    g.init_seed_gaussian([400.0, 250.0], [30.0, 30.0], seed_mass=1.0, rho_kv=pi.RHO_C * pi.KV, C0=8.0)
    n, _, _ = g.get_state()
    g.close()
    np.testing.assert_allclose(n, i3.n0, rtol=1e-13, atol=1e-13 * i3.n0.max())


def test_init_seed_gaussian_rejects_bad_arguments():
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300._lib import PbeError
    inst = pi.config_2d(16)
    g = P.Grid.from_problem(inst.problem)
    for kw in (dict(sd=[0.0, 10.0]), dict(corr=1.0), dict(total_number=-1.0), dict(mean=[1e9, 1e9])):
        args = dict(mean=[100.0, 60.0], sd=[15.0, 10.0], corr=0.3, total_number=1e8, C0=0.2)
        args.update(kw)
        with pytest.raises(PbeError):
            g.init_seed_gaussian(**args)
    g.close()


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_output_times_reused_and_changed(path):
    """Repeated solves on one grid: the same output times (kept on the device
    between calls), new times of the same length, a single step in between."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(40, 24)
    ta = np.array(inst.t_out[:7])
    tb = ta + 30.0
    tb[0] = 0.0
    g = P.Grid.from_problem(inst.problem, path=path)
    runs = []
    for t_out in (ta, ta, tb, None, ta):
        g.set_state(inst.n0, inst.C0, 0.0)
        if t_out is None:
            g.step(45.0)
            continue
        rows, _ = g.solve(t_out)
        runs.append((t_out, rows))
    g.close()
    for t_out, rows in runs:
        want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, t_out)
        assert_rows_close(rows, want["rows"])
    assert np.array_equal(runs[0][1], runs[1][1]) and np.array_equal(runs[0][1], runs[3][1])


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_kernel_timing(path):
    """pbe_set_timing / pbe_kernel_time: the recorded device time of the main
    launch is positive and below the wall time of the whole call."""
    import time

    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(64)
    g = P.Grid.from_problem(inst.problem, path=path)
    assert g.kernel_time_ms() == -1.0
    g.set_state(inst.n0, inst.C0, 0.0)
    g.solve(inst.t_out)
    assert g.kernel_time_ms() == -1.0       # timing off
    g.set_timing(True)
    g.set_state(inst.n0, inst.C0, 0.0)
    t0 = time.perf_counter()
    rows, _ = g.solve(inst.t_out)
    wall_ms = 1e3 * (time.perf_counter() - t0)
    ms = g.kernel_time_ms()
    assert 0.0 < ms < wall_ms
    g.set_timing(False)
    g.close()
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)
    assert_rows_close(rows, want["rows"])


@pytest.mark.parametrize("shape", [(1, 1), (3, 200), (37, 53), (64, 64), (100, 251), (129, 31)])
def test_2d_window_kernel_ragged_sizes(shape):
    """The register-window stage kernel (forced on small ragged grids: one block,
    columns and rows not multiples of its 125 x 32 block)."""
    inst = pi.config_2d(*shape)
    want = oracle.solve_instance(inst)
    import paper_2411_00742_gb300 as P
    g = P.Grid.from_problem(inst.problem)
    g.set_window(1)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    n, C, t = g.get_state()
    g.close()
    assert steps == want["steps"]
    assert_rows_close(rows, want["rows"])
    assert_n_close(n, want["n"])


def test_2d_window_kernel_chosen_on_large_grids():
    """A grid with more window blocks than SMs takes the window kernel by
    default (the same rows as forcing it); the tile kernel agrees to rounding.
    Three output times of the 1000 x 777 workload keep the oracle short."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(1000, 777)
    t_out = np.array(inst.t_out[:3])
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, t_out)
    out = {}
    for mode in (-1, 1, 0):
        g = P.Grid.from_problem(inst.problem)
        g.set_window(mode)
        g.set_state(inst.n0, inst.C0, 0.0)
        rows, _ = g.solve(t_out)
        n, _, _ = g.get_state()
        g.close()
        assert_rows_close(rows, want["rows"])
        assert_n_close(n, want["n"])
        out[mode] = rows
    assert np.array_equal(out[-1], out[1])


def test_2d_window_kernel_forty_row_blocks():
    """768 x 768: the window kernel takes 40-row blocks there (the block count
    that spreads best over the SMs); three output times against the oracle."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(768)
    t_out = np.array(inst.t_out[:3])
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, t_out)
    g = P.Grid.from_problem(inst.problem)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, _ = g.solve(t_out)
    n, _, _ = g.get_state()
    g.close()
    assert_rows_close(rows, want["rows"])
    assert_n_close(n, want["n"])


def test_window_mode_rejects_bad_values():
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(16)
    g = P.Grid.from_problem(inst.problem)
    with pytest.raises(P.PbeError):
        g.set_window(2)
    g.close()
