"""Pins of the oracle's learned-closure kinetics and its adjoint."""
import math

import numpy as np
import pytest

import oracle
import pbe_closure_data as cd
import pbe_inputs as pi


def test_zero_network_gives_the_reference_rates():
    p = pi.config_2d(16).problem
    w = np.zeros(oracle.MLP_NW)
    C = 1.3 * 0.168   # S = 1.3 at 20 C (t >= 3600)
    G1, G2, B = oracle.kinetics_mlp(p, w, C, 4000.0, 3.7e5)
    assert G1 == pytest.approx(0.01, rel=1e-15)
    assert G2 == pytest.approx(0.005, rel=1e-15)
    assert B == pytest.approx(1e5, rel=1e-15)
    assert oracle.kinetics_mlp(p, w, 0.168, 4000.0, 3.7e5) == (0.0, 0.0, 0.0)   # S = 1: gate


def test_single_hidden_unit_closed_form():
    """One active path through the network: o2 = W3[2][0] silu(W2[0][0] silu(W1[0][0] x0))."""
    p = pi.config_1d(16).problem
    H = 64
    w = np.zeros(oracle.MLP_NW)
    w[0] = 0.7                           # W1[0][0]
    w[H * 3 + H] = -1.3                  # W2[0][0]
    w[H * 3 + 2 * H + H * H + 2 * H] = 0.45   # W3[2][0]
    silu = lambda z: z / (1 + math.exp(-z))
    S = 1.2
    C = S * 0.168
    x0 = 4 * (S - 1)
    o2 = 0.45 * silu(-1.3 * silu(0.7 * x0)) + 0.0
    # W2 row 0 reads a1[0]; hidden unit 0 of layer 2 feeds W3[2][0]; other units see silu(0) = 0
    G1, G2, B = oracle.kinetics_mlp(p, w, C, 4000.0, 1e6)
    assert B == pytest.approx(1e5 * math.exp(o2), rel=1e-14)
    assert G1 == pytest.approx(0.01, rel=1e-15) and G2 == 0.0


@pytest.mark.parametrize("ndim", [1, 2])
def test_closure_adjoint_matches_complex_step(ndim):
    inst = pi.config_1d(120) if ndim == 1 else cd.trajectories(1, seed=5, N=20)[0]
    inst.t_out = pi.loss_times()[:25]
    w = cd.stored_weights(cd.initial_weights(9, 0.2))
    rng = np.random.default_rng(2)
    r = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)["rows"]
    seeds = rng.standard_normal(r.shape) / (np.abs(r) + 1.0)
    seeds[:, 0] = 0.0
    _, dn0, dC0, dW = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=w)
    H = 64
    for k in (0, 5, H * 3 + 7, H * 3 + H + 100, H * 3 + H + H * H + 3, oracle.MLP_NW - 2, oracle.MLP_NW - 1):
        _, dr = oracle.solve_cs(inst.problem, 6 + k, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
        assert dW[k] == pytest.approx(float(np.sum(seeds * dr)), rel=1e-10, abs=1e-14 * np.max(np.abs(dW))), k


def _x0_along(problem, rows):
    """Closure input x0 = 4 (S - 1) at the output rows (t, ..., C)."""
    T = np.array([oracle.temperature(problem, t) for t in rows[:, 0]])
    cs = problem.csat[0] + problem.csat[1] * T + problem.csat[2] * T * T
    return 4.0 * (rows[:, -1] / cs - 1.0)


@pytest.mark.parametrize("ndim", [1, 2])
def test_closure_fallback_box_limits(ndim):
    """A training box that no input reaches makes the closure solve the power-law
    solve bit for bit (every rate from the fallback); a box holding every input
    leaves the closure solve unchanged bit for bit."""
    import dataclasses
    inst = pi.config_1d(120) if ndim == 1 else cd.trajectories(1, seed=5, N=20)[0]
    w = cd.stored_weights(cd.initial_weights(9, 0.2))
    p = inst.problem
    plain = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)
    closure = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
    assert not np.array_equal(plain["rows"], closure["rows"])
    none = dataclasses.replace(p, mlp_box=((50.0, 50.0, 50.0), (60.0, 60.0, 60.0)))
    allin = dataclasses.replace(p, mlp_box=((-1e300, -1e300, -1e300), (1e300, 1e300, 1e300)))
    got = oracle.solve(none, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
    np.testing.assert_array_equal(got["rows"], plain["rows"])
    np.testing.assert_array_equal(got["n"], plain["n"])
    got = oracle.solve(allin, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
    np.testing.assert_array_equal(got["rows"], closure["rows"])


def test_closure_nonfinite_rate_falls_back_to_the_power_law():
    """A network whose nucleation output overflows exp() gives the power-law
    rates at that state, not an infinite rate."""
    p = pi.config_2d(16).problem
    w = np.zeros(oracle.MLP_NW)
    w[-1] = 800.0     # b3[2]: ln B = 800 + ln 1e5 overflows
    C, t = 1.3 * 0.168, 4000.0
    got = oracle.kinetics_mlp(p, w, C, t, 3.7e5)
    want = oracle.kinetics(p, C, t)
    assert got == want and all(math.isfinite(v) for v in got)


@pytest.mark.parametrize("ndim", [1, 2])
def test_closure_adjoint_with_partial_fallback_matches_complex_step(ndim):
    """A box that cuts the supersaturation input at its median value: the
    stages above it take the power law, the rest the network.  The adjoint
    differentiates whichever the forward pass took: the kinetic parameters'
    derivatives (from the fallback stages) and the weights' (from the network
    stages) against complex-step derivatives."""
    import dataclasses
    inst = pi.config_1d(120) if ndim == 1 else cd.trajectories(1, seed=5, N=20)[0]
    inst.t_out = pi.loss_times()[:25]
    w = cd.stored_weights(cd.initial_weights(9, 0.2))
    r0 = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)["rows"]
    x0 = _x0_along(inst.problem, r0)
    cut = float(np.median(x0[x0 > 0]))
    p = dataclasses.replace(inst.problem, mlp_box=((-10.0, -10.0, -10.0), (cut, 10.0, 10.0)))
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)["rows"]
    assert not np.array_equal(r, r0)
    rng = np.random.default_rng(3)
    seeds = rng.standard_normal(r.shape) / (np.abs(r) + 1.0)
    seeds[:, 0] = 0.0
    dth, _, _, dW = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=w)
    for j in ((0, 1, 4, 5) if ndim == 1 else range(6)):
        _, dr = oracle.solve_cs(p, j, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
        assert dth[j] == pytest.approx(float(np.sum(seeds * dr)), rel=1e-10), j
    assert np.any(dth != 0.0)
    H = 64
    for k in (0, 5, H * 3 + 7, H * 3 + H + 100, oracle.MLP_NW - 1):
        _, dr = oracle.solve_cs(p, 6 + k, inst.n0, inst.C0, 0.0, inst.t_out, mlp=w)
        assert dW[k] == pytest.approx(float(np.sum(seeds * dr)), rel=1e-10, abs=1e-14 * np.max(np.abs(dW))), k
