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
