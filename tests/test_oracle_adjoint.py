"""Pins of the oracle's hand-written discrete adjoint (reverse mode through
the step, the parameter estimation gradient of Sec. 4.1) against independent
derivatives: complex-step differentiation of the same forward arithmetic
(exact to rounding, no cancellation) and central finite differences."""
import dataclasses

import numpy as np
import pytest

import oracle
import pbe_inputs as pi


def _setup(inst):
    p = inst.problem
    inst.t_out = pi.loss_times()
    tgt = oracle.solve(p.with_theta(p.theta * pi.TARGET_FACTOR), inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    cols = [1, 2, 3, 4, 5] if p.ndim == 1 else [1, 2, 3, 9, 11]
    return p, tgt, cols


def _loss(p, inst, tgt, cols, n0=None, C0=None):
    r = oracle.solve(p, inst.n0 if n0 is None else n0, inst.C0 if C0 is None else C0, 0.0, inst.t_out)["rows"]
    return oracle.relative_loss(r, tgt, cols), r


CASES = {
    "1d_clipped_steps": lambda: pi.config_1d(200),
    "1d_cfl_steps": lambda: pi.config_1d(800),
    "2d": lambda: pi.config_2d(40),
    "2d_anisotropic_rect": lambda: pi.config_2d(36, 52),
}


@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_matches_complex_step(case):
    inst = CASES[case]()
    p, tgt, cols = _setup(inst)
    L, r = _loss(p, inst, tgt, cols)
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    dth, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    for j in range(6):
        _, dr = oracle.solve_cs(p, j, inst.n0, inst.C0, 0.0, inst.t_out)
        want = float(np.sum(seeds * dr))
        assert dth[j] == pytest.approx(want, rel=1e-11, abs=1e-300), (case, j)
    if p.ndim == 1:
        assert dth[2] == 0.0 and dth[3] == 0.0


def test_complex_step_matches_central_differences():
    """Pins the complex-step instrument itself (independent of the adjoint)."""
    inst = pi.config_2d(32)
    p, tgt, cols = _setup(inst)
    th = p.theta
    for j in range(6):
        h = 1e-6 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        rp = oracle.solve(p.with_theta(tp), inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
        rm = oracle.solve(p.with_theta(tm), inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
        fd = (rp - rm) / (2 * h)
        _, dr = oracle.solve_cs(p, j, inst.n0, inst.C0, 0.0, inst.t_out)
        scale = np.max(np.abs(dr[:, 1:]), axis=0)
        noise = 8 * np.finfo(float).eps * np.max(np.abs(rp[:, 1:]), axis=0) / h   # rounding of the difference
        err = np.max(np.abs(fd[:, 1:] - dr[:, 1:]), axis=0)
        assert np.all(err <= 3e-5 * scale + noise), (j, err / scale)


@pytest.mark.parametrize("case", ["1d_cfl_steps", "2d"])
def test_adjoint_matches_central_differences(case):
    """The parameter gradient against central differences with h = 1e-6 relative
    (the forward branch sequence is the same for the +h and -h runs)."""
    inst = CASES[case]()
    p, tgt, cols = _setup(inst)
    L, r = _loss(p, inst, tgt, cols)
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    dth, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    th = p.theta
    idx = [0, 1, 4, 5] if p.ndim == 1 else range(6)
    for j in idx:
        h = 1e-6 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        sp = oracle.solve(p.with_theta(tp), inst.n0, inst.C0, 0.0, inst.t_out)
        sm = oracle.solve(p.with_theta(tm), inst.n0, inst.C0, 0.0, inst.t_out)
        assert sp["steps"] == sm["steps"]
        fd = (oracle.relative_loss(sp["rows"], tgt, cols) - oracle.relative_loss(sm["rows"], tgt, cols)) / (2 * h)
        assert dth[j] == pytest.approx(fd, rel=1e-6), (case, j)


def test_adjoint_initial_state_and_concentration():
    inst = pi.config_1d(400)
    p, tgt, cols = _setup(inst)
    L, r = _loss(p, inst, tgt, cols)
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    _, dn0, dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    x = (np.arange(400) + 0.5) * 2.5
    # smooth relative perturbations (zeros stay zero, so no limiter branch flips)
    for v in (inst.n0 * np.sin(x / 40.0), inst.n0 * (x / 1000.0), inst.n0):
        h = 1e-6
        Lp, _ = _loss(p, inst, tgt, cols, n0=inst.n0 + h * v)
        Lm, _ = _loss(p, inst, tgt, cols, n0=inst.n0 - h * v)
        assert np.dot(dn0, v) == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5)
    h = 1e-9
    Lp, _ = _loss(p, inst, tgt, cols, C0=inst.C0 + h)
    Lm, _ = _loss(p, inst, tgt, cols, C0=inst.C0 - h)
    assert dC0 == pytest.approx((Lp - Lm) / (2 * h), rel=1e-4)


def test_adjoint_fixed_kinetics_and_output_at_start():
    inst = pi.config_1d(300)
    p = dataclasses.replace(inst.problem, fixed_kinetics=True, kg=(0.2, 0.0), kb=30.0)
    t_out = np.array([0.0, 100.0, 700.0, 1500.0])
    rows = oracle.solve(p, inst.n0, inst.C0, 0.0, t_out)["rows"]
    rng = np.random.default_rng(1)
    seeds = rng.standard_normal(rows.shape) / np.abs(rows + 1.0)
    dth, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, t_out, seeds)
    for j in (0, 4):
        _, dr = oracle.solve_cs(p, j, inst.n0, inst.C0, 0.0, t_out)
        seeds_nt = seeds.copy()
        seeds_nt[:, 0] = 0.0
        assert dth[j] == pytest.approx(float(np.sum(seeds_nt * dr)), rel=1e-11)
