"""Pins of the oracle's polynomial growth law (Eq. 6, the growth model of the
parameter-estimation study of Sec. 4.1: G_m = a_m1 (S-1) + ... + a_mK (S-1)^K)
and of its hand-written adjoint, which gives the gradient with respect to all
K coefficients in one reverse pass (the paper's AD), against the power law it
reduces to, an independent polynomial evaluation, complex-step derivatives of
the same forward arithmetic, and forward differences (the paper's ND)."""
import dataclasses

import numpy as np
import pytest

import oracle
import pbe_inputs as pi


def _with_poly(p, coeffs):
    return dataclasses.replace(p, growth_form=2, poly=tuple(float(c) for c in coeffs))


@pytest.mark.parametrize("ndim", [1, 2])
def test_one_and_two_terms_reduce_to_the_power_law(ndim):
    # a = (kg) is the power law with g = 1; a = (0, kg) the power law with g = 2:
    # both evaluate to the same IEEE products, so the solves agree bit for bit
    inst = pi.config_1d(150) if ndim == 1 else pi.config_2d(24, 20)
    p = inst.problem
    for g, coeffs in ((1.0, lambda kg: [kg]), (2.0, lambda kg: [0.0, kg])):
        pw = dataclasses.replace(p, g=(g, g))
        a = [c for m in range(ndim) for c in coeffs(p.kg[m])]
        want = oracle.solve(pw, inst.n0, inst.C0, 0.0, inst.t_out)
        got = oracle.solve(_with_poly(p, a), inst.n0, inst.C0, 0.0, inst.t_out)
        assert got["steps"] == want["steps"]
        np.testing.assert_array_equal(got["rows"], want["rows"])
        np.testing.assert_array_equal(got["n"], want["n"])


def test_kinetics_against_numpy_polyval():
    p = pi.poly_growth(pi.config_2d(8).problem, K=7)
    a = np.array(p.poly).reshape(2, 7)
    for T_frac, S in ((0.0, 1.3), (0.4, 1.05), (0.9, 1.8), (0.5, 1.0), (0.2, 0.7)):
        t = T_frac * p.t_cool
        T = p.T0 + (p.T1 - p.T0) * T_frac
        C = S * pi.csat_at(T)
        G1, G2, B = oracle.kinetics(p, C, t)
        s = C / pi.csat_at(T) - 1.0
        if s <= 0.0:
            assert (G1, G2, B) == (0.0, 0.0, 0.0)
            continue
        for m, G in ((0, G1), (1, G2)):
            want = np.polynomial.polynomial.polyval(s, np.concatenate([[0.0], a[m]]))
            assert G == pytest.approx(want, rel=1e-14)
        assert B == pytest.approx(p.kb * s ** p.b, rel=1e-13)


def _loss_setup(inst, K):
    """Polynomial model fitted against the power-law data of the same problem
    (the paper fits Eq. 6 to data made with another growth law)."""
    p0 = inst.problem
    inst.t_out = pi.loss_times()
    tgt = oracle.solve(p0, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    cols = [1, 2, 3, 4, 5] if p0.ndim == 1 else [1, 2, 3, 9, 11]
    p = pi.poly_growth(p0, K)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    return p, tgt, cols, seeds


CASES = {"1d": lambda: pi.config_1d(200), "1d_cfl_steps": lambda: pi.config_1d(800),
         "2d": lambda: pi.config_2d(32, 28)}


@pytest.mark.parametrize("case,K", [("1d", 6), ("1d_cfl_steps", 6), ("2d", 4)])
def test_adjoint_matches_complex_step(case, K):
    inst = CASES[case]()
    p, tgt, cols, seeds = _loss_setup(inst, K)
    if case == "1d_cfl_steps":   # most steps CFL-limited: dt depends on G and so on every a_mk
        assert oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["steps"] >= 2 * len(inst.t_out)
    dth, _, _, da = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    assert da.shape == (p.ndim * K,)
    assert dth[0] == dth[1] == dth[2] == dth[3] == 0.0   # the power-law growth entries
    assert np.any(da != 0.0)
    for j in range(p.ndim * K):
        _, dr = oracle.solve_cs(p, 6 + j, inst.n0, inst.C0, 0.0, inst.t_out)
        want = float(np.sum(seeds * dr))
        assert da[j] == pytest.approx(want, rel=1e-10, abs=1e-300), j
    for j in (4, 5):   # nucleation parameters keep their power-law derivatives
        _, dr = oracle.solve_cs(p, j, inst.n0, inst.C0, 0.0, inst.t_out)
        assert dth[j] == pytest.approx(float(np.sum(seeds * dr)), rel=1e-10)


def test_adjoint_matches_forward_differences():
    """The paper's ND: one extra solve per coefficient, forward difference with a
    relative step of 1e-7; agrees with the one-pass adjoint to the difference's
    truncation and rounding error."""
    inst = pi.config_1d(200)
    K = 5
    p, tgt, cols, seeds = _loss_setup(inst, K)
    _, _, _, da = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    L0 = oracle.relative_loss(oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"], tgt, cols)
    a = np.array(p.poly)
    for j in range(K):
        h = 1e-7 * a[j]
        ap = a.copy()
        ap[j] += h
        Lp = oracle.relative_loss(oracle.solve(_with_poly(p, ap), inst.n0, inst.C0, 0.0, inst.t_out)["rows"],
                                  tgt, cols)
        fd = (Lp - L0) / h
        assert fd == pytest.approx(da[j], rel=1e-4, abs=1e-4 * np.max(np.abs(da))), j


def test_thousand_coefficients_in_one_pass():
    """1000 parameters (500 per direction of a 2-D grid), the largest case of the
    AD-vs-ND study: one adjoint pass gives every coefficient's derivative;
    sampled coefficients, low and high order, match complex-step derivatives."""
    inst = pi.config_2d(12, 10)
    K = 500
    p, tgt, cols, seeds = _loss_setup(inst, K)
    dth, _, _, da = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    assert da.shape == (1000,) and np.all(np.isfinite(da))
    for j in (0, 1, 2, 40, 499, 500, 501, 999):
        _, dr = oracle.solve_cs(p, 6 + j, inst.n0, inst.C0, 0.0, inst.t_out)
        want = float(np.sum(seeds * dr))
        assert da[j] == pytest.approx(want, rel=1e-10, abs=1e-300), j
