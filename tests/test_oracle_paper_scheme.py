"""Pins of the oracle's paper-faithful variant: Eq. 3 (one-step high-resolution
update, van Leer limiter) with Godunov dimensional splitting and the CFL step
of SI Sec. S1.1, Arrhenius growth and exponential solubility (Appendix A), and
the base case of Table 1."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import mom
import pbe_inputs as pi


def _line_problem(N, lmax, G, cfl):
    return pi.Problem(ndim=1, ncells=(N,), lmax=(lmax,), kg=(G, 0.0), kb=0.0, cfl=cfl, fixed_kinetics=True,
                      scheme=1)


def test_courant_one_is_an_exact_shift():
    """At nu = 1 the (1 - nu) factor of Eq. 3 removes the limiter term and the
    update is f_i <- f_{i-1}: an exact one-cell shift."""
    p = _line_problem(125, 1000.0, 0.5, 1.0)     # dL = 8, dt = 16, nu = 1 exactly
    rng = np.random.default_rng(0)
    n = rng.uniform(0, 1, 125)
    n[-10:] = 0.0
    out, info = oracle.step(p, n, 0.2, 0.0, 1e9)
    assert info["dt"] == 16.0
    assert out[0] == 0.0 and np.array_equal(out[1:], n[:-1])


def test_closed_forms_of_appendix_a():
    p = pi.paper_base_case(60).problem
    cs = 3.37 * math.exp(0.036 * 15.0)
    s = 8.0 / cs - 1.0
    G1 = 8.86e6 / 60.0 * math.exp(-2450.0 / 288.15) * s ** 3.7
    G2 = 4.088e5 / 60.0 * math.exp(-2400.0 / 288.15) * s ** 2.5
    got = oracle.kinetics(p, 8.0, 100.0)
    assert got[0] == pytest.approx(G1, rel=1e-13) and got[1] == pytest.approx(G2, rel=1e-13) and got[2] == 0.0
    assert oracle.kinetics(p, cs, 0.0) == (0.0, 0.0, 0.0)
    # CFL step of SI Sec. S1.1: nu min(dL1/G1, dL2/G2)
    dt, _, _ = oracle.timestep(p, G1, G2, 0.0, 1e9)
    d1, d2 = 1200.0 / 60, 600.0 / 30
    assert dt == pytest.approx(0.9 * min(d1 / G1, d2 / G2), rel=1e-15)


def _cell_avg_tanh_front(x_edges, c, w):
    def prim(L):
        z = (L - c) / w
        return 0.5 * (L + w * (np.abs(z) + np.log1p(np.exp(-2 * np.abs(z))) - math.log(2.0)))
    return (prim(x_edges[1:]) - prim(x_edges[:-1])) / np.diff(x_edges)


def test_translation_second_order():
    errs = []
    for N in (200, 400, 800, 1600):
        p = _line_problem(N, 1000.0, 0.5, 0.5)
        edges = np.linspace(0.0, 1000.0, N + 1)
        prof = lambda s: _cell_avg_tanh_front(edges, 300.0 + s, 25.0) - _cell_avg_tanh_front(edges, 600.0 + s, 25.0)
        r = oracle.solve(p, prof(0.0), 0.2, 0.0, np.array([200.0]))
        mask = (edges[:-1] > 100.0) & (edges[1:] < 800.0)
        errs.append(np.sum(np.abs(r["n"] - prof(100.0))[mask]) * 1000.0 / N)
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order >= 1.8), (errs, order)


def test_tvd_and_positivity_up_to_courant_one():
    rng = np.random.default_rng(3)
    n0 = np.clip(rng.standard_normal(150).cumsum(), 0, None) + (rng.uniform(size=150) > 0.8) * 5
    n0[-25:] = 0.0
    for cfl in (0.3, 0.9, 1.0):
        p = _line_problem(150, 600.0, 0.37, cfl)
        n, t = n0.copy(), 0.0
        tv = lambda v: np.sum(np.abs(np.diff(np.concatenate([[0.0], v, [0.0]]))))
        for _ in range(30):
            tv0 = tv(n)
            n, info = oracle.step(p, n, 0.2, t, 1e9)
            t = info["t"]
            assert tv(n) <= tv0 * (1 + 1e-14)
            assert n.min() >= -1e-15 * n.max()


def test_split_reduces_to_1d_per_direction():
    N1, N2 = 40, 30
    u = pi.gaussian_seed_1d(N1, 500.0, 150.0, 30.0, 1.0)
    v = pi.gaussian_seed_1d(N2, 500.0, 200.0, 40.0, 1.0)
    for kg, (Nd, vec, other) in (((0.5, 0.0), (N1, u, v)), ((0.0, 0.5), (N2, v, u))):
        p2 = pi.Problem(ndim=2, ncells=(N1, N2), lmax=(500.0, 500.0), kg=kg, kb=0.0, cfl=0.9,
                        fixed_kinetics=True, scheme=1)
        p1 = _line_problem(Nd, 500.0, 0.5, 0.9)
        r2 = oracle.solve(p2, np.outer(u, v), 0.2, 0.0, np.array([150.0]))
        r1 = oracle.solve(p1, vec, 0.2, 0.0, np.array([150.0]))
        want = np.outer(r1["n"], other) if kg[0] > 0 else np.outer(other, r1["n"])
        assert np.max(np.abs(r2["n"] - want)) <= 1e-14 * want.max()


def test_base_case_conserves_mass_and_follows_moments():
    """Table 1 base case on coarse grids: solute + crystal mass conserved to
    rounding; crystal volume and concentration approach the method of moments
    (Sec. 3.1 verification) as the bins shrink."""
    errs = []
    for N in (120, 240, 480):
        inst = pi.paper_base_case(N, every=600.0)
        p = inst.problem
        r = oracle.solve_instance(inst)
        tot = r["rows"][:, 11] + p.kappa * r["rows"][:, 9]
        assert np.max(np.abs(tot - tot[0])) <= 1e-12 * tot[0]
        ref = mom.solve(dataclasses.replace(p), r["rows"][0, 1:-1], inst.C0, 0.0, inst.t_out, (0.0, 0.0), dt_max=0.5)
        errs.append(np.max(np.abs(r["rows"][:, [9, 11]] - ref[:, [9, 11]]) / np.abs(ref[:, [9, 11]])))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-2, errs


def test_step_count_consistent_with_the_paper():
    """The paper reports 1339 time steps for 6000 x 3000 bins.  Steps are
    CFL-limited, so they scale with 1/dL: 5x the count on 1200 x 600 bins."""
    r = oracle.solve_instance(pi.paper_base_case(1200))
    assert abs(5 * r["steps"] - 1339) <= 0.03 * 1339, r["steps"]
