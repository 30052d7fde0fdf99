"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-computed
closed forms, the literal van Leer formula, exact rational arithmetic, exact
translation of the distribution, the method of moments and invariants of the
scheme.  No GPU is involved.
"""
import dataclasses
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle
from oracle import exact, mom
import pbe_inputs as pi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _golden():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                name, arg, val = line.split()
                rows.append((name, float(arg), float(val)))
    return rows


def test_closed_forms_from_golden():
    inst = pi.config_1d()
    p = inst.problem
    for name, arg, val in _golden():
        if name == "csat":
            # c* enters through S = C / c*: S = 1 exactly when C = c*(T)
            pT = dataclasses.replace(p, T0=arg, T1=arg)
            G = oracle.kinetics(pT, val * 1.5, 0.0)[0]
            assert G == pytest.approx(0.05 * 0.5 ** 1.5, rel=1e-13), (name, arg)
            assert oracle.kinetics(pT, val, 0.0) == (0.0, 0.0, 0.0)
        elif name == "temperature":
            assert oracle.temperature(p, arg) == pytest.approx(val, abs=1e-13)
        elif name == "phi":
            # psi(a, b) = phi(a/b) * b with b = 1
            assert oracle.psi(arg, 1.0) == pytest.approx(val, rel=1e-15, abs=1e-300)
        elif name == "growth_1d":
            C = arg * 0.252
            G, G2, B = oracle.kinetics(p, C, 0.0)
            assert G == pytest.approx(val, rel=1e-14)
            assert G2 == 0.0
        elif name == "nucleation_1d":
            C = arg * 0.252
            assert oracle.kinetics(p, C, 0.0)[2] == pytest.approx(val, rel=1e-12)


def test_kinetics_2d_and_gate():
    p = pi.config_2d(8).problem
    cs = 0.168  # c*(20), reached at t >= 3600
    G1, G2, B = oracle.kinetics(p, 1.25 * cs, 5000.0)
    assert G1 == pytest.approx(0.04 * 0.25 ** 1.3, rel=1e-13)
    assert G2 == pytest.approx(0.02 * 0.25 ** 1.8, rel=1e-13)
    assert B == pytest.approx(1e6 * 0.25 ** 2, rel=1e-13)
    # S <= 1: no growth, no nucleation, no dissolution
    assert oracle.kinetics(p, 0.9 * cs, 5000.0) == (0.0, 0.0, 0.0)
    assert oracle.kinetics(p, 0.252, 0.0) == (0.0, 0.0, 0.0)


def _phi_literal(theta):
    return (theta + abs(theta)) / (1.0 + abs(theta))


def test_limiter_matches_literal_van_leer():
    rng = np.random.default_rng(1)
    for _ in range(20000):
        a, b = rng.standard_normal(2) * 10.0 ** rng.uniform(-6, 6, 2)
        want = _phi_literal(a / b) * b
        got = oracle.psi(a, b)
        assert got == pytest.approx(want, rel=1e-13, abs=1e-300)
    # limits and symmetric special values
    assert oracle.psi(3.0, 0.0) == 0.0 and oracle.psi(-3.0, 0.0) == 0.0
    assert oracle.psi(0.0, 5.0) == 0.0
    assert oracle.psi(2.5, 2.5) == 2.5           # phi(1) = 1
    assert oracle.psi(-1.0, 2.0) == 0.0          # theta < 0
    assert oracle.psi(1e8, 1.0) == pytest.approx(2.0, rel=1e-7)   # phi -> 2
    assert oracle.psi(1e-300, 1e-300) == 1e-300  # no underflow in tails
    assert oracle.psi(2.0, 3.0) == pytest.approx(oracle.psi(3.0, 2.0), rel=1e-15)


def test_timestep_branches():
    p = pi.config_1d().problem   # dL = 5, nu = 0.5
    dt, tn, clipped = oracle.timestep(p, 0.01, 0.0, 100.0, 1000.0)
    assert dt == pytest.approx(250.0, rel=1e-15) and tn == pytest.approx(350.0) and not clipped
    dt, tn, clipped = oracle.timestep(p, 0.01, 0.0, 100.0, 200.0)
    assert dt == 100.0 and tn == 200.0 and clipped
    dt, tn, clipped = oracle.timestep(p, 0.0, 0.0, 100.0, 160.0)
    assert dt == 60.0 and tn == 160.0 and clipped
    p2 = pi.config_2d(250).problem  # dL = 2 in both directions, nu = 0.4
    dt, tn, clipped = oracle.timestep(p2, 0.02, 0.01, 0.0, 1e9)
    assert dt == pytest.approx(0.4 / (0.01 + 0.005), rel=1e-15) and not clipped


def test_rhs_uniform_only_first_cell_changes():
    p = dataclasses.replace(pi.config_1d(16).problem, fixed_kinetics=True)
    n = np.full(16, 3.0)
    L = oracle.rhs(p, n, 0.2, 0.0, 0.0)
    d = 1000.0 / 16
    assert L[0] == pytest.approx(-0.2 * 3.0 / d, rel=1e-15)
    assert np.all(L[1:] == 0.0)
    L = oracle.rhs(p, n, 0.0, 0.0, 7.0)
    assert L[0] == pytest.approx(7.0 / d, rel=1e-15) and np.all(L[1:] == 0.0)


def _rat(x):
    return Fr(x).limit_denominator(1 << 20)


@pytest.mark.parametrize("nsteps", [1, 2, 3])
def test_exact_rational_1d(nsteps):
    rng = np.random.default_rng(10 + nsteps)
    N = 8
    n_r = [_rat(v) for v in rng.uniform(0.0, 5.0, N)]
    n_r[3] = n_r[2]            # a zero difference (b = 0 face)
    n_r[6] = Fr(0)
    G, B = Fr(3, 7), Fr(5, 2)
    d = Fr(1000, N)
    nu = Fr(1, 2)
    p = dataclasses.replace(pi.config_1d(N).problem, fixed_kinetics=True, kg=(float(G), 0.0),
                            kb=float(B), cfl=0.5)
    n = np.array([float(v) for v in n_r])
    t_r, t = Fr(0), 0.0
    for k in range(nsteps):
        t_next = 200 if k < 2 else 1000
        n_r, dt_r, t_r = exact.step1(n_r, G, B, d, nu, t_r, Fr(t_next))
        n, info = oracle.step(p, n, 0.2, t, float(t_next))
        t = info["t"]
        assert info["dt"] == pytest.approx(float(dt_r), rel=1e-15)
        assert t == pytest.approx(float(t_r), rel=1e-15)
    want = np.array([float(v) for v in n_r])
    assert np.max(np.abs(n - want)) <= 1e-14 * np.max(np.abs(want))


def test_exact_rational_2d():
    rng = np.random.default_rng(7)
    N1, N2 = 6, 5
    n_r = [[_rat(v) for v in row] for row in rng.uniform(0.0, 4.0, (N1, N2))]
    n_r[2][1] = n_r[1][1]
    n_r[3][3] = n_r[3][2]
    G1, G2, B = Fr(2, 9), Fr(1, 13), Fr(3, 1)
    d1, d2 = Fr(500, N1), Fr(500, N2)
    nu = Fr(2, 5)
    p = dataclasses.replace(pi.config_2d(N1, N2).problem, fixed_kinetics=True,
                            kg=(float(G1), float(G2)), kb=float(B), cfl=0.4)
    n = np.array([[float(v) for v in row] for row in n_r])
    t_r, t = Fr(0), 0.0
    for k in range(2):
        n_r, dt_r, t_r = exact.step2(n_r, G1, G2, B, d1, d2, nu, t_r, Fr(5000))
        n, info = oracle.step(p, n, 0.2, t, 5000.0)
        t = info["t"]
        assert info["dt"] == pytest.approx(float(dt_r), rel=1e-15)
    want = np.array([[float(v) for v in row] for row in n_r])
    assert np.max(np.abs(n - want)) <= 1e-14 * np.max(np.abs(want))


def test_pure_nucleation_adds_B_dt_over_dL():
    N = 50
    p = dataclasses.replace(pi.config_1d(N).problem, fixed_kinetics=True, kg=(0.0, 0.0), kb=40.0)
    n0 = pi.gaussian_seed_1d(N, 1000.0, 400.0, 50.0, 1e6)
    n, info = oracle.step(p, n0, 0.2, 0.0, 30.0)
    d = 1000.0 / N
    assert info["dt"] == 30.0 and info["clipped"]
    assert n[0] - n0[0] == pytest.approx(40.0 * 30.0 / d, rel=1e-13)
    assert np.array_equal(n[1:], n0[1:])
    mu0 = oracle.moments(p, n)[0]
    assert mu0 - oracle.moments(p, n0)[0] == pytest.approx(40.0 * 30.0, rel=1e-9)


def test_number_conserved_without_nucleation():
    inst = pi.config_1d()
    p = dataclasses.replace(inst.problem, kb=0.0)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)
    mu0 = r["rows"][:, 1]
    assert np.max(np.abs(mu0 - 1e8)) <= 1e-12 * 1e8
    inst2 = pi.config_2d(64)
    p2 = dataclasses.replace(inst2.problem, kb=0.0)
    r2 = oracle.solve(p2, inst2.n0, inst2.C0, 0.0, inst2.t_out)
    assert np.max(np.abs(r2["rows"][:, 1] - 1e8)) <= 1e-12 * 1e8


def _cell_avg_tanh_front(x_edges, c, w):
    # n0(L) = (1 + tanh((L - c)/w)) / 2; integral = (L + w log cosh((L-c)/w)) / 2
    def prim(L):
        z = (L - c) / w
        return 0.5 * (L + w * (np.abs(z) + np.log1p(np.exp(-2 * np.abs(z))) - math.log(2.0)))
    return (prim(x_edges[1:]) - prim(x_edges[:-1])) / np.diff(x_edges)


def _cell_avg_gauss(x_edges, m, s):
    from scipy.special import erf
    prim = 0.5 * s * math.sqrt(2 * math.pi) * erf((x_edges - m) / (s * math.sqrt(2)))
    return np.diff(prim) / np.diff(x_edges)


def _translation_errors(profile, Ns, G=0.5, t_end=200.0):
    errs = []
    for N in Ns:
        p = pi.Problem(ndim=1, ncells=(N,), lmax=(1000.0,), kg=(G, 0.0), kb=0.0, cfl=0.4,
                       fixed_kinetics=True)
        edges = np.linspace(0.0, 1000.0, N + 1)
        n0, exact_end = profile(edges, 0.0), profile(edges, G * t_end)
        r = oracle.solve(p, n0, 0.2, 0.0, np.array([t_end]))
        mask = (edges[:-1] > 100.0) & (edges[1:] < 800.0)
        errs.append(np.sum(np.abs(r["n"] - exact_end)[mask]) * (1000.0 / N))
    return np.array(errs)


def test_translation_smooth_front_second_order():
    # front rising from 0 well inside the domain; exact solution n0(L - G t)
    Ns = [200, 400, 800, 1600]
    def prof(edges, shift):
        f = _cell_avg_tanh_front(edges, 300.0 + shift, 25.0)
        g = _cell_avg_tanh_front(edges, 600.0 + shift, 25.0)
        return f - g   # plateau between two smooth monotone fronts
    e = _translation_errors(prof, Ns)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 1.8), (e, order)


def test_translation_gaussian_converges():
    Ns = [200, 400, 800, 1600]
    e = _translation_errors(lambda ed, s: _cell_avg_gauss(ed, 300.0 + s, 30.0), Ns)
    order = np.log2(e[:-1] / e[1:])
    assert np.all(order >= 1.5), (e, order)   # TVD limiters clip smooth extrema


def _tv(n):
    return np.sum(np.abs(np.diff(np.concatenate([[0.0], n, [0.0]]))))


def test_tvd_and_positivity_fixed_growth():
    rng = np.random.default_rng(3)
    N = 120
    p = pi.Problem(ndim=1, ncells=(N,), lmax=(600.0,), kg=(0.3, 0.0), kb=0.0, cfl=0.5,
                   fixed_kinetics=True)
    n = np.clip(rng.standard_normal(N).cumsum(), 0, None) + (rng.uniform(size=N) > 0.8) * 5
    n[-20:] = 0.0
    t = 0.0
    for _ in range(40):
        tv0 = _tv(n)
        n, info = oracle.step(p, n, 0.2, t, 1e9)
        t = info["t"]
        assert _tv(n) <= tv0 * (1 + 1e-14)
        # positive up to rounding of cancelling tail values
        assert n.min() >= -1e-15 * n.max()


def test_positivity_full_configs():
    r = oracle.solve_instance(pi.config_1d())
    assert np.all(r["n"] >= 0.0)
    r2 = oracle.solve_instance(pi.config_2d(64))
    assert np.all(r2["n"] >= 0.0)


def test_solute_plus_crystal_mass_conserved():
    inst = pi.config_1d()
    r = oracle.solve_instance(inst)
    tot = r["rows"][:, 5] + inst.problem.kappa * r["rows"][:, 4]
    assert np.max(np.abs(tot - tot[0])) <= 1e-12 * tot[0]
    inst2 = pi.config_2d(64)
    r2 = oracle.solve_instance(inst2)
    tot2 = r2["rows"][:, 11] + inst2.problem.kappa * r2["rows"][:, 9]
    assert np.max(np.abs(tot2 - tot2[0])) <= 1e-12 * tot2[0]
    assert r["rows"][-1, 5] < r["rows"][0, 5]   # concentration falls as crystals grow


def test_volume_change_equals_flux_form():
    """sum_i x_i^3 L_i dL == sum over faces F_f (x_f^3 - x_{f-1}^3) + x_0^3 B
    (summation by parts of the conservative update; the outflow face carries
    -F_N x_{N-1}^3)."""
    N = 60
    p = dataclasses.replace(pi.config_1d(N).problem, fixed_kinetics=True)
    rng = np.random.default_rng(5)
    n = rng.uniform(0, 2, N)
    G, B = 0.3, 11.0
    d = 1000.0 / N
    x = (np.arange(N) + 0.5) * d
    L = oracle.rhs(p, n, G, 0.0, B)
    F = oracle.face_fluxes(p, n, G)
    lhs = np.sum(x ** 3 * L * d)
    rhs = np.sum(F[1:N] * (x[1:] ** 3 - x[:-1] ** 3)) - F[N] * x[-1] ** 3 + x[0] ** 3 * B
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert F[0] == 0.0


def test_2d_reduces_to_1d_per_direction():
    N1, N2 = 40, 30
    u = pi.gaussian_seed_1d(N1, 500.0, 150.0, 30.0, 1.0)
    v = pi.gaussian_seed_1d(N2, 500.0, 200.0, 40.0, 1.0)
    n2d = np.outer(u, v)
    p2 = pi.Problem(ndim=2, ncells=(N1, N2), lmax=(500.0, 500.0), kg=(0.5, 0.0), kb=0.0, cfl=0.4,
                    fixed_kinetics=True)
    p1 = pi.Problem(ndim=1, ncells=(N1,), lmax=(500.0,), kg=(0.5, 0.0), kb=0.0, cfl=0.4,
                    fixed_kinetics=True)
    r2 = oracle.solve(p2, n2d, 0.2, 0.0, np.array([150.0]))
    r1 = oracle.solve(p1, u, 0.2, 0.0, np.array([150.0]))
    assert np.max(np.abs(r2["n"] - np.outer(r1["n"], v))) <= 1e-14 * np.max(n2d)
    # the same along L2
    p2b = dataclasses.replace(p2, kg=(0.0, 0.5))
    p1b = pi.Problem(ndim=1, ncells=(N2,), lmax=(500.0,), kg=(0.5, 0.0), kb=0.0, cfl=0.4,
                     fixed_kinetics=True)
    r2b = oracle.solve(p2b, n2d, 0.2, 0.0, np.array([150.0]))
    r1b = oracle.solve(p1b, v, 0.2, 0.0, np.array([150.0]))
    assert np.max(np.abs(r2b["n"] - np.outer(u, r1b["n"]))) <= 1e-14 * np.max(n2d)


def _mu_closed_form_1d(mu0, G, B, L0, t):
    # shift of the seed by G t plus nuclei born at L0 at rate B and grown since
    out = []
    for k in range(4):
        v = sum(math.comb(k, j) * (G * t) ** j * mu0[k - j] for j in range(k + 1))
        if G > 0:
            v += B * ((L0 + G * t) ** (k + 1) - L0 ** (k + 1)) / (G * (k + 1))
        out.append(v)
    return np.array(out)


def test_mom_reference_against_closed_form():
    p = pi.Problem(ndim=1, ncells=(1,), lmax=(1.0,), kg=(0.02, 0.0), kb=300.0, fixed_kinetics=True)
    mu0 = np.array([1e8, 1.5e10, 2.29e12, 3.555e14])
    t_out = np.array([0.0, 600.0, 3600.0])
    rows = mom.solve(p, mu0, 0.25, 0.0, t_out, (2.5,), dt_max=5.0)
    for r in rows:
        want = _mu_closed_form_1d(mu0, 0.02, 300.0, 2.5, r[0])
        assert np.allclose(r[1:5], want, rtol=1e-12)
        assert r[5] == pytest.approx(0.25 - p.kappa * (want[3] - mu0[3]), rel=1e-14)
    # 2-D: separable shift of a product measure, nuclei at (L10, L20)
    p2 = pi.Problem(ndim=2, ncells=(1, 1), lmax=(1.0, 1.0), kg=(0.03, 0.01), kb=50.0,
                    fixed_kinetics=True)
    a = [1.0, 100.0, 1.1e4, 1.3e6]     # moments of a 1-D marginal in L1
    bb = [1.0, 60.0, 3.7e3, 2.4e5]    # and in L2
    m0 = np.array([1e8 * a[p_] * bb[q_] for p_, q_ in mom.PQ_2D])
    rows = mom.solve(p2, m0, 0.25, 0.0, [1000.0], (1.0, 2.0), dt_max=5.0)
    t = 1000.0
    from numpy.polynomial.legendre import leggauss
    xs, ws = leggauss(6)
    for k, (P, Q) in enumerate(mom.PQ_2D):
        v = 1e8 * sum(math.comb(P, i) * (0.03 * t) ** i * a[P - i] for i in range(P + 1)) * \
            sum(math.comb(Q, j) * (0.01 * t) ** j * bb[Q - j] for j in range(Q + 1))
        s = 0.5 * t * (xs + 1.0)
        v += 50.0 * 0.5 * t * np.sum(ws * (1.0 + 0.03 * s) ** P * (2.0 + 0.01 * s) ** Q)
        assert rows[0][1 + k] == pytest.approx(v, rel=1e-12), (P, Q)


def _fvm_vs_mom(ndim, N, kb):
    inst = pi.config_1d(N) if ndim == 1 else pi.config_2d(N)
    p = dataclasses.replace(inst.problem, kb=kb)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)
    L0 = tuple(0.5 * l / n for l, n in zip(p.lmax, p.ncells))   # nuclei enter at the first cell centre
    ref = mom.solve(p, r["rows"][0, 1:-1], inst.C0, 0.0, inst.t_out, L0, dt_max=1.0)
    return (np.abs(r["rows"][:, 1:] - ref[:, 1:]) / np.abs(ref[:, 1:])).max()


@pytest.mark.parametrize("ndim", [1, 2])
def test_fvm_converges_to_method_of_moments_growth_only(ndim):
    """The paper's verification (Sec. 3.1, SI Sec. S1.2): for the growth-only
    model of Eq. 1 the FVM moments and concentration converge to the method of
    moments under grid refinement (spatial error dominates at these grids)."""
    grids = [100, 200, 400] if ndim == 1 else [48, 96, 192]
    errs = [_fvm_vs_mom(ndim, N, 0.0) for N in grids]
    assert errs[0] / errs[1] >= 3.0 and errs[1] / errs[2] >= 3.0, errs
    assert errs[-1] < (1e-4 if ndim == 1 else 5e-4), errs


@pytest.mark.parametrize("ndim", [1, 2])
def test_fvm_approaches_method_of_moments_with_nucleation(ndim):
    """With nucleation at the smallest-size cell the FVM and the moment model
    (nuclei of size dL/2) differ at O(dL) near the boundary; the gap closes."""
    grids = [100, 200, 400] if ndim == 1 else [48, 96, 192]
    errs = [_fvm_vs_mom(ndim, N, 1e6) for N in grids]
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[-1] < 2e-2, errs
