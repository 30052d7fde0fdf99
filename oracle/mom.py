"""Method of moments (SI Sec. S1.2, Eq. for d mu_pq / dt) - test infrastructure only.

For size-independent growth the moment equations close:
    d mu_pq / dt = p G1 mu_{p-1,q} + q G2 mu_{p,q-1} + B L10^p L20^q,
where the last term adds nuclei of size (L10, L20) at rate B (the paper's model
has no nucleation; the term is zero when B = 0).  The solute balance of Eq. 2
closes the system: dC/dt = -kappa d mu_3 / dt (1-D) or -kappa d mu_12 / dt (2-D).
Integrated with classical fourth-order Runge-Kutta on a fixed sub-step, landing
on every output time.  Kinetics are restated here (not shared with the C oracle):
S = C / c*(T), s = max(S - 1, 0), G_m = kg_m s^g_m, B = kb s^b.
"""
from __future__ import annotations

import numpy as np

PQ_2D = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (3, 0), (2, 1), (1, 2), (0, 3)]
_IDX = {pq: k for k, pq in enumerate(PQ_2D)}


def _kin(problem, C, t):
    if problem.fixed_kinetics:
        return problem.kg[0], (problem.kg[1] if problem.ndim == 2 else 0.0), problem.kb
    frac = t / problem.t_cool if t < problem.t_cool else 1.0
    T = problem.T0 + (problem.T1 - problem.T0) * frac
    if getattr(problem, "solubility_form", 0) == 1:
        cs = problem.csat[0] * np.exp(problem.csat[1] * T)
    else:
        cs = problem.csat[0] + problem.csat[1] * T + problem.csat[2] * T * T
    s = C / cs - 1.0
    if not s > 0.0:
        return 0.0, 0.0, 0.0
    a1 = a2 = 1.0
    if getattr(problem, "growth_form", 0) == 1:   # Arrhenius factor of Appendix A
        a1 = np.exp(-problem.ea[0] / (T + 273.15))
        a2 = np.exp(-problem.ea[1] / (T + 273.15))
    G2 = a2 * problem.kg[1] * s ** problem.g[1] if problem.ndim == 2 else 0.0
    return a1 * problem.kg[0] * s ** problem.g[0], G2, problem.kb * s ** problem.b


def _rhs(problem, y, t, L0):
    G1, G2, B = _kin(problem, y[-1], t)
    dy = np.zeros_like(y)
    if problem.ndim == 1:
        for k in range(4):
            dy[k] = (k * G1 * y[k - 1] if k > 0 else 0.0) + B * L0[0] ** k
        dy[4] = -problem.kappa * dy[3]
    else:
        for k, (p, q) in enumerate(PQ_2D):
            v = B * L0[0] ** p * L0[1] ** q
            if p > 0:
                v += p * G1 * y[_IDX[(p - 1, q)]]
            if q > 0:
                v += q * G2 * y[_IDX[(p, q - 1)]]
            dy[k] = v
        dy[10] = -problem.kappa * dy[_IDX[(1, 2)]]
    return dy


def solve(problem, mu0, C0, t0, t_out, L0, dt_max=0.25):
    """Integrate the moment system.  mu0: initial moments (4 in 1-D, 10 in 2-D,
    ordered as PQ_2D).  L0: nucleus size per direction.  Returns rows like the
    oracle: (t, moments..., C)."""
    y = np.concatenate([np.asarray(mu0, dtype=np.float64), [C0]])
    t = float(t0)
    rows = []
    for tn in t_out:
        while t < tn:
            h = min(dt_max, tn - t)
            k1 = _rhs(problem, y, t, L0)
            k2 = _rhs(problem, y + 0.5 * h * k1, t + 0.5 * h, L0)
            k3 = _rhs(problem, y + 0.5 * h * k2, t + 0.5 * h, L0)
            k4 = _rhs(problem, y + h * k3, t + h, L0)
            y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
            t = tn if tn - t <= h else t + h
        rows.append(np.concatenate([[t], y]))
    return np.array(rows)
