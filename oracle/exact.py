"""Exact rational brute force of the SSP-RK2 finite-volume step on tiny grids.

Test infrastructure only.  Written straight from the paper's formulas in Python
``fractions`` so that no rounding enters: smoothness ratio
theta_{i+1/2} = (f_i - f_{i-1}) / (f_{i+1} - f_i) and van Leer
phi = (theta + |theta|) / (1 + |theta|) (SI Sec. S1.1); upwind flux of Eq. 3 in
semi-discrete form; zero ghost cells; nucleation B into the first (corner) cell;
solute balance of Eq. 4.  Kinetics are held fixed (rational G, B) so every
quantity stays rational; the CFL step nu / sum(G_m / dL_m) is rational too.
"""
from __future__ import annotations

from fractions import Fraction as Fr


def _phi_times_b(a: Fr, b: Fr) -> Fr:
    if b == 0:
        return Fr(0)  # theta -> +-inf: phi -> 2 (or 0) times b -> 0
    th = a / b
    return (th + abs(th)) / (1 + abs(th)) * b


def _get(n, i):
    return n[i] if 0 <= i < len(n) else Fr(0)


def rhs1(n, G, B, d):
    N = len(n)

    def F(f):
        return G * (_get(n, f - 1) + Fr(1, 2) * _phi_times_b(_get(n, f - 1) - _get(n, f - 2),
                                                             _get(n, f) - _get(n, f - 1)))
    L = [-(F(i + 1) - F(i)) / d for i in range(N)]
    L[0] += B / d
    return L


def rhs2(n, G1, G2, B, d1, d2):
    N1, N2 = len(n), len(n[0])

    def g(i, j):
        return n[i][j] if 0 <= i < N1 and 0 <= j < N2 else Fr(0)

    def F1(f, j):
        return G1 * (g(f - 1, j) + Fr(1, 2) * _phi_times_b(g(f - 1, j) - g(f - 2, j), g(f, j) - g(f - 1, j)))

    def F2(i, f):
        return G2 * (g(i, f - 1) + Fr(1, 2) * _phi_times_b(g(i, f - 1) - g(i, f - 2), g(i, f) - g(i, f - 1)))
    L = [[-(F1(i + 1, j) - F1(i, j)) / d1 - (F2(i, j + 1) - F2(i, j)) / d2 for j in range(N2)]
         for i in range(N1)]
    L[0][0] += B / (d1 * d2)
    return L


def step1(n, G, B, d, nu, t, t_next):
    """One exact step in 1-D.  Returns (n_new, dt, t_new)."""
    dt = nu / (G / d) if G > 0 else None
    if dt is None or not dt < t_next - t:
        dt, t_new = t_next - t, t_next
    else:
        t_new = t + dt
    L = rhs1(n, G, B, d)
    n1 = [a + dt * l for a, l in zip(n, L)]
    L1 = rhs1(n1, G, B, d)
    return [Fr(1, 2) * a + Fr(1, 2) * (b + dt * l) for a, b, l in zip(n, n1, L1)], dt, t_new


def step2(n, G1, G2, B, d1, d2, nu, t, t_next):
    rate = G1 / d1 + G2 / d2
    dt = nu / rate if rate > 0 else None
    if dt is None or not dt < t_next - t:
        dt, t_new = t_next - t, t_next
    else:
        t_new = t + dt
    L = rhs2(n, G1, G2, B, d1, d2)
    n1 = [[a + dt * l for a, l in zip(ra, rl)] for ra, rl in zip(n, L)]
    L1 = rhs2(n1, G1, G2, B, d1, d2)
    return ([[Fr(1, 2) * a + Fr(1, 2) * (b + dt * l) for a, b, l in zip(ra, rb, rl)]
             for ra, rb, rl in zip(n, n1, L1)], dt, t_new)
