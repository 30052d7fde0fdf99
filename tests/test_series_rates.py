"""The series form of the power-law rates used for the second rate
evaluation of a step (the fused, window and batch kernels): with d = C - c*
at one solubility, G(d) = G(d0) (1 + delta)^p, delta = (d - d0)/d0, and the
kernels evaluate (1 + delta)^p - 1 and log1p(delta) by their series to
delta^5 whenever |delta| <= 2^-10.  Pins the truncation claim (first omitted
term below 1e-18 relative to 1) against exact rational arithmetic, for the
exponents the workloads use and the edge of the range, with the coefficient
recursion and Horner order the kernels use."""
from fractions import Fraction

import pytest


def binom_coefs(p):
    c, out = 1.0, []
    for k in range(1, 6):
        c = c * (p - (k - 1)) / k
        out.append(c)
    return out


def series(coefs, delta):
    P = coefs[4] * delta + coefs[3]
    P = P * delta + coefs[2]
    P = P * delta + coefs[1]
    P = P * delta + coefs[0]
    return P * delta


def exact_pow_minus_one(p, delta, terms=40):
    # (1 + delta)^p - 1 by the binomial series in exact rationals, far past double precision
    p, delta = Fraction(p), Fraction(delta)
    c, s, dk = Fraction(1), Fraction(0), Fraction(1)
    for k in range(1, terms):
        c = c * (p - (k - 1)) / k
        dk *= delta
        s += c * dk
    return s


def exact_log1p(delta, terms=40):
    delta = Fraction(delta)
    return sum(Fraction((-1) ** (k + 1), k) * delta ** k for k in range(1, terms))


@pytest.mark.parametrize("p", [1.0, 1.3, 1.8, 2.0, 2.5, 3.0, 1.0 + 2 ** -20])
@pytest.mark.parametrize("delta", [2 ** -10, -2 ** -10, 3e-6, -4.3e-7, 1e-12, 0.0])
def test_binomial_series_within_rounding(p, delta):
    got = series(binom_coefs(p), delta)
    want = exact_pow_minus_one(p, delta)
    # G = G0 (1 + P): the error relative to 1 is the truncation (< 1e-18) plus
    # a few roundings of P (|P| < 3 * 2^-10)
    assert abs(Fraction(got) - want) <= Fraction(2, 10 ** 18) + Fraction(abs(float(want))) * Fraction(1, 2 ** 50)


@pytest.mark.parametrize("delta", [2 ** -10, -2 ** -10, 3e-6, -1e-9])
def test_log1p_series_within_rounding(delta):
    coefs = [1.0, -0.5, 1.0 / 3, -0.25, 0.2]
    got = series(coefs, delta)
    want = exact_log1p(delta)
    assert abs(Fraction(got) - want) <= Fraction(2, 10 ** 18) + Fraction(abs(float(want))) * Fraction(1, 2 ** 50)


def test_exact_integer_weights():
    # the batch kernels' weights (2i + 1)^k are exact doubles below 2^52 for
    # every cell of the largest instance (6144 cells), and (2i + 1)^k (dL/2)^k
    # equals x_i^k with x_i = (i + 1/2) dL
    for i in (0, 1, 6143):
        w3 = (2 * i + 1) ** 3
        assert w3 < 2 ** 52 and float(w3) == w3
        dL = Fraction(1000, 6144)
        assert Fraction(w3) * (dL / 2) ** 3 == ((i + Fraction(1, 2)) * dL) ** 3
