"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module only describes problems and draws their inputs: parameter sets,
initial distributions and output times.  It holds none of the solver's
arithmetic, so the oracle and the CUDA library can both take their inputs from
it without sharing any of the method.

Workloads (shapes and value ranges of the crystallization problems of
Sec. 2.1 / Sec. 3; the paper's own in-silico data is not used):
  * ``config_1d``   - 1-D seeded cooling crystallization, 200 cells on [0, 1000] um
  * ``config_2d``   - 2-D size-and-shape problem, 256 x 256 cells on [0, 500]^2 um
  * ``batch_1d``    - 4096 independent 1-D instances with sampled sizes and kinetics
  * ``adjoint_*``   - loss-time grids and target perturbations for gradients
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

# polynomial solubility c*(T) = c0 + c1 T + c2 T^2  (g/g, T in deg C)
CSAT = (0.1, 0.003, 2e-5)
# rho_c k_v = 1e-15 g/um^3 times u = 1e-3 (n in #/kg solvent, C in g/g)
KAPPA = 1e-15 * 1e-3


@dataclass(frozen=True)
class Problem:
    """One PBE problem.  Growth G_d = kg[d] s^g[d], nucleation B = kb s^b with
    s = max(C / c*(T) - 1, 0); linear cooling T0 -> T1 over t_cool seconds."""

    ndim: int
    ncells: tuple
    lmax: tuple
    kg: tuple = (0.05, 0.0)
    g: tuple = (1.5, 1.0)
    kb: float = 1e6
    b: float = 2.0
    csat: tuple = CSAT
    T0: float = 40.0
    T1: float = 20.0
    t_cool: float = 3600.0
    kappa: float = KAPPA
    cfl: float = 0.5
    fixed_kinetics: bool = False
    scheme: int = 0            # 0: SSP-RK2 unsplit; 1: Eq. 3 with Godunov splitting
    growth_form: int = 0       # 0: kg s^g; 1: Arrhenius kg exp(-ea/(T+273.15)) s^g; 2: polynomial (Eq. 6)
    solubility_form: int = 0   # 0: polynomial csat; 1: csat[0] exp(csat[1] T)
    ea: tuple = (0.0, 0.0)     # activation temperatures of the Arrhenius form (K)
    poly: tuple = ()           # growth_form 2: ndim x K coefficients, a_m1 .. a_mK of G_m = sum_k a_mk s^k
    mlp_box: tuple = ()        # learned closure: ((lo0, lo1, lo2), (hi0, hi1, hi2)) training box of its
                               # inputs; outside it (or for a non-finite rate) the power law above is used

    @property
    def ncell(self) -> int:
        return int(np.prod(self.ncells))

    @property
    def theta(self) -> np.ndarray:
        """Kinetic parameters in the order (kg1, g1, kg2, g2, kb, b)."""
        return np.array([self.kg[0], self.g[0], self.kg[1], self.g[1], self.kb, self.b])

    def with_theta(self, th) -> "Problem":
        th = [float(v) for v in th]
        return dataclasses.replace(self, kg=(th[0], th[2]), g=(th[1], th[3]), kb=th[4], b=th[5])


@dataclass
class Instance:
    problem: Problem
    n0: np.ndarray  # float64, 1-D (N,) or 2-D (N1, N2) row-major
    C0: float
    t0: float
    t_out: np.ndarray = field(default_factory=lambda: np.zeros(0))


def csat_at(T: float) -> float:
    """Value of the stated solubility polynomial (the initial concentration is
    specified as c*(T0))."""
    return CSAT[0] + CSAT[1] * T + CSAT[2] * T * T


def gaussian_seed_1d(N: int, lmax: float, mean: float, sd: float, total: float) -> np.ndarray:
    """Gaussian seed sampled at cell centres and scaled so that the discrete
    zeroth moment sum(n) * dL equals ``total``."""
    d = lmax / N
    x = (np.arange(N) + 0.5) * d
    f = np.exp(-0.5 * ((x - mean) / sd) ** 2)
    return f * (total / (f.sum() * d))


def gaussian_seed_2d(N1: int, N2: int, lmax1: float, lmax2: float, mean, sd, corr: float,
                     total: float) -> np.ndarray:
    d1, d2 = lmax1 / N1, lmax2 / N2
    x1 = ((np.arange(N1) + 0.5) * d1)[:, None]
    x2 = ((np.arange(N2) + 0.5) * d2)[None, :]
    z1 = (x1 - mean[0]) / sd[0]
    z2 = (x2 - mean[1]) / sd[1]
    q = (z1 * z1 - 2.0 * corr * z1 * z2 + z2 * z2) / (1.0 - corr * corr)
    f = np.exp(-0.5 * q)
    return f * (total / (f.sum() * d1 * d2))


def output_times(t_end: float = 3600.0, every: float = 60.0, include_zero: bool = True) -> np.ndarray:
    k0 = 0 if include_zero else 1
    n = int(round(t_end / every))
    return np.array([k * every for k in range(k0, n + 1)], dtype=np.float64)


def config_1d(N: int = 200) -> Instance:
    """1-D seeded cooling crystallization: [0, 1000] um, Gaussian seed (150, 20) um
    scaled to 1e8 #/kg, G = 0.05 s^1.5 um/s, B = 1e6 s^2, cooling 40 -> 20 C over
    3600 s, CFL 0.5, outputs every 60 s."""
    p = Problem(ndim=1, ncells=(N,), lmax=(1000.0,), kg=(0.05, 0.0), g=(1.5, 1.0), kb=1e6, b=2.0,
                cfl=0.5)
    n0 = gaussian_seed_1d(N, 1000.0, 150.0, 20.0, 1e8)
    return Instance(p, n0, csat_at(40.0), 0.0, output_times())


def config_2d(N1: int = 256, N2: int | None = None) -> Instance:
    """2-D size-and-shape problem: [0, 500]^2 um, Gaussian seed means (100, 60),
    sd (15, 10), correlation 0.3, total 1e8 #/kg; G1 = 0.04 s^1.3, G2 = 0.02 s^1.8,
    B = 1e6 s^2 into the corner cell; CFL 0.4; same cooling and solubility."""
    N2 = N1 if N2 is None else N2
    p = Problem(ndim=2, ncells=(N1, N2), lmax=(500.0, 500.0), kg=(0.04, 0.02), g=(1.3, 1.8),
                kb=1e6, b=2.0, cfl=0.4)
    n0 = gaussian_seed_2d(N1, N2, 500.0, 500.0, (100.0, 60.0), (15.0, 10.0), 0.3, 1e8)
    return Instance(p, n0, csat_at(40.0), 0.0, output_times())


def batch_1d(count: int = 4096, seed: int = 2411, N_fixed: int | None = None,
             t_out: np.ndarray | None = None) -> list[Instance]:
    """Independent 1-D instances of the ``config_1d`` model with sampled grid size
    N ~ U{100..2000}, kg log-U[0.01, 0.2], g U[1, 2], kb log-U[1e5, 1e7],
    b U[1.5, 3], cooling end temperature U[15, 30] C, seed mean U[80, 250] um."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = int(rng.integers(100, 2001)) if N_fixed is None else int(N_fixed)
        kg = math.exp(rng.uniform(math.log(0.01), math.log(0.2)))
        g = rng.uniform(1.0, 2.0)
        kb = math.exp(rng.uniform(math.log(1e5), math.log(1e7)))
        b = rng.uniform(1.5, 3.0)
        T1 = rng.uniform(15.0, 30.0)
        mean = rng.uniform(80.0, 250.0)
        p = Problem(ndim=1, ncells=(N,), lmax=(1000.0,), kg=(kg, 0.0), g=(g, 1.0), kb=kb, b=b,
                    T1=T1, cfl=0.5)
        n0 = gaussian_seed_1d(N, 1000.0, mean, 20.0, 1e8)
        out.append(Instance(p, n0, csat_at(40.0), 0.0,
                            output_times() if t_out is None else np.asarray(t_out, np.float64)))
    return out


def loss_times() -> np.ndarray:
    """50 evenly spaced loss times t_k = 72 k s, k = 1..50."""
    return np.array([72.0 * k for k in range(1, 51)], dtype=np.float64)


TARGET_FACTOR = 1.10  # target trajectory: every kinetic parameter scaled by 1.1


def adjoint_2d(N: int = 128) -> Instance:
    inst = config_2d(N)
    inst.t_out = loss_times()
    return inst


def adjoint_batch_1d(count: int = 256, seed: int = 2412) -> list[Instance]:
    return batch_1d(count, seed=seed, N_fixed=500, t_out=loss_times())


# ---------------------------------------------------------------------------
# The paper's own base case (Table 1 and Appendix A, Table A.1): 2-D growth-only
# batch crystallizer at constant 15 C, exponential solubility, Arrhenius growth,
# seed normal in both lengths scaled by the seed mass, one-step high-resolution
# scheme with Godunov splitting at Courant number 0.9.
# ---------------------------------------------------------------------------
RHO_C = 1.11e-12            # g / um^3
KV = math.pi / 4.0          # cylinder


def paper_seed_2d(N1: int, N2: int, lmax1: float = 1200.0, lmax2: float = 600.0, mean=(400.0, 250.0),
                  sd=(30.0, 30.0), seed_mass: float = 1.0) -> np.ndarray:
    """Normal seed in both lengths, scaled so that rho_c k_v sum x1 x2^2 n dA equals
    the seed mass (SI Sec. S1.3, scale factor beta)."""
    d1, d2 = lmax1 / N1, lmax2 / N2
    x1 = ((np.arange(N1) + 0.5) * d1)[:, None]
    x2 = ((np.arange(N2) + 0.5) * d2)[None, :]
    f = np.exp(-0.5 * ((x1 - mean[0]) / sd[0]) ** 2 - 0.5 * ((x2 - mean[1]) / sd[1]) ** 2)
    mass = RHO_C * KV * float(np.sum(x1 * x2 * x2 * f)) * d1 * d2
    return f * (seed_mass / mass)


def paper_base_case(N1: int = 1200, N2: int | None = None, t_end: float = 3600.0, every: float | None = None) -> Instance:
    """Table 1 / Table A.1: 1200 x 600 um, 1 um bins at N1 = 1200 (N2 = N1 / 2), T = 15 C,
    c0 = 8 g/kg, seed mass 1 g (means 400/250 um, sd 30 um), rho_c = 1.11e-12 g/um^3,
    k_v = pi/4, c* = 3.37 exp(0.036 T) g/kg, G1 = 8.86e6 um/min exp(-2450/(T+273.15)) (S-1)^3.7,
    G2 = 4.088e5 um/min exp(-2400/(T+273.15)) (S-1)^2.5, no nucleation, Courant number 0.9.
    Concentration in g/kg and n in # per kg per um^2, so kappa = rho_c k_v.  The simulated
    time is read as one hour (the table's "1000 [hour]" is garbled)."""
    N2 = N1 // 2 if N2 is None else N2
    p = Problem(ndim=2, ncells=(N1, N2), lmax=(1200.0, 600.0), kg=(8.86e6 / 60.0, 4.088e5 / 60.0),
                g=(3.7, 2.5), kb=0.0, b=2.0, csat=(3.37, 0.036, 0.0), T0=15.0, T1=15.0, t_cool=3600.0,
                kappa=RHO_C * KV, cfl=0.9, scheme=1, growth_form=1, solubility_form=1, ea=(2450.0, 2400.0))
    n0 = paper_seed_2d(N1, N2)
    t_out = np.array([t_end]) if every is None else output_times(t_end, every)
    return Instance(p, n0, 8.0, 0.0, t_out)


def config_1d_fine(N: int = 1 << 20, horizon: float = 10.0, every: float = 1.0, S0: float = 1.5) -> Instance:
    """1-D problem of ``config_1d`` on a fine grid (up to 2^20 cells of ~1e-3 um on
    [0, 1000] um), started supersaturated at S = S0 so that every step is CFL-limited
    (dt ~ 0.5 dL / G): the grid-size sweep of the 1-D path.  Outputs every ``every``
    seconds up to ``horizon``."""
    inst = config_1d(N)
    n_out = int(round(horizon / every))
    t_out = np.array([k * every for k in range(n_out + 1)], dtype=np.float64)
    return Instance(inst.problem, inst.n0, S0 * csat_at(40.0), 0.0, t_out)


def poly_growth(problem: Problem, K: int, seed: int = 2414) -> Problem:
    """The problem with the polynomial growth law of Eq. 6 (growth_form 2) in place
    of the power law: K non-negative coefficients per growth direction,
    a_mk = kg_m u_mk 2^-(k-1) with u_mk ~ U[0.5, 1.5] (seeded), so that the
    leading term is of the size of the power-law rate and the series decays."""
    rng = np.random.default_rng(seed)
    a = []
    for m in range(problem.ndim):
        u = rng.uniform(0.5, 1.5, size=K)
        a.extend(float(problem.kg[m] * u[k] * 0.5 ** k) for k in range(K))
    return dataclasses.replace(problem, growth_form=2, poly=tuple(a))
