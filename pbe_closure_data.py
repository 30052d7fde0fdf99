"""Seeded inputs of the learned-closure workload (2-D, 128 x 128 grid).

Holds no solver arithmetic: the hidden power-law kinetics, the per-trajectory
cooling end temperatures and seed shifts, and an initial weight draw for the
closure network.  Shared by the training driver, its tests and the benchmark.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

import pbe_inputs as pi

CLOSURE_SIZE = 64 * 3 + 64 + 64 * 64 + 64 + 3 * 64 + 3


def hidden_law(seed: int = 2413) -> tuple:
    """(kg1, g1, kg2, g2, kb, b) drawn once: kg log-U[0.01, 0.2], g U[1, 2],
    kb log-U[1e5, 1e7], b U[1.5, 3]."""
    rng = np.random.default_rng(seed)
    kg1 = math.exp(rng.uniform(math.log(0.01), math.log(0.2)))
    kg2 = math.exp(rng.uniform(math.log(0.01), math.log(0.2)))
    g1, g2 = rng.uniform(1.0, 2.0, 2)
    kb = math.exp(rng.uniform(math.log(1e5), math.log(1e7)))
    b = rng.uniform(1.5, 3.0)
    return (kg1, float(g1), kg2, float(g2), kb, float(b))


def trajectories(count: int, seed: int, N: int = 128, hidden_seed: int = 2413):
    """Instances of the 2-D problem that differ in the cooling end temperature
    (U[15, 30] C) and in the seed means (+-20 %), all with the hidden law; the
    output times are the 50 loss times."""
    rng = np.random.default_rng(seed)
    law = hidden_law(hidden_seed)
    out = []
    for _ in range(count):
        T1 = rng.uniform(15.0, 30.0)
        f1, f2 = rng.uniform(0.8, 1.2, 2)
        base = pi.config_2d(N)
        p = dataclasses.replace(base.problem, T1=T1).with_theta(law)
        n0 = pi.gaussian_seed_2d(N, N, 500.0, 500.0, (100.0 * f1, 60.0 * f2), (15.0, 10.0), 0.3, 1e8)
        out.append(pi.Instance(p, n0, base.C0, 0.0, pi.loss_times()))
    return out


def misspecified(inst):
    """The same instance with the nominal power-law kinetics of the 2-D
    configuration (the model without the learned closure)."""
    nominal = pi.config_2d(inst.problem.ncells[0]).problem
    return dataclasses.replace(inst.problem, kg=nominal.kg, g=nominal.g, kb=nominal.kb, b=nominal.b)


def initial_weights(seed: int = 7, scale: float = 0.1) -> np.ndarray:
    """Small random initial closure weights (float32 flat layout)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(CLOSURE_SIZE).astype(np.float32) * np.float32(scale)
    # biases start at zero
    H = 64
    w[H * 3:H * 3 + H] = 0.0
    o = H * 3 + H + H * H
    w[o:o + H] = 0.0
    w[-3:] = 0.0
    return w


def bf16_round(w) -> np.ndarray:
    """Round float32 values to bf16 (round to nearest even) and return them as float64."""
    a = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((a + 0x7FFF + ((a >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def stored_weights(w) -> np.ndarray:
    """The closure weights as the library stores them: matrices rounded to bf16,
    biases kept in float32 (float64 copy, for the oracle)."""
    w32 = np.ascontiguousarray(w, dtype=np.float32)
    out = w32.astype(np.float64)
    H = 64
    segs = [(0, H * 3), (H * 3 + H, H * 3 + H + H * H), (H * 3 + 2 * H + H * H, H * 3 + 2 * H + H * H + 3 * H)]
    for a, b in segs:
        out[a:b] = bf16_round(w32[a:b])
    return out
