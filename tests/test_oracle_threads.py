"""The oracle's OpenMP loops (used only to time the CPU baseline on every
core) leave every result unchanged: a multi-threaded solve equals the
single-threaded one bit for bit."""
import numpy as np

import oracle
import pbe_inputs as pi


def test_threaded_oracle_solve_is_bitwise_equal():
    inst = pi.config_2d(160, 130)   # above the 16384-cell threshold of the parallel loops
    t_out = inst.t_out[:8]
    try:
        oracle.set_threads(1)
        a = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, t_out)
        n = oracle.set_threads(4)
        b = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, t_out)
    finally:
        oracle.set_threads(1)
    assert n >= 1
    assert a["steps"] == b["steps"]
    assert np.array_equal(a["rows"], b["rows"])
    assert np.array_equal(a["n"], b["n"])
