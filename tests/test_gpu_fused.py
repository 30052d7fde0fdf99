"""Parity of the fused persistent path (one cooperative launch per solve) with
the CPU oracle, at the same tolerances as the plain path."""
import numpy as np
import pytest

import oracle
import pbe_inputs as pi
from gpu_helpers import REL_ROWS, assert_n_close, assert_rows_close, compare_instance, gpu_solve

pytestmark = pytest.mark.gpu


def test_fused_1d_config():
    compare_instance(pi.config_1d(200), path="fused")


@pytest.mark.parametrize("N", [1, 2, 7, 1023, 1024, 1025, 3000, 70001])
def test_fused_1d_ragged(N):
    compare_instance(pi.config_1d(N), path="fused")


@pytest.mark.parametrize("shape", [(1, 1), (3, 200), (37, 53), (64, 64), (129, 31)])
def test_fused_2d_ragged(shape):
    compare_instance(pi.config_2d(*shape), path="fused")


def test_fused_2d_full_size():
    compare_instance(pi.config_2d(256), path="fused")


@pytest.mark.parametrize("shape", [(300, 333), (1000, 150), (600, 400)])
def test_fused_2d_tall_tiles(shape):
    # one tile per block of 17..64 rows (the tall-tile kernel, dynamic shared
    # memory), ragged in both directions
    compare_instance(pi.config_2d(*shape), path="fused")


def test_fused_2d_larger_than_one_wave():
    # tiles taller than 64 rows would be needed for one per block: blocks loop
    # over several 16 x 32 tiles (window kernel off)
    compare_instance(pi.config_2d(1200, 300), path="fused", window=0)


@pytest.mark.parametrize("shape", [(1200, 300), (700, 530), (333, 1000)])
def test_fused_2d_window_kernel(shape):
    # grids too large for one tile per block, on the persistent window kernel
    # (the default there): blocks loop over 2R x 125 window tiles, halo rows
    # and columns from the other blocks through L2, ragged in both directions
    compare_instance(pi.config_2d(*shape), path="fused", window=1)


def test_fused_window_kernel_matches_tile_loop_closely():
    inst = pi.config_2d(1200, 300)
    a = gpu_solve(inst, path="fused", window=0)
    b = gpu_solve(inst, path="fused", window=1)
    assert a["steps"] == b["steps"]
    np.testing.assert_allclose(b["rows"], a["rows"], rtol=1e-12)
    c = gpu_solve(inst, path="fused", window=1)
    assert np.array_equal(b["rows"], c["rows"]) and np.array_equal(b["n"], c["n"])


@pytest.mark.parametrize("blocks", [8, 19])
def test_fused_block_limit(blocks):
    """A block limit (grids solved side by side): the one-tile launch takes
    taller tiles, or blocks loop over several; parity with the oracle and
    with the unlimited launch."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(128)
    ref = gpu_solve(inst, path="fused")
    g = P.Grid.from_problem(inst.problem, path="fused")
    g.set_block_limit(blocks)
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
    rows, steps = g.solve(inst.t_out)
    n, C, _ = g.get_state()
    g.close()
    assert steps == ref["steps"]
    np.testing.assert_allclose(rows, ref["rows"], rtol=1e-12)
    want = oracle.solve_instance(inst)
    assert_rows_close(rows, want["rows"])
    assert_n_close(n, want["n"])


def test_fused_state_at_every_output_time():
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(48, 40)
    g = P.Grid.from_problem(inst.problem, path="fused")
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
    n, C, t = np.array(inst.n0), inst.C0, inst.t0
    for tk in inst.t_out[1:]:
        rows, _ = g.solve([tk])
        ng, Cg, tg = g.get_state()
        r = oracle.solve(inst.problem, n, C, t, [tk])
        n, C, t = r["n"], r["C"], r["t"]
        assert_n_close(ng, n)
        assert abs(Cg - C) <= REL_ROWS * abs(C)
        assert_rows_close(rows, r["rows"])
    g.close()


def test_fused_matches_plain_closely():
    a = gpu_solve(pi.config_2d(128), path="plain")
    b = gpu_solve(pi.config_2d(128), path="fused")
    assert a["steps"] == b["steps"]
    np.testing.assert_allclose(b["rows"], a["rows"], rtol=1e-12)


def test_fused_deterministic_bitwise():
    a = gpu_solve(pi.config_2d(200), path="fused")
    b = gpu_solve(pi.config_2d(200), path="fused")
    assert np.array_equal(a["rows"], b["rows"]) and np.array_equal(a["n"], b["n"])


def test_auto_path_is_the_fused_path_with_the_plain_fallback():
    # SSP-RK2: "auto" runs the fused kernels (the same bits); the paper scheme
    # (plain path only) still solves under "auto", as on the plain path; other
    # values are rejected
    import dataclasses
    import paper_2411_00742_gb300 as P
    a = gpu_solve(pi.config_2d(96, 80), path="auto")
    b = gpu_solve(pi.config_2d(96, 80), path="fused")
    assert a["steps"] == b["steps"]
    assert np.array_equal(a["rows"], b["rows"]) and np.array_equal(a["n"], b["n"])
    inst = pi.config_1d(300)
    paper = dataclasses.replace(inst.problem, scheme=1)
    rows = {}
    for path in ("auto", "plain"):
        g = P.Grid.from_problem(paper, path=path)
        g.set_state(inst.n0, inst.C0, 0.0)
        rows[path], _ = g.solve(inst.t_out)
        g.close()
    assert np.array_equal(rows["auto"], rows["plain"])
    g = P.Grid.from_problem(inst.problem)
    with pytest.raises(P.PbeError):
        P._lib.check(g.lib.pbe_set_path(g.h, 3))
    g.close()


def test_fused_step_budget_and_nonfinite():
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(64)
    g = P.Grid.from_problem(inst.problem, path="fused")
    g.set_max_steps(5)
    g.set_state(inst.n0, inst.C0, 0.0)
    with pytest.raises(P.PbeError) as e:
        g.solve(inst.t_out)
    assert e.value.status == 5
    g.set_max_steps(10 ** 6)
    n = inst.n0.copy()
    n[10, 10] = np.inf
    g.set_state(n, inst.C0, 0.0)
    with pytest.raises(P.PbeError) as e:
        g.solve(inst.t_out)
    assert e.value.status == 4
    g.close()


def test_fused_wait_limit_runs_out_and_context_survives():
    """Failure detection without a fault: a zero wait limit makes the device-wide
    barrier give up (status PBE_ETIMEOUT read by the host); the grid and the
    context stay usable and the next solve with the default limit is exact."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_2d(256)
    g = P.Grid.from_problem(inst.problem, path="fused")
    g.set_wait_limit(0.0)
    g.set_state(inst.n0, inst.C0, 0.0)
    with pytest.raises(P.PbeError) as e:
        g.solve(inst.t_out)
    assert e.value.status == 5
    g.set_wait_limit(-1.0)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    g.close()
    want = oracle.solve_instance(inst)
    assert steps == want["steps"]
    assert_rows_close(rows, want["rows"])


@pytest.fixture(scope="module")
def fine_1d():
    # the largest 1-D grid (2^20 cells), supersaturated start: ~40 CFL-limited steps
    inst = pi.config_1d_fine(1 << 20, horizon=1.0, every=0.5)
    return inst, oracle.solve_instance(inst)


@pytest.mark.parametrize("path", ["fused", "plain"])
def test_1d_max_cells(fine_1d, path):
    inst, want = fine_1d
    got = gpu_solve(inst, path=path)
    assert got["steps"] == want["steps"] >= 30
    assert_rows_close(got["rows"], want["rows"])
    assert_n_close(got["n"], want["n"])
