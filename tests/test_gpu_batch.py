"""Parity of the batched persistent 1-D path (one warp per instance, one
launch for the whole batch) with the CPU oracle, instance by instance."""
import dataclasses

import numpy as np
import pytest

import oracle
import pbe_inputs as pi
from gpu_helpers import REL_N, REL_ROWS, assert_rows_close

pytestmark = pytest.mark.gpu


def _run_batch(insts, wpb=None, autotune=False):
    import paper_2411_00742_gb300 as P
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], [x.t0 for x in insts])
    b.set_state(b.pack([x.n0 for x in insts]))
    t_out = insts[0].t_out
    chosen = None
    if autotune:
        chosen = b.autotune(t_out)
    elif wpb is not None:
        b.set_config(wpb)
    rows, steps = b.solve(t_out)
    n, C, t = b.get_state()
    b.close()
    return rows, steps, n, C, t, chosen


def _check_against_oracle(insts, rows, steps, n, C):
    tot = 0
    for i, inst in enumerate(insts):
        want = oracle.solve_instance(inst)
        tot += want["steps"]
        assert_rows_close(rows[i], want["rows"])
        scale = np.max(np.abs(want["n"])) if np.any(want["n"]) else 1.0
        assert np.max(np.abs(n[i] - want["n"])) <= REL_N * scale, i
        assert abs(C[i] - want["C"]) <= REL_ROWS * abs(want["C"]), i
    assert steps == tot


def test_batch_sampled_instances_match_oracle():
    insts = pi.batch_1d(96, seed=2411)
    rows, steps, n, C, t, _ = _run_batch(insts)
    _check_against_oracle(insts, rows, steps, n, C)
    assert np.all(t == 3600.0)


def test_batch_edge_sizes_and_kinetics():
    base = pi.batch_1d(8, seed=7)
    insts = []
    for N in (1, 2, 31, 32, 33, 63, 64, 65, 6144):
        inst = pi.config_1d(N)
        insts.append(inst)
    z = pi.config_1d(120)
    z.n0 = np.zeros(120)                    # empty seed: nucleation only
    insts.append(z)
    fx = pi.config_1d(500)
    fx.problem = dataclasses.replace(fx.problem, fixed_kinetics=True, kg=(0.3, 0.0), kb=2.0)
    insts.append(fx)
    insts += base
    rows, steps, n, C, t, _ = _run_batch(insts)
    _check_against_oracle(insts, rows, steps, n, C)


@pytest.mark.parametrize("wpb", [1, 2, 3, 6, 8])
def test_batch_config_independent_bitwise(wpb):
    # instances small enough that 8 per block fit in shared memory
    insts = [x for x in pi.batch_1d(120, seed=99) if x.problem.ncells[0] <= 1500][:40]
    ref = _run_batch(insts, wpb=4)
    got = _run_batch(insts, wpb=wpb)
    assert np.array_equal(ref[0], got[0]) and ref[1] == got[1]
    assert all(np.array_equal(a, b) for a, b in zip(ref[2], got[2]))


def _run_schedule(insts, wpb, nteam, wcells=6144):
    import paper_2411_00742_gb300 as P
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], [x.t0 for x in insts])
    b.set_state(b.pack([x.n0 for x in insts]))
    b.set_schedule(wpb, nteam, wcells)
    assert b.schedule() == (wpb, nteam, wcells)
    rows, steps = b.solve(insts[0].t_out)
    n, C, t = b.get_state()
    b.close()
    return rows, steps, n, C, t


@pytest.mark.parametrize("wpb,nteam,wcells", [(1, 3, 6144), (2, 7, 6144), (3, 40, 6144), (4, 13, 6144),
                                              (6, 1, 6144), (8, -1, 6144), (4, 0, 300), (2, 5, 0), (3, 2, 257)])
def test_batch_team_schedules_bitwise(wpb, nteam, wcells):
    """Instances solved by a whole block (team) give the same bits as the
    same instances solved by one warp: the moment sums are formed per fixed
    segment whichever warp forms them.  Teams chosen by cost and by a size
    cut; sizes from 1 cell to 2 segments per warp of the widest block, ragged
    tails included."""
    insts = [x for x in pi.batch_1d(60, seed=31) if x.problem.ncells[0] <= 1500][:40]
    for N in (1, 31, 255, 256, 257, 1500):
        insts.append(pi.config_1d(N))
    ref = _run_schedule(insts, 4, 0)
    got = _run_schedule(insts, wpb, len(insts) if nteam < 0 else nteam, wcells)
    assert np.array_equal(ref[0], got[0]) and ref[1] == got[1]
    assert all(np.array_equal(a, b) for a, b in zip(ref[2], got[2]))
    assert np.array_equal(ref[3], got[3]) and np.array_equal(ref[4], got[4])


def test_batch_team_instances_match_oracle():
    """Every instance a team instance, including the largest admissible grid
    (6144 cells: 24 segments over 8 warps)."""
    insts = pi.batch_1d(10, seed=8)
    for N in (6144, 3000, 520):
        insts.append(pi.config_1d(N))
    import paper_2411_00742_gb300 as P
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], [x.t0 for x in insts])
    b.set_state(b.pack([x.n0 for x in insts]))
    b.set_schedule(8, len(insts))
    rows, steps = b.solve(insts[0].t_out)
    n, C, t = b.get_state()
    b.close()
    _check_against_oracle(insts, rows, steps, n, C)


def test_batch_autotune_keeps_results():
    insts = pi.batch_1d(200, seed=5)
    ref = _run_batch(insts, wpb=4)
    got = _run_batch(insts, autotune=True)
    assert got[5] in (1, 2, 3, 4, 6, 8)
    assert np.array_equal(ref[0], got[0])
    assert all(np.array_equal(a, b) for a, b in zip(ref[2], got[2]))


def test_batch_continues_from_state():
    import paper_2411_00742_gb300 as P
    insts = pi.batch_1d(16, seed=3)
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts])
    b.set_state(b.pack([x.n0 for x in insts]))
    b.solve(np.array([0.0, 600.0]))
    rows, _ = b.solve(np.array([1200.0, 1800.0]))
    b.close()
    for i, inst in enumerate(insts):
        r1 = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, [0.0, 600.0])
        r2 = oracle.solve(inst.problem, r1["n"], r1["C"], r1["t"], [1200.0, 1800.0])
        assert_rows_close(rows[i], r2["rows"])


def test_batch_full_workload_sampled():
    """The 4096-instance workload at full size, in the configuration the
    benchmark times (autotuned), checked on a sample of instances."""
    insts = pi.batch_1d(4096, seed=2411)
    rows, steps, n, C, t, _ = _run_batch(insts, autotune=True)
    rng = np.random.default_rng(0)
    for i in rng.choice(4096, size=24, replace=False):
        want = oracle.solve_instance(insts[i])
        assert_rows_close(rows[i], want["rows"])
        assert np.max(np.abs(n[i] - want["n"])) <= REL_N * np.max(np.abs(want["n"]))
    assert np.all(t == 3600.0)
    assert steps >= 60 * 4096


def test_batch_rejects_config_that_does_not_fit():
    import paper_2411_00742_gb300 as P
    insts = [pi.config_1d(6000) for _ in range(4)]
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts])
    with pytest.raises(P.PbeError):
        b.set_config(8)
    with pytest.raises(P.PbeError):
        b.set_schedule(4, 5)            # more team instances than instances
    with pytest.raises(P.PbeError):
        b.set_schedule(3, 0)            # 3 warp instances of 6000 cells: 3 x 97 KB, ...
    b.set_schedule(4, 4)                # ... all four as team instances: 97 KB a block
    assert b.schedule() == (4, 4, 6144)
    b.set_schedule(4, 0, 5999)          # the same four by the size cut
    with pytest.raises(P.PbeError):
        b.set_schedule(4, 0, 6145)
    b.close()


def test_batch_rejects_oversized_instance():
    import paper_2411_00742_gb300 as P
    with pytest.raises(P.PbeError) as e:
        P.Batch([pi.config_1d(6145).problem], [0.252])
    assert e.value.status == 1
