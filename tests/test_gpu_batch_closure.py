"""The learned kinetics closure in the batched 1-D kernel (bf16 weights,
fp32 arithmetic, the moment ratio V / mu0 summed at every stage) against the
FP64 oracle evaluating the same stored weights, instance by instance."""
import dataclasses

import numpy as np
import pytest

import oracle
import pbe_closure_data as cd
import pbe_inputs as pi

pytestmark = pytest.mark.gpu

REL_ROWS_MLP = 2e-5   # fp32 in the 64-wide layers, as for the single-grid closure


def _physical(inst, w):
    """The oracle's trajectory with the closure stays physical (C > 0 at
    every row): with random initial weights the network's rates can blow up
    and drive C far below zero within a step, where every path (and the
    oracle) only amplifies rounding."""
    r = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
    return bool(np.all(r["rows"][:, 5] > 0.0))


def _insts(w=None):
    w = cd.initial_weights(3, 0.2) if w is None else w
    insts = [x for x in pi.batch_1d(16, seed=23) if _physical(x, w)]
    assert len(insts) >= 8
    for N in (33, 700):
        insts.append(pi.config_1d(N))
    return insts


def _solve(insts, w, schedule=None, box=None):
    import paper_2411_00742_gb300 as P
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], closure=True)
    b.set_state(b.pack([x.n0 for x in insts]))
    b.set_closure(w)
    if box is not None:
        b.set_closure_box(*box)
    if schedule:
        b.set_schedule(*schedule)
    rows, steps = b.solve(insts[0].t_out)
    n, C, t = b.get_state()
    b.close()
    return rows, steps, n, C


def test_batch_closure_matches_oracle():
    insts = _insts()
    w = cd.initial_weights(3, 0.2)
    rows, _, _, _ = _solve(insts, w)
    for i, inst in enumerate(insts):
        want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
        err = np.max(np.abs(rows[i][:, 1:] - want["rows"][:, 1:]) / np.abs(want["rows"][:, 1:]))
        assert err <= REL_ROWS_MLP, (i, err)


def test_batch_closure_schedules_bitwise():
    """Team and warp instances with the closure give the same bits (the chain
    runs the same network in every warp, the sums are per fixed segment)."""
    insts = _insts()
    w = cd.initial_weights(3, 0.2)
    a = _solve(insts, w, schedule=(4, 0))
    b = _solve(insts, w, schedule=(3, 5))
    assert np.array_equal(a[0], b[0]) and a[1] == b[1]
    assert all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))


def test_batch_closure_box_falls_back_to_the_power_law():
    """A training box that no input reaches: every rate comes from the power
    law, as the oracle's fallback computes it."""
    insts = _insts()[:4]
    w = cd.initial_weights(3, 0.2)
    lo, hi = (100.0, 100.0, 100.0), (101.0, 101.0, 101.0)
    rows, _, _, _ = _solve(insts, w, box=(lo, hi))
    for i, inst in enumerate(insts):
        p = dataclasses.replace(inst.problem, mlp_box=(lo, hi))
        want = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
        plain = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)
        np.testing.assert_allclose(want["rows"], plain["rows"], rtol=1e-12)
        err = np.max(np.abs(rows[i][:, 1:] - want["rows"][:, 1:]) / np.abs(want["rows"][:, 1:]))
        assert err <= 1e-10, (i, err)


def test_batch_closure_needs_weights():
    import paper_2411_00742_gb300 as P
    insts = _insts()[:3]
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], closure=True)
    b.set_state(b.pack([x.n0 for x in insts]))
    with pytest.raises(P.PbeError) as e:
        b.solve(insts[0].t_out)
    assert "ESTATE" in str(e.value)
    b.close()
