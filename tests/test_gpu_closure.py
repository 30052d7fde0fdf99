"""The learned kinetics closure on the GPU (bf16 weights, fp32 arithmetic)
against the FP64 oracle evaluating the same stored weights.

Tolerances follow from fp32 arithmetic in the 64-wide layers (relative
rounding ~1e-7 per accumulated product, ~1e-6 on the outputs, which enter the
rates through exp): rows within 2e-5 relative, weight gradients within 2e-3
of the largest gradient entry."""
import numpy as np
import pytest

import oracle
import pbe_closure_data as cd
import pbe_inputs as pi

pytestmark = pytest.mark.gpu

REL_ROWS_MLP = 2e-5
REL_GRAD_MLP = 2e-3


def _grid(inst, w, path="plain"):
    import paper_2411_00742_gb300 as P
    g = P.Grid.from_problem(inst.problem, path=path)
    g.set_closure(w)
    g.set_kinetics(inst.problem, closure=True)
    return g


@pytest.mark.parametrize("path", ["plain", "fused"])
@pytest.mark.parametrize("ndim", [1, 2])
def test_closure_forward_matches_oracle(ndim, path):
    inst = pi.config_1d(200) if ndim == 1 else cd.trajectories(1, seed=11, N=48)[0]
    w = cd.initial_weights(3, 0.2)
    g = _grid(inst, w, path)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    g.close()
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
    assert steps == want["steps"]
    err = np.max(np.abs(rows[:, 1:] - want["rows"][:, 1:]) / np.abs(want["rows"][:, 1:]))
    assert err <= REL_ROWS_MLP, err


def test_closure_forward_window_kernel_matches_oracle():
    """The learned closure on the plain path's register-window stage kernel
    (forced on a small grid; it reads every moment at every stage)."""
    inst = cd.trajectories(1, seed=11, N=48)[0]
    w = cd.initial_weights(3, 0.2)
    g = _grid(inst, w)
    g.set_window(1)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    g.close()
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
    assert steps == want["steps"]
    err = np.max(np.abs(rows[:, 1:] - want["rows"][:, 1:]) / np.abs(want["rows"][:, 1:]))
    assert err <= REL_ROWS_MLP, err


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_closure_gradients_match_oracle(path):
    inst = cd.trajectories(1, seed=12, N=40)[0]
    w = cd.initial_weights(4, 0.2)
    ws = cd.stored_weights(w)
    tgt = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]   # hidden-law truth
    cols = [1, 2, 3, 9, 11]
    r = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=ws)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    _, _, _, want = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=ws)
    g = _grid(inst, w, path)
    g.set_state(inst.n0, inst.C0, 0.0)
    dW = np.zeros(cd.CLOSURE_SIZE)
    g.vjp(inst.t_out, seeds, 64, dweights_out=dW)
    g.close()
    scale = np.max(np.abs(want))
    assert np.max(np.abs(dW - want)) <= REL_GRAD_MLP * scale, np.max(np.abs(dW - want)) / scale
    # gradient direction agrees closely
    cos = float(np.dot(dW, want) / (np.linalg.norm(dW) * np.linalg.norm(want)))
    assert cos > 0.99999


def test_closure_gradient_matches_central_differences_on_gpu():
    import paper_2411_00742_gb300 as P
    inst = cd.trajectories(1, seed=13, N=32)[0]
    w = cd.initial_weights(5, 0.2)
    tgt = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    cols = [1, 2, 3, 9, 11]

    def loss(wv):
        g = _grid(inst, wv)
        g.set_state(inst.n0, inst.C0, 0.0)
        rows, _ = g.solve(inst.t_out)
        g.close()
        return oracle.relative_loss(rows, tgt, cols), rows

    L0, rows = loss(w)
    g = _grid(inst, w)
    g.set_state(inst.n0, inst.C0, 0.0)
    dW = np.zeros(cd.CLOSURE_SIZE)
    g.vjp(inst.t_out, oracle.relative_loss_seeds(rows, tgt, cols), 64, dweights_out=dW)
    g.close()
    # biases are stored in fp32 (no bf16 rounding): differentiate through them
    H = 64
    for k in (H * 3 + 5, H * 3 + H + H * H + 9, cd.CLOSURE_SIZE - 1, cd.CLOSURE_SIZE - 3):
        h = 2e-3
        wp, wm = w.copy(), w.copy()
        wp[k] += h
        wm[k] -= h
        fd = (loss(wp)[0] - loss(wm)[0]) / (2 * h)
        assert dW[k] == pytest.approx(fd, rel=2e-2, abs=1e-6 * np.max(np.abs(dW))), k


def test_trained_closure_beats_the_plain_kinetics():
    """Train the closure briefly through the solver's adjoint on trajectories of
    the hidden law and compare, on held-out trajectories, with the solver
    that uses the nominal (wrong) power law: the trained closure must cut the
    relative moment-trajectory error."""
    from paper_2411_00742_gb300.train_closure import main
    res = main(["--train", "96", "--heldout", "24", "--grid", "48", "--epochs", "5", "--batch", "16",
                "--lr", "3e-3", "--workers", "8"])
    assert res["loss_history"][-1] < 0.5 * res["loss_history"][0]
    assert res["gain"] > 1.3, res["heldout_rel_rms_error"]


def _partial_box(inst, w):
    """A training box cutting the supersaturation input x0 = 4 (S - 1) at its
    median along the oracle's closure solve: the stages above it take the
    power-law fallback, the others the network."""
    import dataclasses
    r0 = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))["rows"]
    p = inst.problem
    T = np.array([oracle.temperature(p, t) for t in r0[:, 0]])
    x0 = 4.0 * (r0[:, -1] / (p.csat[0] + p.csat[1] * T + p.csat[2] * T * T) - 1.0)
    cut = float(np.median(x0[x0 > 0]))
    inst.problem = dataclasses.replace(p, mlp_box=((-10.0, -10.0, -10.0), (cut, 10.0, 10.0)))
    return inst


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_closure_fallback_forward_matches_oracle(path):
    inst = cd.trajectories(1, seed=11, N=48)[0]
    w = cd.initial_weights(3, 0.2)
    inst = _partial_box(inst, w)
    g = _grid(inst, w, path)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    g.close()
    want = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=cd.stored_weights(w))
    assert steps == want["steps"]
    err = np.max(np.abs(rows[:, 1:] - want["rows"][:, 1:]) / np.abs(want["rows"][:, 1:]))
    assert err <= REL_ROWS_MLP, err


def test_closure_box_excluding_every_input_gives_the_power_law_solve():
    import dataclasses
    import paper_2411_00742_gb300 as P
    inst = cd.trajectories(1, seed=11, N=48)[0]
    w = cd.initial_weights(3, 0.2)
    inst.problem = dataclasses.replace(inst.problem, mlp_box=((50.0, 50.0, 50.0), (60.0, 60.0, 60.0)))
    g = _grid(inst, w)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, steps = g.solve(inst.t_out)
    g.close()
    gp = P.Grid.from_problem(inst.problem)
    gp.set_state(inst.n0, inst.C0, 0.0)
    want, wsteps = gp.solve(inst.t_out)
    gp.close()
    assert steps == wsteps
    np.testing.assert_allclose(rows[:, 1:], want[:, 1:], rtol=1e-14)


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_closure_fallback_gradients_match_oracle(path):
    """With a partly active box the adjoint differentiates the network on some
    stages and the power law on the others: dL/dweights and dL/d(kinetic
    parameters) against the oracle's adjoint."""
    inst = cd.trajectories(1, seed=12, N=40)[0]
    w = cd.initial_weights(4, 0.2)
    ws = cd.stored_weights(w)
    inst = _partial_box(inst, w)
    tgt = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    cols = [1, 2, 3, 9, 11]
    r = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=ws)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    want_th, _, _, want = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=ws)
    g = _grid(inst, w, path)
    g.set_state(inst.n0, inst.C0, 0.0)
    dW = np.zeros(cd.CLOSURE_SIZE)
    dth, _, _ = g.vjp(inst.t_out, seeds, 64, dweights_out=dW)
    g.close()
    scale = np.max(np.abs(want))
    assert np.max(np.abs(dW - want)) <= REL_GRAD_MLP * scale, np.max(np.abs(dW - want)) / scale
    assert np.any(want_th != 0.0)
    for j in range(6):
        assert dth[j] == pytest.approx(want_th[j], rel=REL_GRAD_MLP, abs=1e-12 * np.max(np.abs(want_th))), j


def test_fused_closure_solve_at_the_workload_size_and_its_timeout():
    """The closure's fused-path solve (the persistent kernel's forward pass) on
    the 128 x 128 closure workload against the plain path; a zero wait limit
    ends it with PBE_ETIMEOUT and the grid solves normally afterwards."""
    from paper_2411_00742_gb300 import _lib
    inst = cd.trajectories(1, seed=21, N=128)[0]
    w = cd.initial_weights(3, 0.2)
    out = {}
    for path in ("plain", "fused"):
        g = _grid(inst, w, path)
        g.set_state(inst.n0, inst.C0, 0.0)
        out[path] = g.solve(inst.t_out)
        if path == "fused":
            g.set_wait_limit(0.0)
            g.set_state(inst.n0, inst.C0, 0.0)
            with pytest.raises(_lib.PbeError) as ei:
                g.solve(inst.t_out)
            assert "ETIMEOUT" in str(ei.value)
            g.set_wait_limit(-1.0)
            g.set_state(inst.n0, inst.C0, 0.0)
            again, _ = g.solve(inst.t_out)
            np.testing.assert_array_equal(again, out["fused"][0])
        g.close()
    assert out["plain"][1] == out["fused"][1]
    np.testing.assert_allclose(out["fused"][0][:, 1:], out["plain"][0][:, 1:], rtol=REL_ROWS_MLP)


def _closure_grad_case(seed, N=40, w_seed=4):
    inst = cd.trajectories(1, seed=seed, N=N)[0]
    w = cd.initial_weights(w_seed, 0.2)
    ws = cd.stored_weights(w)
    tgt = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    r = oracle.solve(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, mlp=ws)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, [1, 2, 3, 9, 11])
    return inst, w, ws, seeds


def _assert_dw_close(got, want, rel):
    """Element-wise where the entry is not negligible against the largest one."""
    scale = np.max(np.abs(want))
    big = np.abs(want) >= 1e-3 * scale
    err = np.abs(got - want)
    assert np.all(err[big] <= rel * np.abs(want[big])), np.max(err[big] / np.abs(want[big]))
    assert np.all(err[~big] <= rel * 1e-3 * scale)


def test_tensor_core_weight_gradient_matches_fp64_per_stage_accumulation():
    """The fused path's weight gradient (rows recorded by the adjoint, tensor-core
    contractions with split bf16 operands) against the plain path's fp64
    accumulation of the same per-stage products, element by element, and both
    against the oracle."""
    inst, w, ws, seeds = _closure_grad_case(12)
    dws = {}
    for path in ("plain", "fused"):
        g = _grid(inst, w, path)
        g.set_state(inst.n0, inst.C0, 0.0)
        dws[path] = np.zeros(cd.CLOSURE_SIZE)
        g.vjp(inst.t_out, seeds, 64, dweights_out=dws[path])
        g.close()
    _assert_dw_close(dws["fused"], dws["plain"], 1e-4)
    _, _, _, want = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=ws)
    _assert_dw_close(dws["fused"], want, 2e-3)


def test_closure_grad_over_several_trajectories_in_one_launch():
    """pbe_closure_grad over three grids' recorded rows equals the sum of their
    single-trajectory gradients and the sum of the oracle's."""
    import paper_2411_00742_gb300 as P
    cases = [_closure_grad_case(s) for s in (31, 32, 33)]
    grids, singles, wants = [], [], []
    for inst, w, ws, seeds in cases:
        g = _grid(inst, w, "fused")
        g.set_state(inst.n0, inst.C0, 0.0)
        d = np.zeros(cd.CLOSURE_SIZE)
        g.vjp(inst.t_out, seeds, 64, dweights_out=d)
        singles.append(d)
        grids.append(g)
        wants.append(oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds, mlp=ws)[3])
    tot = P.closure_grad(grids)
    for g in grids:
        g.close()
    _assert_dw_close(tot, sum(singles), 1e-5)
    _assert_dw_close(tot, sum(wants), 2e-3)
