"""GPU discrete adjoint (pbe_vjp) against the FP64 CPU adjoint of the oracle
and against central finite differences of the GPU forward path (the
gradient bar: 1e-6 relative), on both paths: the per-stage kernels (plain)
and the persistent kernel that runs forward, recomputation and reverse
sweep in one launch (fused)."""
import numpy as np
import pytest

import oracle
import pbe_inputs as pi

pytestmark = pytest.mark.gpu

REL_GRAD = 1e-6


def _problem(case):
    # 1d_big: several 512-cell tiles and blocks; 2d_tall: 16-row tiles, several per block
    return {"1d": lambda: pi.config_1d(200), "1d_cfl": lambda: pi.config_1d(800),
            "2d": lambda: pi.config_2d(40), "2d_rect": lambda: pi.config_2d(36, 52),
            "2d_128": lambda: pi.adjoint_2d(128), "1d_big": lambda: pi.config_1d(2500),
            "2d_tall": lambda: pi.config_2d(300, 70)}[case]()


def _setup(inst):
    p = inst.problem
    inst.t_out = pi.loss_times()
    tgt = oracle.solve(p.with_theta(p.theta * pi.TARGET_FACTOR), inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    cols = [1, 2, 3, 4, 5] if p.ndim == 1 else [1, 2, 3, 9, 11]
    return p, tgt, cols


def _gpu_grad(inst, seeds, K, window=-1, path="plain"):
    import torch
    import paper_2411_00742_gb300 as P
    g = P.Grid.from_problem(inst.problem, path=path)
    g.set_window(window)
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, 0.0)
    dn0 = torch.zeros(inst.problem.ncells, dtype=torch.float64, device="cuda")
    rows = torch.zeros(seeds.shape, dtype=torch.float64, device="cuda")
    dth, _, dC0 = g.vjp(inst.t_out, seeds, K, dn0_out=dn0, rows_out=rows)
    _, C, t = g.get_state()
    g.close()
    return dth, dn0.cpu().numpy(), dC0, rows.cpu().numpy(), t


@pytest.mark.parametrize("path", ["plain", "fused"])
@pytest.mark.parametrize("case,K", [("1d", 64), ("1d_cfl", 7), ("2d", 64), ("2d_rect", 5), ("2d_128", 64),
                                    ("1d_big", 16), ("2d_tall", 9)])
def test_vjp_matches_cpu_adjoint(case, K, path):
    inst = _problem(case)
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    want, want_dn0, want_dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    dth, dn0, dC0, rows, t_end = _gpu_grad(inst, seeds, K, path=path)
    for j in range(6):
        assert dth[j] == pytest.approx(want[j], rel=REL_GRAD, abs=1e-300), (case, j, dth, want)
    # d/dn0 on the seed's support; outside it the derivative runs through the
    # limiter in numerically-zero tails, where rounding decides its branch
    supp = inst.n0 > 1e-3 * inst.n0.max()
    assert np.max(np.abs(dn0 - want_dn0)[supp]) <= REL_GRAD * np.max(np.abs(want_dn0))
    assert np.all(np.isfinite(dn0))
    v = inst.n0 * np.cos(np.linspace(0, 3, inst.n0.size)).reshape(inst.n0.shape)
    assert float(np.sum(dn0 * v)) == pytest.approx(float(np.sum(want_dn0 * v)), rel=REL_GRAD)
    assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD)
    np.testing.assert_allclose(rows[:, 1:], r[:, 1:], rtol=1e-10)
    assert t_end == pytest.approx(inst.t_out[-1])


def test_vjp_with_window_stage_kernel_matches_cpu_adjoint():
    """Forward passes and segment recomputation in the register-window stage
    kernel (forced on a small rectangular grid)."""
    inst = _problem("2d_rect")
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    want, want_dn0, want_dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    dth, dn0, dC0, rows, _ = _gpu_grad(inst, seeds, 16, window=1)
    for j in range(6):
        assert dth[j] == pytest.approx(want[j], rel=REL_GRAD, abs=1e-300), (j, dth, want)
    assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD)
    np.testing.assert_allclose(rows[:, 1:], r[:, 1:], rtol=1e-10)


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_vjp_checkpoint_interval_does_not_change_result(path):
    inst = _problem("2d")
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    a = _gpu_grad(inst, seeds, 1, path=path)
    b = _gpu_grad(inst, seeds, 64, path=path)
    c = _gpu_grad(inst, seeds, 1000, path=path)
    assert np.array_equal(a[0], b[0]) and np.array_equal(b[0], c[0])
    assert np.array_equal(a[1], b[1])


@pytest.mark.parametrize("case,blocks", [("2d_128", 19), ("1d", 2)])
def test_fused_vjp_with_block_limit_matches_cpu_adjoint(case, blocks):
    """The persistent adjoint on a limited number of blocks (several tiles a
    block), as the closure trainer runs its concurrent trajectories."""
    import torch
    import paper_2411_00742_gb300 as P
    inst = _problem(case)
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    want, want_dn0, want_dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    g = P.Grid.from_problem(p, path="fused")
    g.set_block_limit(blocks)
    g.set_state(np.ascontiguousarray(inst.n0), inst.C0, 0.0)
    dn0 = torch.zeros(p.ncells, dtype=torch.float64, device="cuda")
    dth, _, dC0 = g.vjp(inst.t_out, seeds, 64, dn0_out=dn0)
    g.close()
    for j in range(6):
        assert dth[j] == pytest.approx(want[j], rel=REL_GRAD, abs=1e-300), (j, dth, want)
    assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD)
    supp = inst.n0 > 1e-3 * inst.n0.max()
    assert np.max(np.abs(dn0.cpu().numpy() - want_dn0)[supp]) <= REL_GRAD * np.max(np.abs(want_dn0))


def test_fused_vjp_grows_its_checkpoint_store_and_repeats_bitwise():
    """Two output times, the second reached by CFL-limited steps, and a
    checkpoint every step: the persistent adjoint's first checkpoint store
    (sized from the output count) is too small and is grown until the solve
    fits; repeated calls on the same grid reuse the buffers and give the same
    gradient bit for bit."""
    import paper_2411_00742_gb300 as P
    inst = pi.config_1d(800)
    p = inst.problem
    inst.t_out = np.array([720.0, 3600.0])
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)
    assert r["steps"] > 20
    seeds = np.zeros((2, 6))
    seeds[:, 1:] = 1.0 / np.abs(r["rows"][:, 1:])
    want, _, want_dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    g = P.Grid.from_problem(p, path="fused")
    got = []
    for K in (1, 1, 3):
        g.set_state(inst.n0, inst.C0, 0.0)
        dth, _, dC0 = g.vjp(inst.t_out, seeds, K)
        got.append((dth, dC0))
    g.close()
    for dth, dC0 in got:
        for j in (0, 1, 4, 5):
            assert dth[j] == pytest.approx(want[j], rel=REL_GRAD), j
        assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD)
    assert np.array_equal(got[0][0], got[1][0]) and np.array_equal(got[0][0], got[2][0])


def test_fused_vjp_wait_limit_ends_in_timeout_and_grid_stays_usable():
    """A zero wait limit makes the persistent adjoint's first device-wide
    barrier run out (a multi-block grid): PBE_ETIMEOUT, no hang; the grid
    then solves and differentiates normally."""
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    inst = _problem("2d")
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    g = P.Grid.from_problem(p, path="fused")
    g.set_state(inst.n0, inst.C0, 0.0)
    g.set_wait_limit(0.0)
    with pytest.raises(_lib.PbeError) as ei:
        g.vjp(inst.t_out, seeds, 64)
    assert "ETIMEOUT" in str(ei.value)
    g.set_wait_limit(-1.0)
    g.set_state(inst.n0, inst.C0, 0.0)
    dth, _, _ = g.vjp(inst.t_out, seeds, 64)
    g.close()
    want, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    for j in range(6):
        assert dth[j] == pytest.approx(want[j], rel=REL_GRAD), j


def test_vjp_matches_central_differences_of_gpu_forward():
    import paper_2411_00742_gb300 as P
    inst = _problem("1d_cfl")
    p, tgt, cols = _setup(inst)

    def loss(theta):
        g = P.Grid.from_problem(p)
        g.set_kinetics(p, theta=theta)
        g.set_state(inst.n0, inst.C0, 0.0)
        rows, steps = g.solve(inst.t_out)
        g.close()
        return oracle.relative_loss(rows, tgt, cols), steps

    g = P.Grid.from_problem(p)
    g.set_state(inst.n0, inst.C0, 0.0)
    rows, _ = g.solve(inst.t_out)
    seeds = oracle.relative_loss_seeds(rows, tgt, cols)
    g.set_state(inst.n0, inst.C0, 0.0)
    dth, _, _ = g.vjp(inst.t_out, seeds, 64)
    g.close()
    th = p.theta
    for j in (0, 1, 4, 5):
        h = 1e-6 * abs(th[j])
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        (Lp, sp), (Lm, sm) = loss(tp), loss(tm)
        assert sp == sm
        assert dth[j] == pytest.approx((Lp - Lm) / (2 * h), rel=REL_GRAD), j


@pytest.mark.parametrize("path", ["plain", "fused"])
def test_autograd_function(path):
    import torch
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300.autograd import PBESolve
    inst = _problem("2d")
    p, tgt, cols = _setup(inst)
    g = P.Grid.from_problem(p, path=path)
    theta = torch.tensor(p.theta, dtype=torch.float64, requires_grad=True)
    n0 = torch.as_tensor(inst.n0).cuda().requires_grad_(True)
    rows = PBESolve.apply(theta, n0, g, p, inst.C0, 0.0, inst.t_out, 64)
    tgt_t = torch.as_tensor(tgt).cuda()
    L = (((rows[:, cols] - tgt_t[:, cols]) / tgt_t[:, cols]) ** 2).sum()
    L.backward()
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    want, want_dn0, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, oracle.relative_loss_seeds(r, tgt, cols))
    np.testing.assert_allclose(theta.grad.numpy(), want, rtol=REL_GRAD)
    supp = inst.n0 > 1e-3 * inst.n0.max()
    assert np.max(np.abs(n0.grad.cpu().numpy() - want_dn0)[supp]) <= REL_GRAD * np.max(np.abs(want_dn0))
    g.close()


@pytest.mark.parametrize("K,warps", [(64, 0), (9, 0), (64, 1), (9, 2), (64, 8)])
def test_batched_vjp_matches_cpu_adjoint(K, warps):
    """The batched adjoint (a team of warps per instance; warps 0 = chosen
    from the batch size, 4 for these 29 instances) against the CPU adjoint,
    instance by instance: 1-D instances with 500 cells and sampled kinetics
    (the gradient batch workload), plus mixed sizes down to 33 cells (two
    rows: teams of 8 warps leave warps without rows)."""
    import torch
    import paper_2411_00742_gb300 as P
    insts = pi.adjoint_batch_1d(20) + [x for x in pi.batch_1d(8, seed=77, t_out=pi.loss_times())]
    insts.append(pi.config_1d(33))
    insts[-1].t_out = pi.loss_times()
    b = P.Batch([x.problem for x in insts], [x.C0 for x in insts])
    b.set_state(b.pack([x.n0 for x in insts]))
    b.set_vjp_schedule(warps)
    cols = [1, 2, 3, 4, 5]
    seeds = np.zeros((len(insts), 50, 6))
    wants = []
    for i, inst in enumerate(insts):
        p = inst.problem
        tgt = oracle.solve(p.with_theta(p.theta * pi.TARGET_FACTOR), inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
        r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
        seeds[i] = oracle.relative_loss_seeds(r, tgt, cols)
        wants.append(oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds[i]))
    dn0 = torch.zeros(b.total_cells, dtype=torch.float64, device="cuda")
    dth, dC0 = b.vjp(pi.loss_times(), seeds, K, dn0_out=dn0)
    dn0 = dn0.cpu().numpy()
    b.close()
    for i, (want, wdn0, wdC0) in enumerate(wants):
        for j in (0, 1, 4, 5):
            assert dth[i, j] == pytest.approx(want[j], rel=REL_GRAD, abs=1e-300), (i, j)
        assert dC0[i] == pytest.approx(wdC0, rel=REL_GRAD)
        mine = dn0[b.offsets[i]:b.offsets[i + 1]]
        supp = insts[i].n0 > 1e-3 * insts[i].n0.max()
        assert np.max(np.abs(mine - wdn0)[supp]) <= REL_GRAD * np.max(np.abs(wdn0)), i


def _subnormal_tail(inst):
    """Overwrite the far tail with a halving sequence that runs from 2^-1020
    into subnormal numbers: neighbouring differences of equal sign whose sum
    is too small for its reciprocal to be finite."""
    n0 = inst.n0.copy()
    k = np.arange(n0.size - 150)
    n0[150:] = np.ldexp(1.0, -1020) * 0.5 ** k
    inst.n0 = n0
    return inst


def test_vjp_with_subnormal_tails_matches_cpu_adjoint():
    import paper_2411_00742_gb300 as P
    inst = _subnormal_tail(pi.config_1d(200))
    assert np.any((inst.n0 > 0) & (inst.n0 < np.finfo(np.float64).tiny))
    p, tgt, cols = _setup(inst)
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    seeds = oracle.relative_loss_seeds(r, tgt, cols)
    want, want_dn0, want_dC0 = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    for path in ("plain", "fused"):
        dth, dn0, dC0, rows, _ = _gpu_grad(inst, seeds, 64, path=path)
        assert np.all(np.isfinite(dth)) and np.all(np.isfinite(dn0)), path
        for j in (0, 1, 4, 5):
            assert dth[j] == pytest.approx(want[j], rel=REL_GRAD), (path, j)
        assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD), path
    # the batched adjoint on the same instance
    b = P.Batch([p], [inst.C0])
    b.set_state(b.pack([inst.n0]))
    bth, bC0 = b.vjp(inst.t_out, seeds[None], 64)
    b.close()
    assert np.all(np.isfinite(bth))
    for j in (0, 1, 4, 5):
        assert bth[0, j] == pytest.approx(want[j], rel=REL_GRAD), j
    assert bC0[0] == pytest.approx(want_dC0, rel=REL_GRAD)
