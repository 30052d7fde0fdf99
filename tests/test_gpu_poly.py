"""The polynomial growth law of Eq. 6 on the GPU (the growth model of the
parameter estimation study of Sec. 4.1): forward solves on both paths
against the oracle at the parity tolerances, and the persistent adjoint's
gradient with respect to every coefficient against the oracle's one-pass
adjoint (up to 500 coefficients a direction, the study's 1000 parameters)
and against forward differences of the GPU solve."""
import numpy as np
import pytest

import oracle
import pbe_inputs as pi
from gpu_helpers import assert_n_close, assert_rows_close, gpu_solve

pytestmark = pytest.mark.gpu

REL_GRAD = 1e-6


def _poly_inst(ndim, K, N=40):
    inst = pi.config_1d(N * 5) if ndim == 1 else pi.config_2d(N)
    inst.problem = pi.poly_growth(inst.problem, K)
    return inst


@pytest.mark.parametrize("path", ["plain", "fused"])
@pytest.mark.parametrize("ndim,K", [(1, 1), (1, 7), (2, 3), (2, 50), (2, 500)])
def test_poly_growth_solve_matches_oracle(ndim, K, path):
    inst = _poly_inst(ndim, K)
    want = oracle.solve_instance(inst)
    got = gpu_solve(inst, path=path)
    assert got["steps"] == want["steps"]
    assert_rows_close(got["rows"], want["rows"])
    assert_n_close(got["n"], want["n"])


def _seeds(inst):
    p = inst.problem
    inst.t_out = pi.loss_times()
    r = oracle.solve(p, inst.n0, inst.C0, 0.0, inst.t_out)["rows"]
    tgt = r.copy()
    tgt[:, 1:] *= 1.05
    cols = [1, 2, 3, 4, 5] if p.ndim == 1 else [1, 2, 3, 9, 11]
    return oracle.relative_loss_seeds(r, tgt, cols), tgt, cols


@pytest.mark.parametrize("ndim,K,Kc", [(1, 5, 64), (2, 4, 64), (2, 20, 7), (2, 500, 64)])
def test_poly_growth_gradient_matches_oracle_adjoint(ndim, K, Kc):
    import paper_2411_00742_gb300 as P
    inst = _poly_inst(ndim, K)
    seeds, _, _ = _seeds(inst)
    want_th, want_dn0, want_dC0, want_da = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds)
    g = P.Grid.from_problem(inst.problem, path="fused")
    g.set_state(inst.n0, inst.C0, 0.0)
    dth, _, dC0 = g.vjp(inst.t_out, seeds, Kc)
    da = g.growth_poly_grad()
    g.close()
    for j in (4, 5):
        assert dth[j] == pytest.approx(want_th[j], rel=REL_GRAD), j
    assert dC0 == pytest.approx(want_dC0, rel=REL_GRAD)
    # every coefficient; the high-order terms' gradients are tiny (s^k), compare
    # to the largest entry of each direction as well as element-wise where large
    da, want_da = da.reshape(ndim, K), want_da.reshape(ndim, K)
    for m in range(ndim):
        scale = np.max(np.abs(want_da[m]))
        err = np.abs(da[m] - want_da[m])
        assert np.all(err <= REL_GRAD * np.maximum(np.abs(want_da[m]), 1e-9 * scale)), (m, np.max(err / scale))


def test_poly_growth_gradient_matches_forward_differences_of_the_gpu_solve():
    """The paper's ND: one forward solve per perturbed coefficient."""
    import paper_2411_00742_gb300 as P
    import dataclasses
    inst = _poly_inst(2, 4)
    seeds, tgt, cols = _seeds(inst)
    p = inst.problem

    def loss(a):
        pp = dataclasses.replace(p, poly=tuple(a))
        g = P.Grid.from_problem(pp, path="fused")
        g.set_state(inst.n0, inst.C0, 0.0)
        rows, steps = g.solve(inst.t_out)
        g.close()
        return oracle.relative_loss(rows, tgt, cols), steps

    g = P.Grid.from_problem(p, path="fused")
    g.set_state(inst.n0, inst.C0, 0.0)
    g.vjp(inst.t_out, seeds, 64)
    da = g.growth_poly_grad()
    g.close()
    a0 = np.array(p.poly)
    L0, s0 = loss(a0)
    for k in (0, 1, 4, 6):
        h = 1e-6 * abs(a0[k])
        ap, am = a0.copy(), a0.copy()
        ap[k] += h
        am[k] -= h
        (Lp, sp), (Lm, sm) = loss(ap), loss(am)
        assert sp == sm == s0
        assert da[k] == pytest.approx((Lp - Lm) / (2 * h), rel=1e-5), k


def test_poly_growth_rejected_where_unsupported():
    import paper_2411_00742_gb300 as P
    from paper_2411_00742_gb300 import _lib
    inst = _poly_inst(2, 3)
    seeds, _, _ = _seeds(inst)
    g = P.Grid.from_problem(inst.problem, path="plain")
    g.set_state(inst.n0, inst.C0, 0.0)
    with pytest.raises(_lib.PbeError) as ei:
        g.vjp(inst.t_out, seeds, 64)
    assert "EINVAL" in str(ei.value)
    g.close()
    # growth_form 2 without coefficients
    g = P.Grid(2, (8, 8), (500.0, 500.0))
    k = P.kinetics_struct(inst.problem)
    assert g.lib.pbe_set_kinetics(g.h, __import__("ctypes").byref(k)) == _lib.PBE_ESTATE
    g.close()
