"""torch.autograd.Function over the solver: forward = pbe_solve, backward =
pbe_vjp (the hand-written discrete adjoint with checkpointing).  Argument
marshalling only; all arithmetic runs in the CUDA library."""
from __future__ import annotations

import numpy as np
import torch

from . import Grid, ncols


class PBESolve(torch.autograd.Function):
    """rows = PBESolve.apply(theta, n0, grid, problem, C0, t0, t_out, checkpoint_every)

    theta: float64 tensor (kg1, g1, kg2, g2, kb, b); n0: float64 CUDA tensor
    with the grid's shape; returns the output rows (t, moments, C) as a CUDA
    tensor.  Gradients flow to theta and n0."""

    @staticmethod
    def forward(ctx, theta, n0, grid: Grid, problem, C0: float, t0: float, t_out, checkpoint_every: int = 64):
        th = theta.detach().double().cpu().numpy()
        grid.set_kinetics(problem, theta=th)
        n0c = n0.detach().contiguous()
        grid.set_state(n0c, C0, t0)
        rows = torch.zeros((len(t_out), ncols(grid.ndim)), dtype=torch.float64, device=n0.device)
        grid.solve(np.asarray(t_out, dtype=np.float64), out=rows)
        ctx.save_for_backward(theta, n0c)
        ctx.grid, ctx.problem, ctx.C0, ctx.t0 = grid, problem, C0, t0
        ctx.t_out, ctx.K = np.asarray(t_out, dtype=np.float64), int(checkpoint_every)
        return rows

    @staticmethod
    def backward(ctx, grad_rows):
        theta, n0 = ctx.saved_tensors
        g = ctx.grid
        g.set_kinetics(ctx.problem, theta=theta.detach().double().cpu().numpy())
        g.set_state(n0, ctx.C0, ctx.t0)
        dn0 = torch.zeros_like(n0) if ctx.needs_input_grad[1] else None
        dth, _, _ = g.vjp(ctx.t_out, grad_rows.detach().contiguous().double(), ctx.K, dn0_out=dn0)
        dtheta = torch.as_tensor(dth, dtype=theta.dtype, device=theta.device) if ctx.needs_input_grad[0] else None
        return dtheta, dn0, None, None, None, None, None, None
