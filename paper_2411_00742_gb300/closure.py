"""Training and evaluation of the learned kinetics closure through the solver.

The closure (a 3-64-64-3 perceptron replacing the growth and nucleation
expressions, the empirical hybrid model of Sec. 4.2) is trained by gradient
descent through the differentiable solver.  One minibatch: for every
trajectory a forward solve and the persistent discrete adjoint (pbe_vjp on the
fused path), which backpropagates through the closure inside every stage and
records each closure evaluation; then one launch of the weight-gradient kernel
over the whole minibatch's evaluations (pbe_closure_grad, tensor cores); the
optimizer is Adam (pbe_adam_update) on device arrays.  The trajectories of a
minibatch run concurrently, one CUDA stream and grid each.  This module only
orchestrates calls into the CUDA library.
"""
from __future__ import annotations

import ctypes
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from . import CLOSURE_SIZE, Grid, _lib, closure_grad

LOSS_COLS_2D = [1, 2, 3, 9, 11]   # mu00, mu10, mu01, mu12, C
LOSS_COLS_1D = [1, 2, 3, 4, 5]


def loss_cols(ndim):
    return LOSS_COLS_1D if ndim == 1 else LOSS_COLS_2D


def relative_loss_and_seeds(rows, target, cols):
    r = (rows[:, cols] - target[:, cols]) / target[:, cols]
    seeds = np.zeros_like(rows)
    seeds[:, cols] = 2.0 * r / target[:, cols]
    return float(np.sum(r * r)), seeds


class _Worker:
    def __init__(self, problem, path="plain", block_limit=0):
        self.stream = torch.cuda.Stream()
        self.grid = Grid.from_problem(problem, stream=self.stream, path=path)
        if block_limit:
            self.grid.set_block_limit(block_limit)

    def grad_rows(self, inst, target, weights, cols, checkpoint_every=64):
        """Loss of one trajectory and its adjoint (fused path): the closure
        evaluations it differentiates stay recorded in the grid for
        closure_grad."""
        g = self.grid
        g.set_closure(weights)
        g.set_kinetics(inst.problem, closure=True)
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        rows, _ = g.solve(inst.t_out)
        L, seeds = relative_loss_and_seeds(rows, target, cols)
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        g.vjp(inst.t_out, seeds, checkpoint_every)
        return L

    def grad(self, inst, target, weights, cols, checkpoint_every=64):
        g = self.grid
        g.set_closure(weights)
        g.set_kinetics(inst.problem, closure=True)
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        rows, _ = g.solve(inst.t_out)
        L, seeds = relative_loss_and_seeds(rows, target, cols)
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        dW = np.zeros(CLOSURE_SIZE)
        g.vjp(inst.t_out, seeds, checkpoint_every, dweights_out=dW)
        return L, dW

    def rows(self, inst, weights=None, problem=None):
        g = self.grid
        if weights is not None:
            g.set_closure(weights)
            g.set_kinetics(inst.problem, closure=True)
        else:
            g.set_kinetics(problem if problem is not None else inst.problem)
        g.set_state(np.ascontiguousarray(inst.n0), inst.C0, inst.t0)
        rows, _ = g.solve(inst.t_out)
        return rows


class ClosureTrainer:
    """Adam on the closure weights through the solver's adjoint."""

    def __init__(self, w0, problem_like, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, workers=8, grid_blocks=None):
        """grid_blocks: the block limit of each trajectory's grid (default: the
        SMs shared by the `workers` concurrent trajectories, so that their
        cooperative launches run side by side; 0 = one block per SM)."""
        self.lib = _lib.load()
        if grid_blocks is None:
            grid_blocks = max(8, torch.cuda.get_device_properties(0).multi_processor_count // workers)
        self.grid_blocks = grid_blocks
        self.w = torch.as_tensor(np.asarray(w0, dtype=np.float64)).cuda()
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.lr, self.betas, self.eps = lr, betas, eps
        self.step_count = 0
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self._local = threading.local()
        self._problem = problem_like
        self.workers = []
        self.slots = []   # one fused-path grid per minibatch trajectory
        self._lock = threading.Lock()

    def _worker(self):
        w = getattr(self._local, "w", None)
        if w is None:
            w = _Worker(self._problem, path="fused", block_limit=self.grid_blocks)
            self._local.w = w
            with self._lock:
                self.workers.append(w)
        return w

    def weights32(self):
        return self.w.float().cpu().numpy()

    def batch_grad(self, insts, targets):
        """Mean loss and mean weight gradient of a minibatch: the trajectories'
        solves and adjoints on concurrent streams (one fused-path grid each),
        then one weight-gradient launch over all their closure evaluations."""
        w32 = self.weights32()
        cols = loss_cols(insts[0].problem.ndim)
        n = len(insts)
        while len(self.slots) < n:
            self.slots.append(_Worker(self._problem, path="fused", block_limit=self.grid_blocks))
        Ls = list(self.pool.map(lambda i: self.slots[i].grad_rows(insts[i], targets[i], w32, cols), range(n)))
        g = closure_grad([sl.grid for sl in self.slots[:n]]) / n
        return float(np.mean(Ls)), g

    def step(self, insts, targets):
        L, g = self.batch_grad(insts, targets)
        gt = torch.as_tensor(g).cuda()
        self.step_count += 1
        torch.cuda.synchronize()
        _lib.check(self.lib.pbe_adam_update(ctypes.c_void_p(self.w.data_ptr()), ctypes.c_void_p(gt.data_ptr()),
                                            ctypes.c_void_p(self.m.data_ptr()), ctypes.c_void_p(self.v.data_ptr()),
                                            self.w.numel(), self.lr, self.betas[0], self.betas[1], self.eps,
                                            self.step_count, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
        torch.cuda.synchronize()
        return L

    def rows(self, insts, weights=None, problems=None):
        w32 = None if weights is None else np.asarray(weights, dtype=np.float32)
        probs = problems if problems is not None else [None] * len(insts)
        return list(self.pool.map(lambda it: self._worker().rows(it[0], w32, it[1]), zip(insts, probs)))

    def close(self):
        self.pool.shutdown()
        for w in self.workers + self.slots:
            w.grid.close()


def trajectory_error(rows, target, cols):
    """Relative RMS error of the chosen columns over all output times."""
    r = (rows[:, cols] - target[:, cols]) / target[:, cols]
    return float(np.sqrt(np.mean(r * r)))
