"""Benchmark of the PBE finite-volume solver on GB300.

One benchmark step = one full solve of the 2-D size-and-shape crystallization
problem (256 x 256 cells on [0, 500]^2 um, Gaussian seed, power-law growth and
nucleation, cooling 40 -> 20 C over 3600 s, 61 output rows) - the whole hot
path: kinetics, CFL step, limited fluxes, nucleation inflow, SSP-RK2 update,
moment reduction and solute balance, repeated to every output time.

Metric: FVM cell-steps/s (cells x SSP-RK2 steps / second) of the fused path,
with the plain path reported beside it.  ``--impl reference`` times the CPU
oracle on the same workload instead (the comparison arm).

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torchrun each rank runs its own replica (the 2-D grid is not sharded).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import pbe_inputs as pi  # noqa: E402

METRIC = "FVM cell-steps/s and adjoint grads/s, fused vs plain GPU, at stated FP64 error"
# algorithmic FP64 operations per cell-step of the 2-D SSP-RK2 step (FMA = 2,
# division = 1): per stage two faces (difference, sum, division, FMA = 5 each),
# update (2 differences + 2 FMA = 6), volume moment (FMA = 2); stage 2 adds the
# Runge-Kutta average (3): 18 + 21 = 39.
FLOPS_PER_CELL_STEP_2D = 39
# 1-D: per stage one face (5), the update (difference + FMA = 3) and the volume
# moment (FMA = 2) = 10; two stages and the Runge-Kutta average (3): 23
FLOPS_PER_CELL_STEP_1D = 23
# the paper's split scheme (Eq. 3, two sweeps): per direction and cell one
# difference, one sum, one division, one product, the face value (FMA = 2), the
# flux difference and the update (FMA = 2) = 9; two directions and the volume
# moment (FMA = 2): 20 flops; HBM: read and write the state once = 16 bytes
FLOPS_PER_CELL_STEP_PAPER = 20
BYTES_PER_CELL_STEP_PAPER = 16
FP64_PEAK_TFLOPS_NOMINAL = 1.25  # GB300 dense FP64 (2 FMA/clk/SM x 152 SMs x ~2.07 GHz)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_fused launch on the
# 256 x 256 solve, from one ncu capture of the current kernel (the state stays in L2)
FUSED_DRAM_BYTES_PER_LAUNCH = 595968
L2_FLUSH_BYTES = 256 << 20


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _workload():
    inst = pi.config_2d(256)
    return inst, {"workload": "2-D size-and-shape crystallization, 256x256 cells on [0,500]^2 um, "
                              "full 0-3600 s solve, 61 output rows of (t, mu_pq p+q<=3, C)",
                  "cells": inst.problem.ncell, "grid": [256, 256], "outputs": len(inst.t_out),
                  "l2": "state (0.5 MB/array) stays L2-resident inside a solve; a 256 MB buffer is "
                        "written between timed solves to flush L2"}


def _oracle_rate(inst, budget_s: float, min_reps: int = 1):
    """CPU oracle cell-steps/s on the same workload (single thread)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    reps, cells = 0, 0
    while True:
        r = oracle.solve_instance(inst)
        reps += 1
        cells += inst.problem.ncell * r["steps"]
        el = time.perf_counter() - t0
        if reps >= min_reps and el >= budget_s:
            break
    return cells / el, reps, el, r


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return 0
    inst, cfg = _workload()
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.solve_instance(inst)
    t0 = time.perf_counter()
    cells = 0
    for _ in range(args.steps):
        r = oracle.solve_instance(inst)
        cells += inst.problem.ncell * r["steps"]
    el = time.perf_counter() - t0
    v = cells / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full solves of the 256x256 workload, single thread"},
            "e2e": {"value": v, "unit": "cell-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    import paper_2411_00742_gb300 as P

    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    inst, cfg = _workload()
    cfg["parallelism"] = f"replicas x{ws}" if ws > 1 else "single GPU"
    n0_dev = torch.as_tensor(inst.n0).to("cuda")
    nrow, ncol = len(inst.t_out), P.ncols(2)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def measure(path):
        g = P.Grid.from_problem(inst.problem, stream=stream, path=path)
        rows = torch.zeros((nrow, ncol), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.set_state(n0_dev, inst.C0, 0.0)
                _, steps = g.solve(inst.t_out, out=rows)
        torch.cuda.synchronize()
        got = rows.cpu().numpy()
        times, ktimes = [], []
        # the library records CUDA events on its stream around the launch that
        # advances the state (the persistent kernel on the fused path)
        g.set_timing(True)
        with torch.cuda.stream(stream):
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.set_state(n0_dev, inst.C0, 0.0)
                _, steps = g.solve(inst.t_out, out=rows)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) * 1e-3)
                ktimes.append(g.kernel_time_ms() * 1e-3)
        g.close()
        return sum(times), steps, got, sum(ktimes) / len(ktimes)

    def e2e(path):
        g = P.Grid.from_problem(inst.problem, stream=stream, path=path)
        n0_host = torch.as_tensor(inst.n0).pin_memory()
        rows_host = torch.zeros((nrow, ncol), dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                g.set_state(n0_host, inst.C0, 0.0)
                g.solve(inst.t_out, out=rows_host)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                g.set_state(n0_host, inst.C0, 0.0)
                _, steps = g.solve(inst.t_out, out=rows_host)
            el = time.perf_counter() - t0
        g.close()
        return inst.problem.ncell * steps * args.steps / el, n0_host.numel() * 8 + nrow * 8, nrow * ncol * 8

    def batch_leg():
        """4096 independent 1-D instances in one persistent launch (autotuned), vs the
        plain single-grid path on a sample of the same instances."""
        insts = pi.batch_1d(4096, seed=2411)
        b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], stream=stream)
        packed = torch.as_tensor(b.pack([x.n0 for x in insts])).to("cuda")
        rows = torch.zeros((len(insts), len(insts[0].t_out), 6), dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            b.set_state(packed)
            wpb = b.autotune(insts[0].t_out)
            for _ in range(args.warmup):
                b.set_state(packed)
                _, bsteps = b.solve(insts[0].t_out, out=rows)
        torch.cuda.synchronize()
        times = []
        with torch.cuda.stream(stream):
            for _ in range(max(2, args.steps // 4)):
                b.set_state(packed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, bsteps = b.solve(insts[0].t_out, out=rows)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) * 1e-3)
        bsteps_cells = b.cell_steps()
        b.close()
        tb = sum(times) / len(times)
        # plain single-grid path, instance by instance, on a sample
        sample = insts[:64]
        g_cells, g_time = 0, 0.0
        with torch.cuda.stream(stream):
            for inst in sample:
                g = P.Grid.from_problem(inst.problem, stream=stream, path="plain")
                g.set_state(torch.as_tensor(inst.n0).cuda(), inst.C0, 0.0)
                g.solve(inst.t_out)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                g.set_state(torch.as_tensor(inst.n0).cuda(), inst.C0, 0.0)
                e0.record(stream)
                _, st = g.solve(inst.t_out)
                e1.record(stream)
                e1.synchronize()
                g.close()
                g_cells += inst.problem.ncell * st
                g_time += e0.elapsed_time(e1) * 1e-3
        return {"instances": len(insts), "warps_per_block": wpb, "total_steps": bsteps,
                "cell_steps": bsteps_cells, "ms_per_solve": 1e3 * tb, "value": bsteps_cells / tb,
                "unit": "cell-steps/s",
                "plain_per_instance": {"value": g_cells / g_time, "sample": "first 64 instances, one grid each"}}

    def loss_seeds(rows, target, cols):
        """dL/drows of the relative-error loss sum_k sum_c ((r - t) / t)^2 (Eq. 5 with
        relative residuals) over the columns `cols`."""
        sd = np.zeros_like(rows)
        sd[..., cols] = 2.0 * (rows[..., cols] - target[..., cols]) / target[..., cols] ** 2
        return sd

    def adjoint_leg():
        """Gradients of the relative-error loss (50 loss times, target = kinetics x1.1) with
        respect to the kinetic parameters: (a) 2-D 128x128 grid, (b) 1-D 500-cell instances.
        One gradient = forward with checkpoints every 64 steps + reverse sweep.  Targets
        and seeds come from GPU solves; the CPU adjoint (timing and agreement) is part of
        the CPU baseline leg."""
        out, cases = {}, {}
        for name, inst, cols in (("2d_128x128", pi.adjoint_2d(128), [1, 2, 3, 9, 11]),
                                 ("1d_500", pi.adjoint_batch_1d(16)[0], [1, 2, 3, 4, 5])):
            p = inst.problem
            gt = P.Grid.from_problem(p.with_theta(p.theta * pi.TARGET_FACTOR), stream=stream)
            gt.set_state(inst.n0, inst.C0, 0.0)
            tgt, _ = gt.solve(inst.t_out)
            gt.close()
            g = P.Grid.from_problem(p, stream=stream)
            n0d = torch.as_tensor(inst.n0).cuda()
            rows = torch.zeros((len(inst.t_out), P.ncols(p.ndim)), dtype=torch.float64, device="cuda")
            tgt_t = torch.as_tensor(tgt).cuda()
            times = []
            with torch.cuda.stream(stream):
                for it in range(args.warmup + max(3, args.steps // 2)):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    g.set_state(n0d, inst.C0, 0.0)
                    e0.record(stream)
                    g.solve(inst.t_out, out=rows)
                    sd = torch.zeros_like(rows)
                    sd[:, cols] = 2.0 * (rows[:, cols] - tgt_t[:, cols]) / tgt_t[:, cols] ** 2
                    g.set_state(n0d, inst.C0, 0.0)
                    dth, _, _ = g.vjp(inst.t_out, sd, 64)
                    e1.record(stream)
                    e1.synchronize()
                    if it >= args.warmup:
                        times.append(e0.elapsed_time(e1) * 1e-3)
            g.close()
            tg = sum(times) / len(times)
            out[name] = {"grads_per_s": 1.0 / tg, "ms_per_grad": 1e3 * tg, "max_rel_err_vs_cpu_adjoint": None,
                         "cpu_adjoint_grads_per_s": None, "checkpoint_every": 64}
            cases[name] = (inst, tgt, cols, dth, sd.cpu().numpy())
        # (b') the batched form: 256 instances of 500 cells, one launch (one warp per instance)
        insts = pi.adjoint_batch_1d(256)
        cols = [1, 2, 3, 4, 5]
        bt = P.Batch([x.problem.with_theta(x.problem.theta * pi.TARGET_FACTOR) for x in insts],
                     [x.C0 for x in insts], stream=stream)
        bt.set_state(bt.pack([x.n0 for x in insts]))
        tgts, _ = bt.solve(pi.loss_times())
        bt.close()
        b = P.Batch([x.problem for x in insts], [x.C0 for x in insts], stream=stream)
        packed = b.pack([x.n0 for x in insts])
        b.set_state(packed)
        fwd, _ = b.solve(pi.loss_times())
        seeds = loss_seeds(fwd, tgts, cols)
        seeds_d = torch.as_tensor(seeds).cuda()
        times = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + max(3, args.steps // 2)):
                b.set_state(packed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dth_b, _ = b.vjp(pi.loss_times(), seeds_d, 64)
                e1.record(stream)
                e1.synchronize()
                if it >= args.warmup:
                    times.append(e0.elapsed_time(e1) * 1e-3)
        b.close()
        tb = sum(times) / len(times)
        out["batch_1d_256x500"] = {"grads_per_s": 256 / tb, "ms_per_batch": 1e3 * tb,
                                   "max_rel_err_vs_cpu_adjoint_sampled": None, "checkpoint_every": 64,
                                   "single_instance_path_grads_per_s": out["1d_500"]["grads_per_s"],
                                   "cpu_adjoint_grads_per_s": None}
        cases["batch_1d_256x500"] = (insts, seeds, dth_b)
        return out, cases

    def adjoint_cpu_baseline(adj, cases):
        """The CPU adjoint of the oracle on the same seeds: its gradients/s and the
        agreement of the GPU gradients (part of the CPU baseline leg)."""
        import oracle
        for name in ("2d_128x128", "1d_500"):
            inst, tgt, cols, dth, sd = cases[name]
            p = inst.problem
            idx = [0, 1, 4, 5] if p.ndim == 1 else list(range(6))
            t0 = time.perf_counter()
            want, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, sd)
            tc = time.perf_counter() - t0
            adj[name]["max_rel_err_vs_cpu_adjoint"] = float(np.max(np.abs(dth[idx] - want[idx]) / np.abs(want[idx])))
            adj[name]["cpu_adjoint_grads_per_s"] = 1.0 / tc
        insts, seeds, dth_b = cases["batch_1d_256x500"]
        errs = []
        for i in range(0, 256, 32):
            inst = insts[i]
            want, _, _ = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds[i])
            errs.append(float(np.max(np.abs(dth_b[i, [0, 1, 4, 5]] - want[[0, 1, 4, 5]]) / np.abs(want[[0, 1, 4, 5]]))))
        adj["batch_1d_256x500"]["max_rel_err_vs_cpu_adjoint_sampled"] = max(errs)
        adj["batch_1d_256x500"]["cpu_adjoint_grads_per_s"] = adj["1d_500"]["cpu_adjoint_grads_per_s"]

    def paper_leg():
        """The paper's own base case (Table 1, Appendix A) at its finest bins: 6000 x 3000
        (0.04 um^2), Eq. 3 with Godunov splitting at Courant number 0.9, one hour."""
        inst = pi.paper_base_case(6000)
        g = P.Grid.from_problem(inst.problem, stream=stream, path="plain")
        n0d = torch.as_tensor(inst.n0).cuda()
        times, ktimes, steps = [], [], 0
        g.set_timing(True)
        with torch.cuda.stream(stream):
            for it in range(1 + max(1, args.steps // 5)):
                g.set_state(n0d, inst.C0, 0.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, steps = g.solve(inst.t_out)
                e1.record(stream)
                e1.synchronize()
                if it >= 1:
                    times.append(e0.elapsed_time(e1) * 1e-3)
                    ktimes.append(g.kernel_time_ms() * 1e-3)
        g.close()
        tp = sum(times) / len(times)
        rate = inst.problem.ncell * steps / tp
        # per launch of the step kernel: the graph's device time / steps
        k_launch = sum(ktimes) / len(ktimes) / steps
        achieved = FLOPS_PER_CELL_STEP_PAPER * inst.problem.ncell / k_launch / 1e12
        return {"workload": "paper base case, 6000x3000 bins on 1200x600 um, T = 15 C, 1 h, Eq. 3 + splitting",
                "steps": steps, "paper_reported_steps": 1339, "s_per_solve": tp,
                "value": rate, "unit": "cell-steps/s",
                "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                             "frac": achieved / FP64_PEAK_TFLOPS_NOMINAL,
                             "hbm_gbs": BYTES_PER_CELL_STEP_PAPER * inst.problem.ncell / k_launch / 1e9,
                             "kernel": "k_lw_step2d (one kernel per step, both sweeps)",
                             "launch_ms": 1e3 * k_launch,
                             "note": f"{FLOPS_PER_CELL_STEP_PAPER} algorithmic FP64 flop/cell-step (division = 1) x "
                                     "cells per launch / launch time (CUDA events around the step graph / steps); "
                                     "peak = nominal GB300 FP64"},
                "paper_context": "JAX (GPU) on an RTX 4090 in FP64: 'almost 3x as fast' as a 1.2 s MATLAB run "
                                 "(Sec. 3.2): about 0.4 s read as total time, about 2.3 s read per time step"}

    def small_1d_leg():
        """The small 1-D case (200 cells, the oracle-sized workload): latency-bound,
        reported as solves/s and microseconds per step on both paths, against the
        oracle on the same solve."""
        sinst = pi.config_1d(200)
        n0s = torch.as_tensor(sinst.n0).cuda()
        rows1 = torch.zeros((len(sinst.t_out), P.ncols(1)), dtype=torch.float64, device="cuda")
        out = {"workload": "1-D 200 cells on [0, 1000] um, full 0-3600 s solve, 61 output rows"}
        for path in ("fused", "plain"):
            g = P.Grid.from_problem(sinst.problem, stream=stream, path=path)
            times, nsteps = [], 0
            with torch.cuda.stream(stream):
                for it in range(3 + max(5, args.steps)):
                    g.set_state(n0s, sinst.C0, 0.0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    _, nsteps = g.solve(sinst.t_out, out=rows1)
                    e1.record(stream)
                    e1.synchronize()
                    if it >= 3:
                        times.append(e0.elapsed_time(e1) * 1e-3)
            g.close()
            t = sum(times) / len(times)
            out[path] = {"solves_per_s": 1.0 / t, "us_per_step": 1e6 * t / nsteps, "steps": nsteps,
                         "value": sinst.problem.ncell * nsteps / t, "unit": "cell-steps/s",
                         "max_rel_err_vs_oracle": None, "rows": rows1.cpu().numpy()}
        return out

    def scaling_leg():
        """Grid-size sweep (the paper's Fig. 3b analogue) on the fused and plain paths:
        full 2-D solves at 512^2, 1024^2 and 2048^2, and 1-D solves of 2^18 and 2^20
        cells over a 10 s horizon."""
        out = []
        for N in (512, 1024, 2048):
            sinst = pi.config_2d(N)
            n0s = torch.as_tensor(sinst.n0).cuda()
            row = {"grid": [N, N], "cells": N * N}
            for path in ("fused", "plain"):
                g = P.Grid.from_problem(sinst.problem, stream=stream, path=path)
                times, nsteps = [], 0
                with torch.cuda.stream(stream):
                    for it in range(3 if N < 2048 else 2):
                        g.set_state(n0s, sinst.C0, 0.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        _, nsteps = g.solve(sinst.t_out)
                        e1.record(stream)
                        e1.synchronize()
                        if it >= 1:
                            times.append(e0.elapsed_time(e1) * 1e-3)
                g.close()
                t = min(times)
                rate = N * N * nsteps / t
                row["steps"] = nsteps
                row[path] = {"ms_per_solve": 1e3 * t, "value": rate, "unit": "cell-steps/s",
                             "roofline_frac": FLOPS_PER_CELL_STEP_2D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL}
            out.append(row)
        out1 = []
        # 1-D: 2^18 and 2^20 cells (dL ~ 4e-3 / 1e-3 um), 10 s from a supersaturated
        # start (S = 1.5): every step CFL-limited
        for N in (1 << 18, 1 << 20):
            sinst = pi.config_1d_fine(N)
            n0s = torch.as_tensor(sinst.n0).cuda()
            row = {"grid": [N], "cells": N, "horizon_s": float(sinst.t_out[-1])}
            for path in ("fused", "plain"):
                g = P.Grid.from_problem(sinst.problem, stream=stream, path=path)
                times, nsteps = [], 0
                with torch.cuda.stream(stream):
                    for it in range(3):
                        g.set_state(n0s, sinst.C0, 0.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        _, nsteps = g.solve(sinst.t_out)
                        e1.record(stream)
                        e1.synchronize()
                        if it >= 1:
                            times.append(e0.elapsed_time(e1) * 1e-3)
                g.close()
                t = min(times)
                rate = N * nsteps / t
                row["steps"] = nsteps
                row[path] = {"ms_per_solve": 1e3 * t, "value": rate, "unit": "cell-steps/s",
                             "roofline_frac": FLOPS_PER_CELL_STEP_1D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL}
            out1.append(row)
        return out, out1

    clocks = ClockSampler(dev)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_fused, steps, rows_fused, k_fused = measure("fused")
    t_plain, steps_p, rows_plain, _ = measure("plain")
    clk = clocks.stop()
    e2e_rate, h2d, d2h = e2e("fused")
    batch = batch_leg() if not args.no_batch else None
    adjoint, adjoint_cases = adjoint_leg() if not args.no_adjoint else (None, None)
    paper = paper_leg() if not args.no_paper else None
    scaling, scaling_1d = scaling_leg() if not args.no_scaling else (None, None)
    small_1d = small_1d_leg() if not args.no_scaling else None

    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([t_fused, t_plain], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_fused, t_plain = tt.tolist()
    cells_per_solve = inst.problem.ncell * steps
    value = ws * cells_per_solve * args.steps / t_fused
    plain_value = ws * cells_per_solve * args.steps / t_plain
    ms = 1e3 * t_fused / args.steps
    achieved = FLOPS_PER_CELL_STEP_2D * cells_per_solve / k_fused / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "cell-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
        "ssp_rk2_steps_per_solve": steps,
        "paths": {"fused": {"value": value, "ms_per_solve": ms, "max_rel_err_vs_oracle": None},
                  "plain": {"value": plain_value, "ms_per_solve": 1e3 * t_plain / args.steps,
                            "max_rel_err_vs_oracle": None}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS_NOMINAL,
                     "traffic": FUSED_DRAM_BYTES_PER_LAUNCH if inst.problem.ncells == (256, 256) else None,
                     "kernel": "k_fused (persistent cooperative kernel, one launch per solve)",
                     "launch_ms": 1e3 * k_fused,
                     "note": f"FP64 algorithmic {FLOPS_PER_CELL_STEP_2D} flop/cell-step (division = 1) x "
                             "cell-steps per launch / launch time (CUDA events the library records around the "
                             "launch on its stream, mean over the timed solves); peak = nominal GB300 FP64"},
        "e2e": {"value": ws * e2e_rate, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "batch_1d": batch,
        "small_1d": small_1d,
        "adjoint": adjoint,
        "paper_scheme": paper,
        "scaling_2d": scaling,
        "scaling_1d": scaling_1d,
        # per timed fused solve: k_set_scalars, k_prologue, k_fused, k_fused_rows
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu_baseline:
        # the CPU baseline leg: the oracle timed on the host, and its rows give the
        # stated error of the GPU rows on the same solves
        v, reps, el, want = _oracle_rate(inst, budget_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{reps} full solves of the same 256x256 workload ({el:.1f} s), single thread"}

        def rel_err(got, ref):
            return float(np.max(np.abs(got[:, 1:] - ref["rows"][:, 1:]) / np.abs(ref["rows"][:, 1:])))

        line["paths"]["fused"]["max_rel_err_vs_oracle"] = rel_err(rows_fused, want)
        line["paths"]["plain"]["max_rel_err_vs_oracle"] = rel_err(rows_plain, want)
        if adjoint is not None:
            adjoint_cpu_baseline(adjoint, adjoint_cases)
        if small_1d is not None:
            import oracle
            want1 = oracle.solve_instance(pi.config_1d(200))
            for path in ("fused", "plain"):
                small_1d[path]["max_rel_err_vs_oracle"] = rel_err(small_1d[path]["rows"], want1)
    if small_1d is not None:
        for path in ("fused", "plain"):
            small_1d[path].pop("rows")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-paper", action="store_true")
    ap.add_argument("--no-scaling", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
