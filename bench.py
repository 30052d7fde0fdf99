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
# Algorithmic FP64 work per cell-step of the SSP-RK2 step (FMA = 2, division =
# 1), the counts of the hot-path scope the rooflines use: 1-D 25 flops + 2
# divisions, 2-D 43 flops + 4 divisions.
FLOPS_PER_CELL_STEP_2D = 47
FLOPS_PER_CELL_STEP_1D = 27
# This implementation's own count of the same step (every face value once per
# stage): 2-D per stage two faces (difference, sum, division, FMA = 5 each),
# update (2 differences + 2 FMA = 6), volume moment (FMA = 2), plus the
# Runge-Kutta average (3): 39; 1-D per stage one face (5), update (3), volume
# moment (2), plus the average: 23.  Reported beside the scope's counts.
OWN_FLOPS_PER_CELL_STEP_2D = 39
OWN_FLOPS_PER_CELL_STEP_1D = 23
# Work of one gradient (the scope's model): the forward pass, the recomputed
# segments, and a reverse sweep of about 2.5 times the forward's flops.
ADJOINT_REVERSE_FACTOR = 2.5
# the paper's split scheme (Eq. 3, two sweeps): per direction and cell one
# difference, one sum, one division, one product, the face value (FMA = 2), the
# flux difference and the update (FMA = 2) = 9; two directions and the volume
# moment (FMA = 2): 20 flops; HBM: read and write the state once = 16 bytes
FLOPS_PER_CELL_STEP_PAPER = 20
BYTES_PER_CELL_STEP_PAPER = 16
FP64_PEAK_TFLOPS_NOMINAL = 1.25  # GB300 dense FP64 (2 FMA/clk/SM x 152 SMs x ~2.07 GHz)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_fused launch on the
# 256 x 256 solve, from one ncu capture of the current kernel (the state stays in L2)
FUSED_DRAM_BYTES_PER_LAUNCH = 605440
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
                 "-lms", "25"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def _host_info():
    """Core count and CPU model of the host the CPU baseline ran on."""
    info = {"nproc": os.cpu_count()}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip() in ("Model name", "Architecture", "Socket(s)", "Core(s) per socket", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except Exception:  # lscpu missing: the core count alone
        pass
    return info


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
        wpb, nteam, wcells = b.schedule()
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
        ach = FLOPS_PER_CELL_STEP_1D * bsteps_cells / tb / 1e12
        return {"instances": len(insts), "schedule": {"warps_per_block": wpb, "team_instances": nteam,
                                                      "warp_cells": wcells}, "total_steps": bsteps,
                "cell_steps": bsteps_cells, "ms_per_solve": 1e3 * tb, "value": bsteps_cells / tb,
                "unit": "cell-steps/s",
                "plain_per_instance": {"value": g_cells / g_time, "sample": "first 64 instances, one grid each"},
                "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                             "frac": ach / FP64_PEAK_TFLOPS_NOMINAL,
                             "own_count_frac": OWN_FLOPS_PER_CELL_STEP_1D * bsteps_cells / tb / 1e12 /
                             FP64_PEAK_TFLOPS_NOMINAL,
                             "kernel": "batched 1-D kernel (a warp per instance, a block per costly instance; one graph launch "
                                       "per batch)",
                             "note": f"{FLOPS_PER_CELL_STEP_1D} flop/cell-step x cell-steps / batch time (CUDA events "
                                     "around the graph launch); peak = nominal GB300 FP64"},
                "_insts": insts}

    def loss_seeds(rows, target, cols):
        """dL/drows of the relative-error loss sum_k sum_c ((r - t) / t)^2 (Eq. 5 with
        relative residuals) over the columns `cols`."""
        sd = np.zeros_like(rows)
        sd[..., cols] = 2.0 * (rows[..., cols] - target[..., cols]) / target[..., cols] ** 2
        return sd

    def adjoint_leg():
        """Gradients of the relative-error loss (50 loss times, target = kinetics x1.1) with
        respect to the kinetic parameters on both paths - fused: the persistent adjoint
        (forward, recomputation and reverse sweep in one launch), plain: per-stage kernels
        - for (a) the 2-D 128x128 grid, (b) one 1-D 500-cell instance, and (b') 256 such
        instances in one batched launch.  One gradient = one pbe_vjp with a checkpoint
        every 64 steps; its seeds dL/drows come from a GPU solve beforehand.  The CPU
        adjoint (timing and agreement) is part of the CPU baseline leg."""
        out, cases = {}, {}
        K = 64
        reps = max(3, args.steps // 2)
        for name, inst, cols in (("2d_128x128", pi.adjoint_2d(128), [1, 2, 3, 9, 11]),
                                 ("1d_500", pi.adjoint_batch_1d(16)[0], [1, 2, 3, 4, 5])):
            p = inst.problem
            gt = P.Grid.from_problem(p.with_theta(p.theta * pi.TARGET_FACTOR), stream=stream)
            gt.set_state(inst.n0, inst.C0, 0.0)
            tgt, _ = gt.solve(inst.t_out)
            gt.close()
            g = P.Grid.from_problem(p, stream=stream)
            g.set_state(inst.n0, inst.C0, 0.0)
            rows, steps = g.solve(inst.t_out)
            g.close()
            sd = loss_seeds(rows, tgt, cols)
            sd_d = torch.as_tensor(sd).cuda()
            n0d = torch.as_tensor(inst.n0).cuda()
            fpc = FLOPS_PER_CELL_STEP_1D if p.ndim == 1 else FLOPS_PER_CELL_STEP_2D
            nseg = -(-steps // K)
            recomputed = steps - (steps - (nseg - 1) * K)
            flops = (1.0 + recomputed / steps + ADJOINT_REVERSE_FACTOR) * fpc * p.ncell * steps
            res = {"steps": steps, "checkpoint_every": K, "recomputed_steps": recomputed,
                   "max_rel_err_vs_cpu_adjoint": None, "cpu_adjoint_grads_per_s": None}
            for path in ("fused", "plain"):
                g = P.Grid.from_problem(p, stream=stream, path=path)
                g.set_timing(True)
                times, ktimes = [], []
                with torch.cuda.stream(stream):
                    for it in range(args.warmup + reps):
                        g.set_state(n0d, inst.C0, 0.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        dth, _, _ = g.vjp(inst.t_out, sd_d, K)
                        e1.record(stream)
                        e1.synchronize()
                        if it >= args.warmup:
                            times.append(e0.elapsed_time(e1) * 1e-3)
                            ktimes.append(g.kernel_time_ms() * 1e-3)
                g.close()
                tg = sum(times) / len(times)
                entry = {"grads_per_s": 1.0 / tg, "ms_per_grad": 1e3 * tg}
                if path == "fused":
                    kt = sum(ktimes) / len(ktimes)
                    ach = flops / kt / 1e12
                    entry["roofline"] = {
                        "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS_NOMINAL, "unit": "TFLOP/s",
                        "frac": ach / FP64_PEAK_TFLOPS_NOMINAL, "launch_ms": 1e3 * kt,
                        "kernel": "k_adjoint_persistent (one cooperative launch per gradient)",
                        "note": f"(1 + recomputed/steps + {ADJOINT_REVERSE_FACTOR}) x {fpc} flop/cell-step x "
                                "cells x steps / launch time (CUDA events around the launch on its stream); "
                                "peak = nominal GB300 FP64"}
                    res["dth"] = dth
                res[path] = entry
            res["value"] = res["fused"]["grads_per_s"]
            res["unit"] = "grads/s"
            res["fused_over_plain"] = res["fused"]["grads_per_s"] / res["plain"]["grads_per_s"]
            out[name] = res
            cases[name] = (inst, tgt, cols, res.pop("dth"), sd)
        # (b') the batched form: 256 instances of 500 cells, one launch (a team of warps per instance)
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
        bcells = b.cell_steps()
        bsteps = b.steps()
        seeds = loss_seeds(fwd, tgts, cols)
        seeds_d = torch.as_tensor(seeds).cuda()
        times = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + reps):
                b.set_state(packed)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                dth_b, _ = b.vjp(pi.loss_times(), seeds_d, K)
                e1.record(stream)
                e1.synchronize()
                if it >= args.warmup:
                    times.append(e0.elapsed_time(e1) * 1e-3)
        b.close()
        tb = sum(times) / len(times)
        rec = float(sum(max(0, int(s_) - (int(s_) - ((-(-int(s_) // K)) - 1) * K)) * x.problem.ncell
                        for s_, x in zip(bsteps, insts)))
        bflops = (bcells * (1.0 + ADJOINT_REVERSE_FACTOR) + rec) * FLOPS_PER_CELL_STEP_1D
        bach = bflops / tb / 1e12
        out["batch_1d_256x500"] = {"grads_per_s": 256 / tb, "ms_per_batch": 1e3 * tb, "value": 256 / tb,
                                   "unit": "grads/s", "cell_steps": bcells,
                                   "max_rel_err_vs_cpu_adjoint_sampled": None, "checkpoint_every": K,
                                   "single_instance_fused_grads_per_s": out["1d_500"]["fused"]["grads_per_s"],
                                   "cpu_adjoint_grads_per_s": None,
                                   "roofline": {"bound": "alu", "achieved": bach, "peak": FP64_PEAK_TFLOPS_NOMINAL,
                                                "unit": "TFLOP/s", "frac": bach / FP64_PEAK_TFLOPS_NOMINAL,
                                                "kernel": "batched adjoint (a team of warps per instance, one launch)",
                                                "note": f"((1 + {ADJOINT_REVERSE_FACTOR}) x cell-steps + recomputed "
                                                        f"cell-steps) x {FLOPS_PER_CELL_STEP_1D} flop / batch time "
                                                        "(CUDA events around the call); peak = nominal GB300 FP64"}}
        cases["batch_1d_256x500"] = (insts, seeds, dth_b)
        return out, cases

    def adjoint_cpu_baseline(adj, cases, cores):
        """The CPU adjoint of the oracle on the same seeds: its gradients/s (one thread,
        and on every core - rows in parallel for one grid, instances in parallel for
        the batch) and the agreement of the fused GPU gradients (part of the CPU
        baseline leg)."""
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        for name in ("2d_128x128", "1d_500"):
            inst, tgt, cols, dth, sd = cases[name]
            p = inst.problem
            idx = [0, 1, 4, 5] if p.ndim == 1 else list(range(6))
            t0 = time.perf_counter()
            want, _, _ = oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, sd)
            tc = time.perf_counter() - t0
            adj[name]["max_rel_err_vs_cpu_adjoint"] = float(np.max(np.abs(dth[idx] - want[idx]) / np.abs(want[idx])))
            adj[name]["cpu_adjoint_grads_per_s"] = 1.0 / tc
            if p.ncell >= 16384:
                oracle.set_threads(cores)
                t0 = time.perf_counter()
                oracle.vjp(p, inst.n0, inst.C0, 0.0, inst.t_out, sd)
                tm = time.perf_counter() - t0
                oracle.set_threads(1)
                adj[name]["cpu_adjoint_all_cores"] = {"grads_per_s": 1.0 / tm, "threads": cores,
                                                      "sample": "one gradient, rows of the grid in parallel"}
        insts, seeds, dth_b = cases["batch_1d_256x500"]
        errs = []
        for i in range(0, 256, 32):
            inst = insts[i]
            want, _, _ = oracle.vjp(inst.problem, inst.n0, inst.C0, 0.0, inst.t_out, seeds[i])
            errs.append(float(np.max(np.abs(dth_b[i, [0, 1, 4, 5]] - want[[0, 1, 4, 5]]) / np.abs(want[[0, 1, 4, 5]]))))
        adj["batch_1d_256x500"]["max_rel_err_vs_cpu_adjoint_sampled"] = max(errs)
        adj["batch_1d_256x500"]["cpu_adjoint_grads_per_s"] = adj["1d_500"]["cpu_adjoint_grads_per_s"]

        def one(i):
            x = insts[i]
            return oracle.vjp(x.problem, x.n0, x.C0, 0.0, x.t_out, seeds[i])

        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=cores) as ex:
            list(ex.map(one, range(256)))
        el = time.perf_counter() - t0
        adj["batch_1d_256x500"]["cpu_adjoint_all_cores"] = {
            "grads_per_s": 256 / el, "threads": cores, "sample": "all 256 instances, one per thread at a time"}

    def poly_leg():
        """The AD-vs-ND comparison of the parameter estimation study (Sec. 4.1): the
        polynomial growth law of Eq. 6 with P = 2, 10, 100, 1000 coefficients (K = P/2
        a direction) on the 2-D 128x128 adjoint workload; one gradient by the adjoint
        (pbe_vjp, fused path) against forward differences (P + 1 fused solves, each
        with its coefficients sent to the device)."""
        out = []
        base = pi.adjoint_2d(128)
        for P_ in (2, 10, 100, 1000):
            K = P_ // 2
            prob = pi.poly_growth(base.problem, K)
            g = P.Grid.from_problem(prob, stream=stream, path="fused")
            n0d = torch.as_tensor(base.n0).cuda()
            rows = torch.zeros((len(base.t_out), P.ncols(2)), dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                g.set_state(n0d, base.C0, 0.0)
                _, steps = g.solve(base.t_out, out=rows)
            r = rows.cpu().numpy()
            seeds = np.zeros_like(r)
            seeds[:, [1, 2, 3, 9, 11]] = 1.0 / np.abs(r[:, [1, 2, 3, 9, 11]])
            sd = torch.as_tensor(seeds).cuda()
            ad = []
            with torch.cuda.stream(stream):
                for it in range(2 + 3):
                    g.set_state(n0d, base.C0, 0.0)
                    t0 = time.perf_counter()
                    g.vjp(base.t_out, sd, 64)
                    g.growth_poly_grad()
                    if it >= 2:
                        ad.append(time.perf_counter() - t0)
                a0 = np.array(prob.poly)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for j in range(P_ + 1):   # base point, then one perturbed coefficient at a time
                    a = a0.copy()
                    if j > 0:
                        a[j - 1] *= 1.0 + 1e-6
                    g.set_growth_poly(a)
                    g.set_state(n0d, base.C0, 0.0)
                    g.solve(base.t_out, out=rows)
                nd = time.perf_counter() - t0
            g.close()
            tad = sum(ad) / len(ad)
            out.append({"parameters": P_, "steps": steps, "ad_grads_per_s": 1.0 / tad, "ad_ms": 1e3 * tad,
                        "nd_grads_per_s": 1.0 / nd, "nd_ms": 1e3 * nd, "ad_over_nd": nd / tad})
        return {"workload": "2-D 128x128, polynomial growth law (Eq. 6), 50 loss times; one gradient",
                "rows": out,
                "paper_context": "jax AD with checkpointing about 40x faster than jax ND per iteration at "
                                 "1000 parameters, ND faster below about 20 (Sec. 4.1, RTX 4090)"}

    def closure_leg():
        """The learned closure at the workload's size (1024 training and 256 held-out
        trajectories of the 2-D problem on 128 x 128 grids, Adam at lr 1e-3, minibatches
        of 32): trained through the solver for a bounded time, then the held-out
        moment-trajectory error against the solver with the nominal (misspecified)
        power law; gradients/s of the training (solve + persistent adjoint per
        trajectory, one weight-gradient launch per minibatch)."""
        from paper_2411_00742_gb300.train_closure import main as train_main
        res = train_main(["--train", "1024", "--heldout", "256", "--grid", "128", "--epochs", "24",
                          "--batch", "32", "--lr", "1e-3", "--workers", "8",
                          "--max-seconds", str(args.closure_seconds)], emit=False)
        res["note"] = ("training stopped after max_seconds of wall time; gain = held-out relative RMS error "
                       "of the misspecified power law / that of the trained closure")
        return res

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
                             "roofline_frac": FLOPS_PER_CELL_STEP_2D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL,
                             "roofline_frac_own_count": OWN_FLOPS_PER_CELL_STEP_2D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL}
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
                             "roofline_frac": FLOPS_PER_CELL_STEP_1D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL,
                             "roofline_frac_own_count": OWN_FLOPS_PER_CELL_STEP_1D * rate / 1e12 / FP64_PEAK_TFLOPS_NOMINAL}
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
    poly = poly_leg() if not args.no_adjoint else None
    closure = closure_leg() if not args.no_closure else None
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
    achieved_own = OWN_FLOPS_PER_CELL_STEP_2D * cells_per_solve / k_fused / 1e12
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
                     "launch_ms": 1e3 * k_fused, "flops_per_cell_step": FLOPS_PER_CELL_STEP_2D,
                     "own_count": {"flops_per_cell_step": OWN_FLOPS_PER_CELL_STEP_2D, "achieved": achieved_own,
                                   "frac": achieved_own / FP64_PEAK_TFLOPS_NOMINAL},
                     "note": f"FP64 algorithmic {FLOPS_PER_CELL_STEP_2D} flop/cell-step (43 flops + 4 divisions, "
                             "division = 1) x cell-steps per launch / launch time (CUDA events the library records "
                             "around the launch on its stream, mean over the timed solves); peak = nominal GB300 "
                             "FP64 (of nominal: the measured-peaks file has no FP64 entry)"},
        "e2e": {"value": ws * e2e_rate, "unit": "cell-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "batch_1d": batch,
        "small_1d": small_1d,
        "adjoint": adjoint,
        "paper_scheme": paper,
        "ad_vs_nd": poly,
        "closure": closure,
        "scaling_2d": scaling,
        "scaling_1d": scaling_1d,
        # per timed fused solve: k_set_scalars, k_prologue, k_fused, k_fused_rows
        "gpu_launches": 4 * args.steps,
        "clocks": clk,
    }
    binsts = batch.pop("_insts") if batch is not None else None
    if rank == 0 and not args.no_cpu_baseline:
        # the CPU baseline leg: the oracle timed on the host, and its rows give the
        # stated error of the GPU rows on the same solves
        import oracle
        cores = os.cpu_count() or 1
        v, reps, el, want = _oracle_rate(inst, budget_s=args.cpu_seconds)
        oracle.set_threads(cores)
        t0 = time.perf_counter()
        oracle.solve_instance(inst)
        el_all = time.perf_counter() - t0
        oracle.set_threads(1)
        line["cpu_baseline"] = {"value": v, "unit": "cell-steps/s", "cores": 1, "kind": "oracle",
                                "sample": f"{reps} full solves of the same 256x256 workload ({el:.1f} s), single thread",
                                "all_cores": {"value": inst.problem.ncell * want["steps"] / el_all, "threads": cores,
                                              "sample": "one full solve, rows of the grid in parallel (OpenMP)"},
                                "host": _host_info()}
        if batch is not None:
            # the batch on every core: instances in parallel (all 4096, a few seconds)
            from concurrent.futures import ThreadPoolExecutor
            sample = binsts
            t0 = time.perf_counter()
            with ThreadPoolExecutor(max_workers=cores) as ex:
                res = list(ex.map(oracle.solve_instance, sample))
            elb = time.perf_counter() - t0
            cs = sum(x.problem.ncell * r["steps"] for x, r in zip(sample, res))
            batch["cpu_all_cores"] = {"value": cs / elb, "unit": "cell-steps/s", "threads": cores,
                                      "sample": f"first {len(sample)} instances, one per thread at a time ({elb:.1f} s)"}

        def rel_err(got, ref):
            return float(np.max(np.abs(got[:, 1:] - ref["rows"][:, 1:]) / np.abs(ref["rows"][:, 1:])))

        line["paths"]["fused"]["max_rel_err_vs_oracle"] = rel_err(rows_fused, want)
        line["paths"]["plain"]["max_rel_err_vs_oracle"] = rel_err(rows_plain, want)
        if adjoint is not None:
            adjoint_cpu_baseline(adjoint, adjoint_cases, cores)
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


def profile_case(argv):
    """``bench.py --profile-case PATH N1 [N2] [options]``: a few solves (or gradients)
    of one seeded workload on one execution path - the small, self-contained
    program to put under a profiler (ncu) or a timer.

      fused|plain N1 [N2]   the 2-D size-and-shape problem on an N1 x N2 grid
                            (--ndim 1: the 1-D fine-grid problem of N1 cells)
      paper N1              the paper's base case at N1 x N1/2 bins (plain path)
      batch N1              N1 batched 1-D instances (the batch workload), one solve each repeat
                            (--autotune or --schedule WPB TEAM CELLS first)
      batch-adjoint N1      batched gradients (pbe_batch_vjp) of N1 instances of 500 cells
                            (the gradient batch workload; --vjp-warps W per instance)
      adjoint N1 [N2]       gradients (pbe_vjp, fused path) of the 2-D adjoint workload on
                            N1 x N2 (--ndim 1: one 1-D instance of N1 cells)

    --outputs K keeps the first K output times; --steps K runs K single steps
    (Grid.step) instead of solves, outside the plain path's CUDA graph whose
    conditional nodes a profiler cannot capture.  Prints one line per solve."""
    ap = argparse.ArgumentParser(prog="bench.py --profile-case", description=profile_case.__doc__.splitlines()[0])
    ap.add_argument("path", choices=["fused", "plain", "paper", "batch", "batch-adjoint", "adjoint"])
    ap.add_argument("N1", type=int)
    ap.add_argument("N2", type=int, nargs="?")
    ap.add_argument("--ndim", type=int, default=2, choices=[1, 2])
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--outputs", type=int, default=0)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--window", type=int, default=-1, choices=[-1, 0, 1])
    ap.add_argument("--autotune", action="store_true", help="batch: autotune the schedule first")
    ap.add_argument("--vjp-warps", type=int, default=0, help="batch-adjoint: warps per instance (0: automatic)")
    ap.add_argument("--vjp-blocks", type=int, default=0, help="batch-adjoint: teams per SM (0: automatic)")
    ap.add_argument("--block-limit", type=int, default=0, help="fused/adjoint: most blocks of the launch (0: none)")
    ap.add_argument("--schedule", type=int, nargs=3, metavar=("WPB", "TEAM", "CELLS"),
                    help="batch: set this schedule (warps per block, team instances, warp cells)")
    a = ap.parse_args(argv)
    import torch
    import paper_2411_00742_gb300 as P

    if a.path == "batch":
        insts = pi.batch_1d(a.N1, seed=2411)
        b = P.Batch([x.problem for x in insts], [x.C0 for x in insts])
        packed = torch.as_tensor(b.pack([x.n0 for x in insts])).cuda()
        if a.schedule:
            b.set_schedule(*a.schedule)
        elif a.autotune:
            b.set_state(packed)
            t0 = time.perf_counter()
            b.autotune(insts[0].t_out)
            print(f"batch autotune {time.perf_counter() - t0:.2f} s", flush=True)
        print(f"batch schedule (warps per block, team instances, warp cells) {b.schedule()}", flush=True)
        for _ in range(a.repeat):
            b.set_state(packed)
            t0 = time.perf_counter()
            _, st = b.solve(insts[0].t_out)
            print(f"batch {a.N1} instances steps {st} {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
        b.close()
        return 0
    if a.path == "batch-adjoint":
        insts = pi.adjoint_batch_1d(a.N1)
        bt = P.Batch([x.problem.with_theta(x.problem.theta * pi.TARGET_FACTOR) for x in insts],
                     [x.C0 for x in insts])
        bt.set_state(bt.pack([x.n0 for x in insts]))
        tgts, _ = bt.solve(pi.loss_times())
        bt.close()
        b = P.Batch([x.problem for x in insts], [x.C0 for x in insts])
        packed = b.pack([x.n0 for x in insts])
        b.set_state(packed)
        fwd, _ = b.solve(pi.loss_times())
        cols = [1, 2, 3, 4, 5]
        sd = np.zeros_like(fwd)
        sd[..., cols] = 2.0 * (fwd[..., cols] - tgts[..., cols]) / tgts[..., cols] ** 2   # relative-error loss
        seeds = torch.as_tensor(sd).cuda()
        b.set_vjp_schedule(a.vjp_warps, a.vjp_blocks)
        for _ in range(a.repeat):
            b.set_state(packed)
            t0 = time.perf_counter()
            b.vjp(pi.loss_times(), seeds, 64)
            print(f"batch-adjoint {a.N1} x 500 cells, warps {a.vjp_warps} blocks/SM {a.vjp_blocks} "
                  f"{1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
        b.close()
        return 0
    if a.path == "adjoint":
        inst = pi.adjoint_batch_1d(1)[0] if a.ndim == 1 else pi.adjoint_2d(a.N1)
        if a.ndim == 1 and a.N1 != inst.problem.ncell:
            inst = pi.config_1d(a.N1)
            inst.t_out = pi.loss_times()
        if a.ndim == 2 and a.N2:
            inst = pi.config_2d(a.N1, a.N2)
            inst.t_out = pi.loss_times()
        g = P.Grid.from_problem(inst.problem, path="fused")
        g.set_block_limit(a.block_limit)
        g.set_state(inst.n0, inst.C0, 0.0)
        rows, _ = g.solve(inst.t_out)
        seeds = np.zeros_like(rows)
        seeds[:, 1:] = 1.0 / np.abs(rows[:, 1:])
        for _ in range(a.repeat):
            g.set_state(inst.n0, inst.C0, 0.0)
            t0 = time.perf_counter()
            g.vjp(inst.t_out, seeds, 64)
            print(f"adjoint {inst.problem.ncells} {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
        g.close()
        return 0
    if a.path == "paper":
        inst, path = pi.paper_base_case(a.N1), "plain"
    elif a.ndim == 1:
        inst, path = pi.config_1d_fine(a.N1), a.path
    else:
        inst, path = pi.config_2d(a.N1, a.N2), a.path
    t_out = inst.t_out[: a.outputs] if a.outputs > 0 else inst.t_out
    g = P.Grid.from_problem(inst.problem, path=path)
    g.set_window(a.window)
    g.set_block_limit(a.block_limit)
    n0 = torch.as_tensor(inst.n0).cuda()
    if a.steps > 0:
        g.set_state(n0, inst.C0, 0.0)
        for k in range(a.steps):   # the k-th step ends at the (k+1)-th output time at most
            t0 = time.perf_counter()
            dt = g.step(float(t_out[min(k + 1, len(t_out) - 1)]))
            print(f"{a.path} {inst.problem.ncells} step dt {dt:.6g} {1e3 * (time.perf_counter() - t0):.3f} ms",
                  flush=True)
        g.close()
        return 0
    for _ in range(a.repeat):
        g.set_state(n0, inst.C0, 0.0)
        t0 = time.perf_counter()
        _, steps = g.solve(t_out)
        print(f"{a.path} {inst.problem.ncells} steps {steps} {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
    g.close()
    return 0


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--profile-case":
        return profile_case(sys.argv[2:])
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
    ap.add_argument("--no-closure", action="store_true")
    ap.add_argument("--closure-seconds", type=float, default=60.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
