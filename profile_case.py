"""Run a few solves of one seeded workload on one execution path: the small,
self-contained program to put under a profiler (ncu) or a timer.

    python profile_case.py fused 256
    python profile_case.py plain 4096 --window 1 --steps 3
    python profile_case.py paper 6000 --steps 3
    python profile_case.py fused 1048576 --ndim 1

Workloads: ``fused``/``plain`` run the 2-D size-and-shape problem on an N x N
(or N1 x N2) grid (``pbe_inputs.config_2d``); ``paper`` runs the paper's base
case at N x N/2 bins (``pbe_inputs.paper_base_case``); ``--ndim 1`` runs the 1-D
fine-grid problem of N cells (``pbe_inputs.config_1d_fine``).  ``--outputs K`` keeps
the first K output times (a shorter solve); every solve starts from the same
seeded state.  ``--steps K`` runs K single steps (``Grid.step``) instead of
solves: the plain path then launches its stage kernels one by one, outside
the CUDA graph whose conditional nodes a profiler cannot capture.  Prints one
line per solve or step: path, grid, steps or dt, wall time.
"""
from __future__ import annotations

import argparse
import os
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("path", choices=["fused", "plain", "paper"])
    ap.add_argument("N1", type=int)
    ap.add_argument("N2", type=int, nargs="?")
    ap.add_argument("--ndim", type=int, default=2, choices=[1, 2], help="1: the 1-D fine-grid problem")
    ap.add_argument("--repeat", type=int, default=2)
    ap.add_argument("--outputs", type=int, default=0, help="keep the first K output times (0: all)")
    ap.add_argument("--steps", type=int, default=0, help="run K single steps instead of solves")
    ap.add_argument("--window", type=int, default=-1, choices=[-1, 0, 1],
                    help="plain-path 2-D stage kernel: -1 auto, 0 tile, 1 register window")
    args = ap.parse_args(argv)

    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import torch

    import pbe_inputs as pi
    import paper_2411_00742_gb300 as P

    if args.path == "paper":
        inst = pi.paper_base_case(args.N1)
        path = "plain"
    elif args.ndim == 1:
        inst = pi.config_1d_fine(args.N1)
        path = args.path
    else:
        inst = pi.config_2d(args.N1, args.N2)
        path = args.path
    t_out = inst.t_out[: args.outputs] if args.outputs > 0 else inst.t_out
    g = P.Grid.from_problem(inst.problem, path=path)
    g.set_window(args.window)
    n0 = torch.as_tensor(inst.n0).cuda()
    if args.steps > 0:
        g.set_state(n0, inst.C0, 0.0)
        for k in range(args.steps):   # the k-th step ends at the (k+1)-th output time at most
            t0 = time.perf_counter()
            dt = g.step(float(t_out[min(k + 1, len(t_out) - 1)]))
            print(f"{args.path} {inst.problem.ncells} step dt {dt:.6g} {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
        g.close()
        return
    for _ in range(args.repeat):
        g.set_state(n0, inst.C0, 0.0)
        t0 = time.perf_counter()
        _, steps = g.solve(t_out)
        print(f"{args.path} {inst.problem.ncells} steps {steps} {1e3 * (time.perf_counter() - t0):.3f} ms", flush=True)
    g.close()


if __name__ == "__main__":
    main()
