"""Train the learned kinetics closure through the solver and evaluate it.

    python -m paper_2411_00742_gb300.train_closure --train 1024 --heldout 256 --grid 128 \
        --epochs 4 --batch 32 --out closure_result.json

Truth trajectories come from the FP64 solver with hidden power-law kinetics
(pbe_closure_data.hidden_law); the closure is trained with Adam (lr 1e-3) on
the relative errors of mu00, mu10, mu01, mu12 and C at 50 times, and evaluated
on held-out trajectories against the same solver with the nominal (wrong)
power-law kinetics, i.e. the method without the closure.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np


def main(argv=None, emit=True):
    """Train and report; progress lines go to stderr, the result (a dict) is
    returned and, with emit, printed to stdout as one JSON line."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--heldout", type=int, default=256)
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--grid-blocks", type=int, default=None,
                    help="block limit of each trajectory's grid (default: SMs / workers; 0: one block per SM)")
    ap.add_argument("--max-seconds", type=float, default=1e9)
    ap.add_argument("--out", default=None)
    ap.add_argument("--weights-out", default=None)
    args = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    import pbe_closure_data as cd
    from paper_2411_00742_gb300.closure import ClosureTrainer, loss_cols, trajectory_error

    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    train = cd.trajectories(args.train, seed=24130, N=args.grid)
    held = cd.trajectories(args.heldout, seed=24131, N=args.grid)
    tr = ClosureTrainer(cd.initial_weights(), train[0].problem, lr=args.lr, workers=args.workers,
                        grid_blocks=args.grid_blocks)
    # truth: the FP64 solver with the hidden law
    t_truth = time.perf_counter()
    y_train = tr.rows(train)
    y_held = tr.rows(held)
    t_truth = time.perf_counter() - t_truth
    cols = loss_cols(2)
    rng = np.random.default_rng(0)
    history = []
    steps = 0
    t_train = time.perf_counter()
    for ep in range(args.epochs):
        order = rng.permutation(len(train))
        losses = []
        for b in range(0, len(train), args.batch):
            idx = order[b:b + args.batch]
            L = tr.step([train[i] for i in idx], [y_train[i] for i in idx])
            losses.append(L)
            steps += 1
            if time.perf_counter() - t_train > args.max_seconds:
                break
        history.append(float(np.mean(losses)))
        print(f"epoch {ep}: mean loss {history[-1]:.4e} ({steps} Adam steps, {time.perf_counter() - t_train:.1f} s)",
              file=sys.stderr, flush=True)
        if time.perf_counter() - t_train > args.max_seconds:
            break
    t_train = time.perf_counter() - t_train
    w = tr.weights32()
    rows_closure = tr.rows(held, weights=w)
    rows_plain = tr.rows(held, problems=[cd.misspecified(x) for x in held])
    e_closure = np.array([trajectory_error(r, y, cols) for r, y in zip(rows_closure, y_held)])
    e_plain = np.array([trajectory_error(r, y, cols) for r, y in zip(rows_plain, y_held)])
    grads = steps * args.batch
    res = {"train_trajectories": len(train), "heldout_trajectories": len(held), "grid": [args.grid, args.grid],
           "epochs_run": len(history), "adam_steps": steps, "batch": args.batch, "lr": args.lr,
           "loss_history": history, "train_seconds": t_train, "truth_seconds": t_truth,
           "gradients_per_s": grads / t_train,
           "heldout_rel_rms_error": {"closure_mean": float(e_closure.mean()), "closure_median": float(np.median(e_closure)),
                                     "plain_misspecified_mean": float(e_plain.mean()),
                                     "plain_misspecified_median": float(np.median(e_plain))},
           "gain": float(e_plain.mean() / e_closure.mean()), "total_seconds": time.perf_counter() - t0}
    tr.close()
    if emit:
        print(json.dumps(res), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(res, f, indent=1)
    if args.weights_out:
        np.save(args.weights_out, w)
    return res


if __name__ == "__main__":
    main()
