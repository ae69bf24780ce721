"""Train the schedule network on plain adaptive runs and write its weights.

Training data: plain overlap-bisection schedules (target overlap 0.8, dbeta <= 0.1, beta 0 -> 1)
at L in {16, 32, 64}, R = 5e4, several seeds, with the sweep-count label of
`learned.plain_training_run`.  Training: the library's forward / backward / Adam kernels.

    python -m paper_2102_06611_gb300.train_schedule [--out PATH] [--seeds N] [--steps K]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "schedule_mlp.npz")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--Ls", default="16,32,64")
    ap.add_argument("--R", type=int, default=50_000)
    ap.add_argument("--seeds", type=int, default=4)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=2e-3)
    args = ap.parse_args()

    import torch

    from .learned import ScheduleMLP, plain_training_run

    torch.cuda.set_device(0)
    Ls = [int(x) for x in args.Ls.split(",")]
    X, Y, runs = [], [], []
    t0 = time.perf_counter()
    for L in Ls:
        for s in range(args.seeds):
            x, y = plain_training_run(L, args.R, seed=1000 + 17 * L + s)
            X.append(x)
            Y.append(y)
            runs.append({"L": L, "seed": 1000 + 17 * L + s, "steps": len(x),
                         "theta_mean": float(np.exp(y[:, 1]).mean()), "theta_max": float(np.exp(y[:, 1]).max())})
    X = np.concatenate(X)
    Y = np.concatenate(Y)
    t_data = time.perf_counter() - t0
    model = ScheduleMLP(seed=0)
    t1 = time.perf_counter()
    losses = model.train(X, Y, steps=args.steps, batch=args.batch, lr=args.lr)
    t_train = time.perf_counter() - t1
    model.save(args.out)
    report = {"samples": int(len(X)), "runs": runs, "R": args.R, "data_s": t_data, "train_s": t_train,
              "loss_first": losses[0], "loss_last": losses[-1], "steps": args.steps, "batch": args.batch,
              "lr": args.lr}
    with open(os.path.splitext(args.out)[0] + "_train.json", "w") as f:
        json.dump(report, f, indent=1)
        f.write("\n")
    print(json.dumps(report))


if __name__ == "__main__":
    main()
