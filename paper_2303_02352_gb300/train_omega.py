"""Trains the damping network on the GPU and evaluates it against plain
l1-Jacobi.

Recipe: 64 seeded 7-point random-coefficient problems on 64^3 grids
(log-normal k with sigma_p = 0.5 + 2.5 U, constant on 8^3 blocks, seed
1000 + p), objective (1/m) ln(|r_m| / |r_0|) of m = 3 stationary V-cycle steps
from seeded random r_0, Adam; then PCG to 1e-6 on a held-out 7-point
log-normal problem (sigma = 2, seed 4000) and on 7-point Poisson, with the FP32
and FP64 hierarchies, plain vs learned (the selection keeps the learned damping
only if it needs no more iterations).

    python -m paper_2303_02352_gb300.train_omega [--problems 64] [--N 64] [--epochs 5]
        [--eval-N 256] [--out paper_2303_02352_gb300/weights/omega_mlp.npz]
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np


def timed_solve(h, b, x, reps=3, tol=1e-6):
    import torch
    res = h.solve_into(b, x.zero_(), tol, 1000)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        res = h.solve_into(b, x.zero_(), tol, 1000)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, res


def evaluate(net, A, b_np, desc, precisions=(1, 0)):
    import torch
    from . import amg
    b = torch.as_tensor(b_np, device="cuda")
    x = torch.zeros_like(b)
    out = {"workload": desc}
    for prec in precisions:
        h = amg.Hierarchy(A, precision=prec)
        ms_p, rp = timed_solve(h, b, x)
        h.apply_mlp(net.w)
        ms_l, rl = timed_solve(h, b, x)
        use = rl["iters"] <= rp["iters"] and rl["status"] == 0
        name = {0: "fp64", 1: "fp32", 2: "bf16fine"}[prec]
        out[name] = {"plain_iters": rp["iters"], "plain_ms": ms_p, "plain_true_rel_res": rp["true_rel_res"],
                     "learned_iters": rl["iters"], "learned_ms": ms_l, "learned_true_rel_res": rl["true_rel_res"],
                     "learned_kept": use}
        h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=64)
    ap.add_argument("--N", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=5)
    ap.add_argument("--m", type=int, default=3)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--eval-N", type=int, default=256)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import torch
    from . import build, learned, workloads as W
    build.build()
    out = args.out or learned.DEFAULT_WEIGHTS
    t0 = time.time()
    probs = [W.training_problem(p, N=args.N) for p in range(args.problems)]
    t1 = time.time()
    net, losses = learned.train(probs, steps=args.problems * args.epochs, m=args.m, lr=args.lr, seed=0,
                                log=lambda s: print(s, flush=True))
    torch.cuda.synchronize()
    t2 = time.time()
    net.save(out)
    report = {"recipe": {"problems": args.problems, "N": args.N, "epochs": args.epochs, "m": args.m, "lr": args.lr},
              "train_seconds": t2 - t1, "generate_seconds": t1 - t0,
              "loss_first_epoch": float(np.mean(losses[:args.problems])),
              "loss_last_epoch": float(np.mean(losses[-args.problems:])),
              "losses": [round(x, 5) for x in losses]}
    N = args.eval_N
    A = W.diffusion7(N, 2.0, 4000)
    report["eval_lognormal"] = evaluate(net, A, W.rhs_from_solution(A, W.random_vector(A.n, 4)),
                                        f"7-pt log-normal diffusion {N}^3, sigma 2, seed 4000")
    del A
    A = W.poisson7(N)
    report["eval_poisson"] = evaluate(net, A, W.rhs_from_solution(A, W.random_vector(A.n, 4)), f"7-pt Poisson {N}^3")
    path = os.path.splitext(out)[0] + "_report.json"
    json.dump(report, open(path, "w"), indent=1)
    print(json.dumps({k: v for k, v in report.items() if k != "losses"}, indent=1))


if __name__ == "__main__":
    main()
