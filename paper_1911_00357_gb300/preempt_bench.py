"""Frames per second of DD-PPO workers against the preemption threshold p (Sec. 3; Sec. 5
"heterogeneous workloads").

N virtual workers share the GPU, each with its own envs, seed and CUDA stream; their
gradients are averaged every minibatch (Eq. 4). The workload is heterogeneous: worker w
simulates square grids of side sides[w % len(sides)] (the mixed-size workload's
{64, 128, 256, 512} by default), so the workers on large grids, whose resets run longer
BFS fields and whose depth rays cross larger rooms, are the stragglers. For each p the
tool reports the frames per second of the whole job (all workers' T_valid x envs over the
wall time of the timed iterations) and the workers' mean T_valid.

    python -m paper_1911_00357_gb300.preempt_bench [--workers 8] [--envs 16] [--T 64]
        [--p 1.0 0.8 0.6] [--iters 3] [--warmup 1] [--preset mixed_1024]

A measurement tool; the headline number is bench.py's.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .ddppo import VirtualWorkers, timed_iterations


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="mixed_1024")
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--envs", type=int, default=16)
    ap.add_argument("--T", type=int, default=64)
    ap.add_argument("--sides", type=int, nargs="+", default=[64, 128, 256, 512])
    ap.add_argument("--p", type=float, nargs="+", default=[1.0, 0.8, 0.6])
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--chunk", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    sides = [args.sides[w % len(args.sides)] for w in range(args.workers)]
    vw = VirtualWorkers(args.preset, args.workers, seed=args.seed, grid_sides=sides,
                        num_envs=args.envs, rollout_T=args.T, minibatches=2,
                        encoder_chunk=args.chunk, tune=True)
    try:
        for p in args.p:
            vw.set_threshold(p)
            r = timed_iterations(vw, args.iters, args.warmup)
            tv = [sum(x) / len(x) for x in zip(*r["T_valid"])]
            print(json.dumps({
                "p": p, "workers": args.workers, "envs_per_worker": args.envs, "T": args.T,
                "preset": args.preset, "grid_sides": sides,
                "frames_per_s": round(r["frames_per_s"], 1),
                "s_per_iter": round(r["s_per_iter"], 4),
                "mean_T_valid_per_worker": [round(x, 1) for x in tv],
                "device_status": max(abs(B.ddppo_device_status(w.h)) for w in vw.workers),
            }), flush=True)
    finally:
        vw.close()
        torch.cuda.synchronize()


if __name__ == "__main__":
    main()
