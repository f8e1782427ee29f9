"""Per-phase timing of one worker iteration for any named workload:
collect (the captured act + env-step loop), then GAE + PPO update.

    python -m paper_1911_00357_gb300.phase_bench --preset wide_256_fp8 [--steps 3] [--warmup 2]

Prints one JSON line: median collect and update times (CUDA events on the launching stream)
over the timed iterations, the act-phase frame rate (E * T / collect) and the whole-iteration
frame rate, with the device status word. A measurement tool; the headline number is
bench.py's.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .presets import PRESETS
from .worker import Worker


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="resnet", choices=sorted(PRESETS))
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--precision", type=int, default=None, help="override the preset's precision")
    ap.add_argument("--lstm-mode", type=int, default=0, choices=[0, 1, 2],
                    help="LSTM recurrence: 0 step by step (default), 1 whole segment on CUDA "
                         "cores, 2 tcgen05 forward")
    ap.add_argument("--gn-two-launch", action="store_true",
                    help="GroupNorm statistics and normalisation as two launches")
    ap.add_argument("--no-launch-overlap", action="store_true",
                    help="plain stream order instead of programmatic dependent launch")
    args = ap.parse_args()
    B.ddppo_set_launch_overlap(not args.no_launch_overlap)
    w = Worker(args.preset, seed=args.seed, precision=args.precision)
    B.ddppo_lstm_whole_segment(w.h, args.lstm_mode)
    if args.gn_two_launch:
        B.ddppo_group_norm_one_launch(w.h, False)
    try:
        for _ in range(args.warmup):
            w.iterate()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        col, upd = [], []
        t = w.t
        for i in range(args.steps):
            t["uniforms"].copy_(w._pool[i % w._pool.shape[0]])
            ev[0].record(s)
            B.ddppo_collect(w.h, w.view, True)
            ev[1].record(s)
            B.ddppo_gae(t["rewards"], t["dones"], t["values"], w.T, w.E, w.gamma, w.lam,
                        t["adv"], t["ret"])
            w.hp.update_index = w.updates
            B.ddppo_ppo_update(w.h, w.view, w.hp, w.stats)
            w.updates += 1
            ev[2].record(s)
            torch.cuda.synchronize()
            col.append(ev[0].elapsed_time(ev[1]))
            upd.append(ev[1].elapsed_time(ev[2]))
        c = sorted(col)[len(col) // 2]
        u = sorted(upd)[len(upd) // 2]
        frames = w.E * w.T
        print(json.dumps({
            "preset": args.preset, "precision": w.cfg.precision, "num_envs": w.E, "rollout_T": w.T,
            "seed": args.seed, "lstm_mode": args.lstm_mode,
            "group_norm": "two launches" if args.gn_two_launch else "one launch",
            "launch_overlap": not args.no_launch_overlap,
            "collect_ms": round(c, 2), "update_ms": round(u, 2),
            "act_frames_per_s": round(frames / c * 1e3, 1),
            "frames_per_s": round(frames / (c + u) * 1e3, 1),
            "device_status": B.ddppo_device_status(w.h),
            "stats_finite": bool(torch.isfinite(w.stats).all()),
        }), flush=True)
    finally:
        w.close()


if __name__ == "__main__":
    main()
