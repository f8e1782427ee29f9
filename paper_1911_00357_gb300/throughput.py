"""Experience frames per second of one worker, measured the paper's way (App. "Additional
scaling details": a fixed number of collect + optimise iterations, throughput taken over
the last ones, repeated over seeds) on a named workload:

    python -m paper_1911_00357_gb300.throughput --preset resnet [--precision 0] \
        [--seeds 0 1 2] [--iters 10] [--last 5]

For every seed a fresh worker (new world, new random weights, new tuning pass) runs
`iters` synchronous iterations; the frames of the last `last` iterations (E x T each)
over their device time (CUDA events on the launching stream) give that seed's rate.
Prints one JSON line per seed and a summary line with the mean and the 95% confidence
half-width (Student t over the seeds). Inputs are synthetic and resident in HBM. A
measurement tool; the headline number is bench.py's.
"""
from __future__ import annotations

import argparse
import json
import math

import torch

from . import binding as B
from .presets import PRESETS
from .worker import Worker

# two-sided 95% Student t quantiles, by degrees of freedom
_T95 = {1: 12.706, 2: 4.303, 3: 3.182, 4: 2.776, 5: 2.571, 6: 2.447, 7: 2.365, 8: 2.306,
        9: 2.262, 10: 2.228, 11: 2.201, 12: 2.179, 13: 2.160, 14: 2.145, 15: 2.131}


def ci95(xs):
    """Mean and 95% confidence half-width of the mean (0 for a single value)."""
    n = len(xs)
    mean = sum(xs) / n
    if n < 2:
        return mean, 0.0
    var = sum((x - mean) ** 2 for x in xs) / (n - 1)
    return mean, _T95.get(n - 1, 1.96) * math.sqrt(var / n)


def run_seed(preset, seed, iters, last, precision=None, lstm_mode=2):
    w = Worker(preset, seed=seed, precision=precision)
    try:
        B.ddppo_lstm_whole_segment(w.h, lstm_mode)
        s = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
        torch.cuda.synchronize()
        ev[0].record(s)
        for i in range(iters):
            w.iterate()
            ev[i + 1].record(s)
        torch.cuda.synchronize()
        ms = ev[iters - last].elapsed_time(ev[iters])
        status = B.ddppo_device_status(w.h)
        return w.E * w.T * last / (ms / 1e3), ms / last, w.cfg.precision, status
    finally:
        w.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--preset", default="resnet", choices=sorted(PRESETS))
    ap.add_argument("--precision", type=int, default=None)
    ap.add_argument("--seeds", type=int, nargs="+", default=[0, 1, 2])
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--last", type=int, default=5)
    ap.add_argument("--lstm-mode", type=int, default=2, choices=[0, 1, 2])
    args = ap.parse_args()
    if not 1 <= args.last <= args.iters:
        ap.error("need 1 <= last <= iters")
    rates = []
    prec = None
    for seed in args.seeds:
        fps, ms_it, prec, status = run_seed(args.preset, seed, args.iters, args.last,
                                            args.precision, args.lstm_mode)
        rates.append(fps)
        print(json.dumps({"preset": args.preset, "precision": prec, "seed": seed,
                          "frames_per_s": round(fps, 1), "ms_per_iter": round(ms_it, 2),
                          "device_status": status}), flush=True)
    mean, half = ci95(rates)
    print(json.dumps({"preset": args.preset, "precision": prec, "seeds": args.seeds,
                      "iters": args.iters, "last": args.last,
                      "frames_per_s_mean": round(mean, 1), "ci95_half_width": round(half, 1),
                      "min": round(min(rates), 1), "max": round(max(rates), 1)}), flush=True)


if __name__ == "__main__":
    main()
