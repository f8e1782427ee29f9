"""Throughput of the DD-PPO rollout-then-update step on GB300.

One step = one synchronous DD-PPO iteration of one worker (Sec. 3, Eq. 4 without the
multi-worker allreduce): collect T frames from each of E envs (policy act + simulator
step, captured as a CUDA graph), bootstrap value, GAE, then epochs x minibatches of PPO
(forward, loss, hand-written backward, Adam). Metric: experience frames per second
(E*T per step), measured as in App. "Additional scaling details" (time a run of steps
after warm-up). Workload: 64 envs on 128x128 rooms-and-doors grids at 0.1 m, depth
256x256 pooled to 128x128, ResNet-18-style encoder (32 base, GroupNorm) -> 2-layer LSTM
512, T = 128, 2 epochs x 2 minibatches, Adam 2.5e-4.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32]
  python bench.py --impl reference ...   # the float64 CPU oracle on a bounded sample
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pointnav_resnet18b32_lstm2x512_E64_T128_rooms128"

# the oracle's sample of each named workload for the reference arm: (workload name, sample
# envs, sample frames, SimConfig fields, NetConfig fields, 2x2 pool, minibatches)
ORACLE_SAMPLES = {
    "resnet": (WORKLOAD, 4, 16, {}, {}, True, 2),
    "nature": ("pointnav_nature_cnn_lstm128_E16_T32_bernoulli32", 4, 32,
               dict(gen_kind=0, grid_min=32, grid_max=32, cell_m=0.25, depth_h=64, depth_w=64),
               dict(net_kind=0, hidden=128, lstm_layers=1, in_h=64, in_w=64), False, 2),
    "mixed": ("pointnav_resnet18b32_lstm2x512_E1024_T128_mixed64-512", 4, 16,
              dict(grid_min=64, grid_max=512, depth_h=128, depth_w=128), {}, False, 2),
    "wide": ("pointnav_resnet18b64_lstm2x512_E256_T128_rooms128", 4, 16, {}, dict(base_ch=64),
             True, 2),
    "scale": ("pointnav_resnet18b32_lstm2x512_E4096_T128_rooms128_4mb", 4, 16, {}, {}, True, 4),
    "blind": ("pointnav_blind_lstm2x512_E64_T128_rooms128", 4, 16, {}, dict(net_kind=2), True, 2),
}
METRIC = "experience frames/sec (sim+act+learn) on 1 GB300, BF16 batched vs plain FP32"
UNIT = "frames/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples taken while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic of the update's contractions over their algorithmic bytes, from one ncu
# capture of the same step at T = 16 (dram__bytes_read.sum + dram__bytes_write.sum over the
# update's contraction launches: 10,400 MB against 15,690 MB algorithmic); the full-size
# traffic is reported as this fraction of the live algorithmic bytes
GEMM_TRAFFIC_OVER_ALGORITHMIC = 10400.0 / 15690.0


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1911_00357_gb300 import binding as B
    from paper_1911_00357_gb300.dist import aggregate
    from paper_1911_00357_gb300.worker import Worker

    rank, world, local = _dist()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    precision = 1 if args.precision == "bf16" else 0

    def measure(prec, steps, warmup, timing):
        kw = {"rollout_T": args.rollout_T} if args.rollout_T else {}
        w = Worker("resnet", precision=prec, seed=1000 * rank + 17, **kw)
        cache = args.tune_cache if prec == 1 else None
        if cache and os.path.exists(cache):
            with open(cache, "rb") as f:
                B.ddppo_autotune_import(w.h, f.read())
        for _ in range(warmup):
            w.iterate()
        if cache and not os.path.exists(cache) and rank == 0:
            with open(cache, "wb") as f:
                f.write(B.ddppo_autotune_export(w.h))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk = ClockSampler(local) if timing else None
        if clk:
            clk.start()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(steps):
            w.iterate()
        e1.record(s)
        torch.cuda.synchronize()
        clocks = clk.stop() if clk else None
        ms = e0.elapsed_time(e1)
        gemm = tc = per_launch = None
        if timing and not args.profile:
            # per-launch records of the contractions, from one more step outside the timed
            # region (recording them runs the update uncaptured)
            B.ddppo_timing_enable(w.h, True)
            w.iterate()
            torch.cuda.synchronize()
            gemm = B.ddppo_timing_read(w.h, 0)
            tc = B.ddppo_timing_read(w.h, 2)
            per_launch = B.ddppo_timing_launches(w.h, 0)
            B.ddppo_timing_enable(w.h, False)
        return w, ms, clocks, gemm, tc, per_launch

    w, ms_local, clocks, gemm, tc, per_launch = measure(precision, args.steps, args.warmup, True)
    value, ms, frames = aggregate(w.E * w.T * args.steps, ms_local, torch.device("cuda"))
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms / args.steps}), flush=True)
        return
    rc = w.time_raycast(16)

    # end to end through the public API: uniforms H2D from pinned memory each step,
    # statistics and rewards D2H each step
    e2e_ms, h2d, d2h = w.time_e2e(args.steps)
    e2e_value, _, _ = aggregate(w.E * w.T * args.steps, e2e_ms, torch.device("cuda"))

    # plain FP32 form on the same GPU (the metric's denominator), in its faster launch
    # setting: plain stream order. With programmatic dependent launch its long SIMT
    # contractions run ~12% slower (4,165 against 4,736 frames/s measured), while the BF16
    # form gains from it; results are bit-identical either way.
    fp32_value = None
    if not args.skip_fp32 and precision == 1:
        k32 = max(1, args.steps // 2)
        overlap = B.ddppo_launch_overlap()
        B.ddppo_set_launch_overlap(False)
        try:
            w32, ms32, _, _, _, _ = measure(0, k32, max(3, args.warmup // 2), False)
        finally:
            B.ddppo_set_launch_overlap(overlap)
        fp32_value, _, _ = aggregate(w32.E * w32.T * k32, ms32, torch.device("cuda"))
        w32.close()

    peaks, pk_kind = _peaks()
    g_ms, g_n, g_flops = gemm
    tc_flops_share = (tc[2] / tc[0]) if tc[0] > 0 else 0.0
    if precision == 1 and tc[1] > 0:
        compute, cunit = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]), "tensor"
    else:
        # SIMT FMA path: 152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock
        compute, cunit = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12, "alu"
    hbm = peaks["hbm_gbs"]
    # each launch's own roofline time: max(FLOP / compute peak, bytes / HBM peak)
    l_ms, l_fl, l_by = per_launch
    t_act = sum(l_ms) / 1e3
    t_c = sum(f / (compute * 1e12) for f, b in zip(l_fl, l_by) if f / (compute * 1e12) >= b / (hbm * 1e9))
    t_m = sum(b / (hbm * 1e9) for f, b in zip(l_fl, l_by) if f / (compute * 1e12) < b / (hbm * 1e9))
    mixed_frac = (t_c + t_m) / t_act if t_act > 0 else None
    if t_m >= t_c:
        bound, unit, peak_v = "hbm", "GB/s", hbm
        achieved = sum(l_by) / t_act / 1e9 if t_act > 0 else 0.0
    else:
        bound, unit, peak_v = cunit, "TFLOP/s", compute
        achieved = sum(l_fl) / t_act / 1e12 if t_act > 0 else 0.0
    r_ms, r_n, r_bytes = rc
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if precision == 1 else "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "num_envs": w.E, "rollout_T": w.T, "epochs": 2,
                   "minibatches": 2, "grid": "128x128 rooms, 0.1 m", "depth": "256x256 -> 128x128",
                   "encoder": "resnet18-style base 32, GroupNorm", "lstm": "2x512",
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "working set (activations ~tens of GB) larger than L2; no flush"},
        "fp32_value": round(fp32_value, 2) if fp32_value else None,
        "bf16_over_fp32": round(value / fp32_value, 3) if fp32_value else None,
        "fp32_launch": "plain stream order (its faster setting)" if fp32_value else None,
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": w.launches_per_step() * args.steps,
        "roofline": {"bound": bound, "kernel": "gemm (all contractions of the update)",
                     "achieved": round(achieved, 3), "peak": round(peak_v, 1), "unit": unit,
                     "frac": round(achieved / peak_v, 4) if peak_v else None,
                     "peak_kind": pk_kind, "launches": g_n, "avg_launch_us": round(1e3 * g_ms / max(g_n, 1), 2),
                     "tcgen05_flop_share": round(tc_flops_share, 4),
                     "achieved_tflops": round(g_flops / (g_ms / 1e3) / 1e12, 2) if g_ms > 0 else None,
                     "frac_of_per_launch_roofline": round(mixed_frac, 4) if mixed_frac else None,
                     "algorithmic_bytes_per_launch": round(sum(l_by) / max(len(l_by), 1)),
                     "traffic": round(GEMM_TRAFFIC_OVER_ALGORITHMIC * sum(l_by) / max(len(l_by), 1)),
                     "traffic_source": "dram bytes per launch, the T = 16 ncu capture's traffic / "
                                       "algorithmic ratio (%.3f) times this run's algorithmic "
                                       "bytes" % GEMM_TRAFFIC_OVER_ALGORITHMIC},
        "raycast": {"launches": r_n, "avg_launch_us": round(1e3 * r_ms / max(r_n, 1), 2),
                "kernel": "env_step render (TMA-staged DDA ray cast, 64 x 256x256 -> 128x128 bf16)",
                    "out_GBps": round(r_bytes / (r_ms / 1e3) / 1e9, 2) if r_ms > 0 else None},
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(sample_steps: int = 1):
    """The float64 oracle timed on the host cores on a bounded sample of the workload:
    the same network and world, 4 envs x 16 frames per iteration, 2 epochs x 2 minibatches."""
    from oracle import loop as OL
    import torch
    r = OL.OracleLoop(num_envs=4, T=16, seed=3)
    r.iterate()  # warm-up (allocations, first-touch)
    t0 = time.perf_counter()
    for _ in range(sample_steps):
        r.iterate()
    dt = time.perf_counter() - t0
    frames = r.E * r.T * sample_steps
    return {"value": round(frames / dt, 3), "unit": UNIT, "cores": torch.get_num_threads(),
            "kind": "oracle",
            "sample": "float64 oracle, %d iteration(s) of 4 envs x 16 frames (same ResNet-18/32 + "
                      "2x512 LSTM, 128x128 rooms, 256x256 depth), 2 epochs x 2 minibatches" % sample_steps}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return
    from oracle import loop as OL
    import torch
    name, e, t, sim, net, pool, mb = ORACLE_SAMPLES[args.workload]
    r = OL.OracleLoop(num_envs=e, T=t, seed=3, minibatches=mb, sim=sim, net=net, pool=pool)
    for _ in range(args.warmup):
        r.iterate()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.iterate()
    dt = time.perf_counter() - t0
    frames = r.E * r.T * args.steps
    v = frames / dt
    sample = ("float64 oracle, each step = 1 iteration of %d envs x %d frames of the workload's "
              "worlds and network, %d epochs x %d minibatches" % (e, t, 2, mb))
    WL = name
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WL, "sample": sample},
            "cpu_baseline": {"value": round(v, 3), "unit": UNIT, "cores": torch.get_num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--skip-fp32", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=6,
                    help="oracle iterations timed for cpu_baseline (about 10-20 s of host work)")
    ap.add_argument("--workload", default="resnet", choices=sorted(ORACLE_SAMPLES),
                    help="reference arm only: the workload whose oracle sample is timed")
    ap.add_argument("--rollout-T", type=int, default=None,
                    help="shorter rollout for profiler launch lists (not a bench value)")
    ap.add_argument("--profile", action="store_true",
                    help="timed steps only (for ncu); prints no bench line")
    ap.add_argument("--tune-cache", default=None,
                    help="GEMM tuning table: loaded if the file exists, else written after the "
                         "warm-up (a profiled run then launches the plain run's configurations)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native" and not args.profile:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
