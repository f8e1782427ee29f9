"""Roofline fractions of the bandwidth-bound kernels of the path, each timed through its
C-ABI entry with CUDA events on the launching stream (median of the repetitions, L2
flushed before each one by writing a buffer larger than L2, so every launch reads HBM).

    python -m paper_1911_00357_gb300.kernel_bench [--reps 15] [--peak-gbs 6783.8]

Algorithmic bytes per unit (each operand read once, each result written once):
  gae         17 B per sample: reward 4, done 1, value 4 read; advantage 4, return 4 written
              (Sec. 4 "Training": GAE over the rollout)
  ppo_loss    56 B per sample: logits 16, value 4, action 4, old log-prob 4, advantage 4,
              return 4 read; logit gradient 16, value gradient 4 written (Eq. 2 and its
              exact gradient)
  adam        28 B per parameter: gradient, parameter, m, v read (16); parameter, m, v
              written (12). Timed as the whole optimizer step (ddppo_apply_grad: gradient
              scaling, global-norm clip, Adam, GEMM-layout weight refresh), so the
              fraction charges the other passes to Adam's bytes
  group_norm  12 B per element with a residual (z, residual read; output written), 8 without
              (App. "Visual Encoder": GroupNorm). z is read twice (statistics, then
              normalise): the one-launch form re-reads each block's rows right after summing
              them (an L2 hit when the batch fits L2); the two-launch form, taken when the
              grid cannot be resident at once, reads z from HBM twice (ceiling 2/3, or 3/4
              with a residual)
  env_step    84 B of state, action and outputs per env plus the observation written
              (depth H x W in the operand dtype); the step is bound by the ray cast's ALU
              work, so the HBM fraction is reported for completeness. The next episodes are
              prepared (untimed) before each timed step, as in the collect loop

  lstm        the 2-layer 512 LSTM forward over T = 128 steps of 32 envs (one update
              minibatch of the ResNet workload, BF16) in each recurrence mode: 0 step by
              step, 1 whole segment on CUDA cores, 2 whole segment on tcgen05 (times only)

    python -m paper_1911_00357_gb300.kernel_bench --only lstm group_norm

Each line is one JSON object; `frac` is achieved / peak, the peak being the measured copy
bandwidth passed in (the GB/s of a plain device copy on this GPU model). A measurement
tool; the headline number is bench.py's.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .worker import Worker

L2_FLUSH_BYTES = 512 << 20


class _Timer:
    def __init__(self, reps: int):
        self.reps = reps
        self.flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def __call__(self, fn, pre=None) -> float:
        s = torch.cuda.current_stream()
        if pre:
            pre()
        fn()  # warm-up (first-call allocations, lookups)
        times = []
        for _ in range(self.reps):
            if pre:
                pre()  # untimed set-up on the same stream
            self.flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(s)
            fn()
            e1.record(s)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2]


def _line(kernel, workload, units, unit_name, bytes_per_unit, ms, peak, **extra):
    gbs = bytes_per_unit * units / (ms * 1e-3) / 1e9
    d = {"kernel": kernel, "workload": workload, unit_name: units, "bytes_per_unit": bytes_per_unit,
         "ms": round(ms, 5), "achieved_gbs": round(gbs, 1), "peak_gbs": peak,
         "frac": round(gbs / peak, 4)}
    d.update(extra)
    print(json.dumps(d), flush=True)


def bench_gae(tm, peak):
    for T, E, name in ((128, 64, "T128 x E64 (ResNet-18/32 workload)"),
                       (128, 1024, "T128 x E1024 (mixed-grid workload)"),
                       (128, 4096, "T128 x E4096 (4096-env workload)"),
                       (128, 262144, "T128 x E262144 (HBM-sized)")):
        g = torch.Generator(device="cuda").manual_seed(1)
        r = torch.randn(T, E, device="cuda", generator=g)
        d = (torch.rand(T, E, device="cuda", generator=g) < 0.01).to(torch.uint8)
        v = torch.randn(T + 1, E, device="cuda", generator=g)
        adv = torch.empty(T, E, device="cuda")
        ret = torch.empty(T, E, device="cuda")
        ms = tm(lambda: B.ddppo_gae(r, d, v, T, E, 0.99, 0.95, adv, ret))
        _line("gae", name, T * E, "samples", 17, ms, peak)


def bench_loss(tm, peak):
    for n, name in ((4096, "4096 samples (one minibatch, T128 x E64 / 2)"),
                    (131072, "131072 samples (one minibatch, T128 x E4096 / 4)"),
                    (1048576, "1048576 samples (largest)")):
        g = torch.Generator(device="cuda").manual_seed(2)
        lg = torch.randn(n, 4, device="cuda", generator=g)
        val = torch.randn(n, device="cuda", generator=g)
        act = torch.randint(0, 4, (n,), device="cuda", generator=g, dtype=torch.int32)
        lpo = torch.log_softmax(lg + 0.1 * torch.randn(n, 4, device="cuda", generator=g), -1)
        lpo = lpo.gather(1, act.long()[:, None])[:, 0].contiguous()
        adv = torch.randn(n, device="cuda", generator=g)
        ret = torch.randn(n, device="cuda", generator=g)
        st = torch.zeros(B.NSTATS, device="cuda")
        dl = torch.empty(n, 4, device="cuda")
        dv = torch.empty(n, device="cuda")
        ms = tm(lambda: B.ddppo_ppo_loss_static(n, lg, val, act, lpo, adv, ret, 0.2, 0.5, 0.01,
                                                st, dl, dv))
        _line("ppo_loss", name, n, "samples", 56, ms, peak)


def bench_group_norm(tm, peak):
    for N, HW, C, resid, name in ((256, 64 * 64, 32, True, "256 images x 64x64 x 32 ch, residual + ReLU"),
                                  (256, 64 * 64, 32, False, "256 images x 64x64 x 32 ch, ReLU"),
                                  (1024, 8 * 8, 256, True, "1024 images x 8x8 x 256 ch, residual + ReLU")):
        g = torch.Generator(device="cuda").manual_seed(3)
        z = torch.randn(N, HW, C, device="cuda", generator=g)
        gm = torch.rand(C, device="cuda", generator=g) + 0.5
        bt = torch.randn(C, device="cuda", generator=g)
        rs = torch.randn(N, HW, C, device="cuda", generator=g) if resid else None
        out = torch.empty_like(z)
        mean = torch.empty(N, C // 2, device="cuda")
        rstd = torch.empty(N, C // 2, device="cuda")
        ms = tm(lambda: B.ddppo_group_norm(z, gm, bt, out, mean, rstd, resid=rs, relu=True))
        _line("group_norm", name, N * HW * C, "elements", 12 if resid else 8, ms, peak)


def bench_worker_kernels(tm, peak, presets):
    for preset in presets:
        w = Worker(preset, seed=0)
        try:
            P = B.ddppo_num_params(w.h)
            grad = torch.randn(P, device="cuda") * 1e-3
            hp = B.default_hparams()
            ms = tm(lambda: B.ddppo_apply_grad(w.h, grad, 1.0, hp))
            _line("adam", f"{preset}: {P} parameters (whole optimizer step)", P, "params", 28, ms,
                  peak)
            E = w.E
            t = w.t
            B.ddppo_env_reset(w.h, t["obs"][0], t["goal"][0])
            acts = torch.randint(0, 4, (E,), device="cuda", dtype=torch.int32)
            ob = t["obs"][0]
            obs_bytes = ob[0].numel() * ob.element_size()
            # the next episode of every env prepared beforehand (untimed), as the collect
            # loop does on its side stream: the step adopts it instead of generating one
            ms = tm(lambda: B.ddppo_env_step(w.h, acts, t["obs"][1], t["goal"][1], t["rewards"][0],
                                             t["dones"][0]),
                    pre=lambda: B.ddppo_env_prefetch(w.h))
            _line("env_step", f"{preset}: {E} envs, obs {tuple(ob.shape[1:])} {ob.dtype}", E,
                  "envs", 84 + obs_bytes, ms, peak, bound="alu (ray cast)",
                  env_steps_per_s=round(E / (ms * 1e-3), 1))
            assert B.ddppo_device_status(w.h) == 0
        finally:
            w.close()


def bench_lstm(tm, peak):
    from .presets import make_config
    T, E = 128, 32
    cfg = make_config("resnet", num_envs=64, rollout_T=T, precision=1)
    h = B.ddppo_create(cfg)
    try:
        P = B.ddppo_num_params(h)
        g = torch.Generator(device="cuda").manual_seed(5)
        B.ddppo_set_params(h, torch.randn(P, device="cuda", generator=g) * 0.02)
        x = torch.randn(T, E, cfg.hidden + 64, device="cuda", generator=g)
        m = torch.ones(T, E, dtype=torch.uint8, device="cuda")
        h0 = torch.zeros(cfg.lstm_layers, E, cfg.hidden, device="cuda")
        c0 = torch.zeros_like(h0)
        y = torch.zeros(T, E, cfg.hidden, device="cuda")
        for mode in (0, 1, 2):
            B.ddppo_lstm_whole_segment(h, mode)
            ms = tm(lambda: B.ddppo_lstm_forward(h, T, E, x, m, h0, c0, y))
            print(json.dumps({"kernel": "lstm_forward", "mode": mode, "workload":
                              "2 layers x 512, T 128 x E 32, BF16", "ms": round(ms, 4),
                              "us_per_step_and_layer": round(1e3 * ms / (T * cfg.lstm_layers), 2)}),
                  flush=True)
        assert B.ddppo_device_status(h) == 0
    finally:
        B.ddppo_destroy(h)


BENCHES = {"gae": bench_gae, "ppo_loss": bench_loss, "group_norm": bench_group_norm,
           "lstm": bench_lstm}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--reps", type=int, default=15)
    ap.add_argument("--only", nargs="+", default=None,
                    choices=sorted(BENCHES) + ["adam_env_step"],
                    help="run these benches only (adam_env_step: the worker-based ones)")
    ap.add_argument("--peak-gbs", type=float, default=6783.8,
                    help="measured device-copy bandwidth (GB/s) used as the roofline peak")
    ap.add_argument("--presets", nargs="+", default=["resnet", "wide_256", "mixed_1024"])
    args = ap.parse_args()
    tm = _Timer(args.reps)
    only = args.only or (sorted(BENCHES) + ["adam_env_step"])
    for name in ("gae", "ppo_loss", "group_norm", "lstm"):
        if name in only:
            BENCHES[name](tm, args.peak_gbs)
    if "adam_env_step" in only:
        bench_worker_kernels(tm, args.peak_gbs, args.presets)


if __name__ == "__main__":
    main()
