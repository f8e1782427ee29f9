"""Micro-benchmark of the library's contraction (``ddppo_gemm``) on one shape.

  python -m paper_1911_00357_gb300.gemm_bench --M 524288 --N 32 --K 288 [--a-t] [--b-t]
  python -m paper_1911_00357_gb300.gemm_bench --conv N,H,W,C,Cout,k,s,p [--wgrad]

The --conv form times the implicit-im2col convolution (``ddppo_conv2d``) or its weight
gradient (``ddppo_conv2d_wgrad``) on NHWC bf16 input; its algorithmic bytes are the input,
the output gradient or output, and the weights, each once.

Prints achieved TFLOP/s and the algorithmic HBM bytes per launch (A + B read once, C
written once) over the CUDA-event time of --reps launches after --warmup launches.
The default shape is the forward GEMM of a first-stage 3x3 convolution (32 -> 32
channels at 32x32) over 512 frames of the ResNet-18/32 encoder.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=524288)
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--K", type=int, default=288)
    ap.add_argument("--a-t", action="store_true")
    ap.add_argument("--b-t", action="store_true")
    ap.add_argument("--dtype", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--conv", default=None, help="N,H,W,C,Cout,k,s,p")
    ap.add_argument("--wgrad", action="store_true")
    args = ap.parse_args()
    if args.conv:
        return conv_main(args)
    dt = torch.bfloat16 if args.dtype == "bf16" else torch.float32
    M, N, K = args.M, args.N, args.K
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn(*((K, M) if args.a_t else (M, K)), device="cuda", generator=g).to(dt)
    Bm = torch.randn(*((K, N) if args.b_t else (N, K)), device="cuda", generator=g).to(dt)
    C = torch.empty(M, N, device="cuda")
    for _ in range(args.warmup):
        B.ddppo_gemm(A, Bm, C, a_t=args.a_t, b_t=args.b_t)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        B.ddppo_gemm(A, Bm, C, a_t=args.a_t, b_t=args.b_t)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    es = 2 if dt == torch.bfloat16 else 4
    byts = (M * K + N * K) * es + M * N * 4
    print(json.dumps({"M": M, "N": N, "K": K, "a_t": args.a_t, "b_t": args.b_t, "dtype": args.dtype,
                      "us_per_launch": round(ms * 1e3, 2),
                      "tflops": round(2.0 * M * N * K / (ms / 1e3) / 1e12, 2),
                      "hbm_GBps_algorithmic": round(byts / (ms / 1e3) / 1e9, 1),
                      "tensor_cores": B.ddppo_gemm_backend(A if not args.a_t else A.t(),
                                                           Bm if not args.b_t else Bm.t())}))


def conv_main(args):
    N, H, W, C, Co, k, s, p = (int(v) for v in args.conv.split(","))
    Ho, Wo = (H + 2 * p - k) // s + 1, (W + 2 * p - k) // s + 1
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(N, H, W, C, device="cuda", generator=g).to(torch.bfloat16)
    if args.wgrad:
        dy = torch.randn(N, Ho, Wo, Co, device="cuda", generator=g).to(torch.bfloat16)
        dw = torch.zeros(Co, k * k * C, device="cuda")
        run = lambda: B.ddppo_conv2d_wgrad(x, dy, dw, k, s, p)
        byts = x.numel() * 2 + dy.numel() * 2 + dw.numel() * 4
    else:
        w = torch.randn(Co, k * k * C, device="cuda", generator=g).to(torch.bfloat16)
        y = torch.empty(N, Ho, Wo, Co, device="cuda")
        run = lambda: B.ddppo_conv2d(x, w, y, k, s, p)
        byts = x.numel() * 2 + w.numel() * 2 + y.numel() * 4
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.reps
    flops = 2.0 * N * Ho * Wo * Co * k * k * C
    print(json.dumps({"conv": args.conv, "wgrad": args.wgrad, "us_per_launch": round(ms * 1e3, 2),
                      "tflops": round(flops / (ms / 1e3) / 1e12, 2),
                      "hbm_GBps_algorithmic": round(byts / (ms / 1e3) / 1e9, 1)}))


if __name__ == "__main__":
    main()
