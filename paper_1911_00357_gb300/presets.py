"""Named workloads (synthetic stand-ins for the paper's Gibson/MP3D training runs).

  nature_fp32 : 16 envs, 32x32 Bernoulli grids (0.25 m cells, density 0.15), depth 64x64,
                3-layer conv 32/64/32 -> LSTM 128, T=32, FP32.
  resnet      : 64 envs, 128x128 rooms-and-doors grids at 0.1 m, depth 256x256 pooled to
                128x128, ResNet-18-style encoder (32 base, GroupNorm) -> 2-layer LSTM 512,
                T=128, 2 epochs x 2 minibatches (the paper-shaped single-GPU run).
  mixed_1024  : 1024 envs on grids drawn from {64,128,256,512}^2, depth 128x128, BF16.
  wide_256    : 256 envs, 64-base encoder, depth 256x256 pooled.
  wide_256_fp8: wide_256 with FP8 (E4M3, per-tensor scales) inference and BF16 training.
  scale_4096  : 4096 envs x T=128, 4 minibatches.
  blind       : the resnet workload's worlds with the blind agent (GPS+Compass only, no
                visual encoder; Sec. 5).
"""
from __future__ import annotations

from .binding import Config

_BASE = dict(num_envs=16, gen_kind=0, grid_min=32, grid_max=32, cell_m=0.25, wall_density=0.15,
             door_m=0.8, min_room=8, max_steps=500, terminal_mode=0, depth_h=64, depth_w=64,
             pool2x2=0, cam_h_m=0.88, ceil_h_m=2.5, max_depth_m=10.0, net_kind=0, base_ch=32,
             hidden=128, lstm_layers=1, precision=0, rollout_T=32, minibatches=2,
             encoder_chunk=0, task=0, explore_m=1.0, seed=0)

PRESETS = {
    "nature_fp32": dict(),
    "resnet": dict(num_envs=64, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1, depth_h=256,
                   depth_w=256, pool2x2=1, net_kind=1, base_ch=32, hidden=512, lstm_layers=2,
                   rollout_T=128, minibatches=2, precision=1),
    "mixed_1024": dict(num_envs=1024, gen_kind=1, grid_min=64, grid_max=512, cell_m=0.1,
                       depth_h=128, depth_w=128, pool2x2=0, net_kind=1, base_ch=32, hidden=512,
                       lstm_layers=2, rollout_T=128, minibatches=2, precision=1),
    "wide_256": dict(num_envs=256, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1,
                     depth_h=256, depth_w=256, pool2x2=1, net_kind=1, base_ch=64, hidden=512,
                     lstm_layers=2, rollout_T=128, minibatches=2, precision=1, encoder_chunk=4096),
    "wide_256_fp8": dict(num_envs=256, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1,
                         depth_h=256, depth_w=256, pool2x2=1, net_kind=1, base_ch=64, hidden=512,
                         lstm_layers=2, rollout_T=128, minibatches=2, precision=2,
                         encoder_chunk=4096),
    "blind": dict(num_envs=64, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1, depth_h=256,
                  depth_w=256, pool2x2=1, net_kind=2, hidden=512, lstm_layers=2, rollout_T=128,
                  minibatches=2, precision=1),
    "scale_4096": dict(num_envs=4096, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1,
                       depth_h=256, depth_w=256, pool2x2=1, net_kind=1, base_ch=32, hidden=512,
                       lstm_layers=2, rollout_T=128, minibatches=4, precision=1),
}


def make_config(name: str = "nature_fp32", **overrides) -> Config:
    d = dict(_BASE)
    d.update(PRESETS[name])
    d.update(overrides)
    return Config(**d)
