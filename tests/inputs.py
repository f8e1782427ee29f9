"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds no arithmetic of the method: only named workload sizes and random draws
(numpy / torch generators with fixed seeds). Everything is returned in float64;
GPU tests cast to the kernel's dtype and feed the oracle the cast values.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import policy as P

DT = torch.float64

# Network sizes of the synthetic workloads (and small ones for tests).
#   nature     : 3-layer conv 32/64/32 (8/4/3), LSTM 128, depth 64x64 (16 envs, 32^2 grids)
#   resnet_b32 : ResNet-18-style, 32 base channels, 2-layer LSTM 512, depth 256^2 pooled to 128^2
#   resnet_b64 : the same with 64 base channels
#   tiny*      : small nets for finite differences and multi-tile parity cases
NETS = {
    "nature": dict(net_kind=0, base_ch=32, hidden=128, lstm_layers=1, in_h=64, in_w=64),
    "resnet_b32": dict(net_kind=1, base_ch=32, hidden=512, lstm_layers=2, in_h=128, in_w=128),
    "resnet_b64": dict(net_kind=1, base_ch=64, hidden=512, lstm_layers=2, in_h=128, in_w=128),
    "tiny": dict(net_kind=0, base_ch=32, hidden=8, lstm_layers=2, in_h=36, in_w=36),
    "tiny_resnet": dict(net_kind=1, base_ch=8, hidden=16, lstm_layers=2, in_h=32, in_w=32),
    "tiny_blind": dict(net_kind=2, base_ch=32, hidden=16, lstm_layers=2, in_h=32, in_w=32),
    "tiny_sx": dict(net_kind=3, base_ch=4, hidden=8, lstm_layers=1, in_h=32, in_w=32,
                    sx_blocks=(1, 1, 1, 1), cardinality=2, se_reduction=4),
}


def net_config(name: str) -> P.NetConfig:
    return P.NetConfig(**NETS[name])


def params(cfg: P.NetConfig, seed: int, scale: float = 1.0) -> torch.Tensor:
    """Flat float64 parameters in the canonical order: weights N(0, 1/fan_in),
    GroupNorm gains 1 + N(0, 0.1^2), biases N(0, 0.1^2)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for name, shp in P.param_spec(cfg):
        n = int(np.prod(shp))
        r = torch.randn(n, generator=g, dtype=DT)
        if name.endswith(".g"):
            parts.append(1.0 + 0.1 * r)
        elif len(shp) == 1:
            parts.append(0.1 * r)
        else:
            fan_in = int(np.prod(shp[1:]))
            parts.append(scale * r / np.sqrt(fan_in))
    return torch.cat(parts)


def rollout_inputs(cfg: P.NetConfig, T: int, E: int, seed: int) -> dict:
    g = torch.Generator().manual_seed(seed)
    obs = torch.rand(T, E, 1, cfg.in_h, cfg.in_w, generator=g, dtype=DT)
    ang = torch.rand(T, E, generator=g, dtype=DT) * 2 * np.pi
    r = torch.rand(T, E, generator=g, dtype=DT) * 10
    goal = torch.stack([r, torch.cos(ang), torch.sin(ang)], -1)
    prev_a = torch.randint(0, 5, (T, E), generator=g, dtype=torch.int32)
    masks = (torch.rand(T, E, generator=g) > 0.2).to(torch.uint8)
    return {"obs": obs, "goal": goal, "prev_a": prev_a, "masks": masks}


def minibatch(cfg: P.NetConfig, T: int, E: int, seed: int) -> dict:
    d = rollout_inputs(cfg, T, E, seed)
    g = torch.Generator().manual_seed(seed + 1000)
    d["actions"] = torch.randint(0, 4, (T, E), generator=g, dtype=torch.int32)
    d["logp_old"] = np.log(0.25) + 0.3 * torch.randn(T, E, generator=g, dtype=DT)
    d["adv"] = torch.randn(T, E, generator=g, dtype=DT)
    d["ret"] = torch.randn(T, E, generator=g, dtype=DT)
    d["h0"] = 0.5 * torch.randn(cfg.lstm_layers, E, cfg.hidden, generator=g, dtype=DT)
    d["c0"] = 0.5 * torch.randn(cfg.lstm_layers, E, cfg.hidden, generator=g, dtype=DT)
    return d


def uniforms(T: int, E: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).random((T, E)).astype(np.float32)


def random_actions(T: int, E: int, seed: int, p_stop: float = 0.02) -> np.ndarray:
    """Random navigation actions with a small stop probability."""
    rng = np.random.default_rng(seed)
    a = rng.integers(1, 4, size=(T, E)).astype(np.int32)
    a[rng.random((T, E)) < p_stop] = 0
    return a
