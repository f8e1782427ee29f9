"""Helpers for the GPU parity tests: build the oracle's configuration from the C
ABI configuration (same float32 values) and allocate device buffers."""
from __future__ import annotations

import numpy as np
import torch

from oracle import policy as OP
from oracle import sim as OS
from paper_1911_00357_gb300 import binding as B


def sim_config_from(cfg: B.Config) -> OS.SimConfig:
    f = lambda v: float(np.float32(v))
    return OS.SimConfig(num_envs=cfg.num_envs, gen_kind=cfg.gen_kind, grid_min=cfg.grid_min,
                        grid_max=cfg.grid_max, cell_m=f(cfg.cell_m),
                        wall_density=f(cfg.wall_density), door_m=f(cfg.door_m),
                        min_room=cfg.min_room, max_steps=cfg.max_steps,
                        terminal_mode=cfg.terminal_mode, depth_h=cfg.depth_h, depth_w=cfg.depth_w,
                        cam_h_m=f(cfg.cam_h_m), ceil_h_m=f(cfg.ceil_h_m),
                        max_depth_m=f(cfg.max_depth_m), seed=cfg.seed)


def net_config_from(cfg: B.Config) -> OP.NetConfig:
    h = cfg.depth_h >> cfg.pool2x2
    kw = dict(net_kind=cfg.net_kind, base_ch=cfg.base_ch, hidden=cfg.hidden,
              lstm_layers=cfg.lstm_layers, in_h=h, in_w=h)
    if cfg.net_kind == 4:  # SE-ResNeXt101: the oracle's SE-ResNeXt with [3, 4, 23, 3] blocks
        kw.update(net_kind=3, sx_blocks=(3, 4, 23, 3))
    return OP.NetConfig(**kw)


def obs_shape(cfg: B.Config, *lead):
    h = cfg.depth_h >> cfg.pool2x2
    return (*lead, 1, h, h)


def obs_dtype(cfg: B.Config):
    return torch.bfloat16 if cfg.precision >= 1 else torch.float32


class Env:
    """Device buffers for stepping a worker's environments through the C ABI."""

    def __init__(self, cfg: B.Config):
        self.cfg = cfg
        self.h = B.ddppo_create(cfg)
        E = cfg.num_envs
        dev = "cuda"
        self.obs = torch.zeros(obs_shape(cfg, E), dtype=obs_dtype(cfg), device=dev)
        self.goal = torch.zeros(E, 3, device=dev)
        self.reward = torch.zeros(E, device=dev)
        self.done = torch.zeros(E, dtype=torch.uint8, device=dev)
        self.info = torch.zeros(E, 4, device=dev)
        self.state = torch.zeros(E, B.NSTATE, dtype=torch.int32, device=dev)
        G = cfg.grid_max * cfg.grid_max
        self.grids = torch.zeros(E, G, dtype=torch.uint8, device=dev)
        self.dists = torch.zeros(E, G, dtype=torch.int32, device=dev)
        self.depth = torch.zeros(E, cfg.depth_h, cfg.depth_w, device=dev)

    def close(self):
        if self.h is not None:
            B.ddppo_destroy(self.h)
            self.h = None

    def reset(self):
        B.ddppo_env_reset(self.h, self.obs, self.goal)

    def step(self, actions: np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(actions, np.int32)).cuda()
        B.ddppo_env_step(self.h, a, self.obs, self.goal, self.reward, self.done, self.info)

    def get_state(self) -> np.ndarray:
        B.ddppo_env_state(self.h, self.state)
        return self.state.cpu().numpy()

    def get_grids(self):
        B.ddppo_env_grids(self.h, self.grids, self.dists)
        return self.grids.cpu().numpy(), self.dists.cpu().numpy()

    def get_depth(self) -> np.ndarray:
        B.ddppo_env_depth(self.h, self.depth)
        return self.depth.cpu().numpy()
