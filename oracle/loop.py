"""The whole DD-PPO iteration on the float64 oracle (Sec. 3; Sec. 4 "Training").

TEST INFRASTRUCTURE ONLY: timed as the CPU baseline and the reference arm of the
benchmark. Collect T frames from E envs with the oracle simulator and policy, bootstrap,
GAE, then ppo_update -- in the order the paper's synchronous loop runs them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import policy as P
from . import rl as R
from . import sim as S

DT = torch.float64


def init_params(cfg: P.NetConfig, seed: int) -> torch.Tensor:
    """Seeded initial weights (N(0, 1/fan_in) weights, unit GroupNorm gains, zero biases)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for name, shp in P.param_spec(cfg):
        n = int(np.prod(shp))
        if name.endswith(".g"):
            parts.append(torch.ones(n, dtype=DT))
        elif len(shp) == 1:
            parts.append(torch.zeros(n, dtype=DT))
        else:
            parts.append(torch.randn(n, generator=g, dtype=DT) / np.sqrt(int(np.prod(shp[1:]))))
    return torch.cat(parts)


class OracleLoop:
    """By default the ResNet-18-style (32 base) agent with a 2-layer 512 LSTM on 128x128
    rooms grids at 0.1 m with 256x256 depth pooled to 128x128 (the paper-shaped
    single-GPU workload). sim / net: SimConfig / NetConfig fields that replace those
    defaults (another workload); pool: the 2x2 average pool of the depth image."""

    def __init__(self, num_envs: int = 4, T: int = 16, seed: int = 0, minibatches: int = 2,
                 sim: dict | None = None, net: dict | None = None, pool: bool = True):
        self.E, self.T = num_envs, T
        skw = dict(num_envs=num_envs, gen_kind=1, grid_min=128, grid_max=128, cell_m=0.1,
                   depth_h=256, depth_w=256, seed=seed)
        skw.update(sim or {})
        self.scfg = S.SimConfig(**skw)
        nkw = dict(net_kind=1, base_ch=32, hidden=512, lstm_layers=2, in_h=128, in_w=128)
        nkw.update(net or {})
        self.ncfg = P.NetConfig(**nkw)
        self.pool = pool
        self.hp = R.PPOHParams(minibatches=minibatches)
        self.seed = seed
        self.sim = S.BatchSim(self.scfg)
        self.sim.reset()
        self.flat = init_params(self.ncfg, seed)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.step = 0
        self.update = 0
        L, H = self.ncfg.lstm_layers, self.ncfg.hidden
        self.h = torch.zeros(L, num_envs, H, dtype=DT)
        self.c = torch.zeros(L, num_envs, H, dtype=DT)
        depth, goal = self.sim.render()
        self.obs = torch.from_numpy(S.pool_obs(depth, self.pool, self.scfg.max_depth_m)).unsqueeze(1)
        self.goal = torch.from_numpy(goal)
        self.prev_a = torch.full((num_envs,), 4, dtype=torch.int32)
        self.masks = torch.zeros(num_envs, dtype=torch.uint8)
        self.rng = np.random.default_rng(seed)

    def iterate(self):
        E, T = self.E, self.T
        p = P.unflatten(self.flat, self.ncfg)
        ro = {k: [] for k in ("obs", "goal", "prev_a", "masks", "actions", "logp_old")}
        values, rewards, dones = [], [], []
        h0, c0 = self.h.clone(), self.c.clone()
        with torch.no_grad():
            for t in range(T):
                u = torch.from_numpy(self.rng.random(E))
                a, lp, v, self.h, self.c, _ = P.act(p, self.obs, self.goal, self.prev_a, self.masks,
                                                    self.h, self.c, u, self.ncfg)
                for k, x in (("obs", self.obs), ("goal", self.goal), ("prev_a", self.prev_a),
                             ("masks", self.masks), ("actions", a), ("logp_old", lp)):
                    ro[k].append(x)
                values.append(v)
                r, d, _, _ = self.sim.step(a.numpy().astype(np.int32))
                rewards.append(r)
                dones.append(d)
                depth, goal = self.sim.render()
                self.obs = torch.from_numpy(S.pool_obs(depth, self.pool, self.scfg.max_depth_m)).unsqueeze(1)
                self.goal = torch.from_numpy(goal)
                dt = torch.from_numpy(d.astype(np.int32))
                self.prev_a = torch.where(dt == 1, torch.full_like(a, 4), a).to(torch.int32)
                self.masks = (1 - dt).to(torch.uint8)
            _, _, vT, _, _, _ = P.act(p, self.obs, self.goal, self.prev_a, self.masks, self.h, self.c,
                                      torch.zeros(E, dtype=DT), self.ncfg)
        V = torch.stack(values + [vT]).numpy()
        adv, ret = R.gae(np.stack(rewards), np.stack(dones), V, self.hp.gamma, self.hp.lam)
        rollout = {k: torch.stack(v) for k, v in ro.items()}
        rollout["adv"] = torch.from_numpy(adv)
        rollout["ret"] = torch.from_numpy(ret)
        rollout["h0"], rollout["c0"] = h0, c0
        self.flat, self.m, self.v, self.step, stats = R.ppo_update(
            self.flat, self.m, self.v, self.step, rollout, self.ncfg, self.hp, self.seed, self.update)
        self.update += 1
        return stats
