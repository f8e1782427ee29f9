"""A DD-PPO worker on one GPU: rollout buffers in device memory (allocated with torch)
and the synchronous collect -> GAE -> PPO-update iteration (Sec. 3; Sec. 4 "Training"),
every step of which runs in the CUDA library through the C ABI."""
from __future__ import annotations

import torch

from . import binding as B
from .presets import make_config


class Worker:
    def __init__(self, preset: str = "resnet", precision: int | None = None, seed: int = 0,
                 gamma: float = 0.99, lam: float = 0.95, hparams: dict | None = None, **overrides):
        kw = dict(overrides)
        if precision is not None:
            kw["precision"] = precision
        self.cfg = cfg = make_config(preset, seed=seed, **kw)
        self.h = B.ddppo_create(cfg)
        self.E, self.T, self.L, self.H = cfg.num_envs, cfg.rollout_T, cfg.lstm_layers, cfg.hidden
        self.gamma, self.lam = gamma, lam
        E, T, L, H = self.E, self.T, self.L, self.H
        oh = cfg.depth_h >> cfg.pool2x2
        od = torch.bfloat16 if cfg.precision >= 1 else torch.float32
        dev = "cuda"
        z = lambda *s, dt=torch.float32: torch.zeros(*s, dtype=dt, device=dev)
        self.t = {
            "obs": z(T + 1, E, 1, oh, oh, dt=od), "goal": z(T + 1, E, 3),
            "prev_a": z(T + 1, E, dt=torch.int32), "masks": z(T + 1, E, dt=torch.uint8),
            "actions": z(T, E, dt=torch.int32), "logp": z(T, E), "values": z(T + 1, E),
            "rewards": z(T, E), "dones": z(T, E, dt=torch.uint8), "info": z(T, E, 4),
            "adv": z(T, E), "ret": z(T, E), "h0": z(L, E, H), "c0": z(L, E, H),
            "h": z(L, E, H), "c": z(L, E, H), "uniforms": z(T, E),
        }
        self.view = B.Rollout()
        for k, v in self.t.items():
            setattr(self.view, k, v.data_ptr())
        hp = dict(minibatches=cfg.minibatches)
        hp.update(hparams or {})
        self.hp = B.default_hparams(**hp)
        self.stats = z(self.hp.epochs * self.hp.minibatches, B.NSTATS)
        self.updates = 0
        self._gen = torch.Generator(device=dev)
        self._gen.manual_seed(seed + 12345)
        self._pool = torch.rand(8, T, E, generator=self._gen, device=dev)
        self._k = 0

    def close(self):
        if self.h is not None:
            B.ddppo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # one synchronous iteration; uniforms already resident in HBM
    def iterate(self, uniforms: torch.Tensor | None = None):
        u = self._pool[self._k % self._pool.shape[0]] if uniforms is None else uniforms
        self._k += 1
        self.t["uniforms"].copy_(u, non_blocking=True)
        B.ddppo_collect(self.h, self.view, True)
        t = self.t
        B.ddppo_gae(t["rewards"], t["dones"], t["values"], self.T, self.E, self.gamma, self.lam,
                    t["adv"], t["ret"])
        self.hp.update_index = self.updates
        B.ddppo_ppo_update(self.h, self.view, self.hp, self.stats)
        self.updates += 1

    def save(self, path: str):
        """Checkpoint the worker: the library's state (parameters, Adam, world, tuning
        table, the rollout state carried into the next collect) in `path`, and the loop's
        own counters (updates done, position in the uniform pool) in `path` + ".loop"."""
        B.ddppo_save(self.h, path, self.view)
        with open(path + ".loop", "w") as f:
            f.write("%d %d\n" % (self.updates, self._k))

    def load(self, path: str):
        """Resume from a checkpoint of a worker with the same preset, seed and overrides."""
        B.ddppo_load(self.h, path, self.view)
        with open(path + ".loop") as f:
            self.updates, self._k = (int(v) for v in f.read().split())

    def time_e2e(self, steps: int):
        """Steps through the public API with host buffers: each step copies its action
        uniforms host->device (pinned) and reads the PPO statistics, rewards and done flags
        device->host. Returns (ms, h2d bytes per step, d2h bytes per step)."""
        T, E = self.T, self.E
        host_u = torch.rand(steps, T, E, generator=torch.Generator().manual_seed(7)).pin_memory()
        dev_u = torch.empty(T, E, device="cuda")
        out_stats = torch.empty(steps, *self.stats.shape).pin_memory()
        out_r = torch.empty(steps, T, E).pin_memory()
        out_d = torch.empty(steps, T, E, dtype=torch.uint8).pin_memory()
        torch.cuda.synchronize()
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for i in range(steps):
            dev_u.copy_(host_u[i], non_blocking=True)
            self.iterate(dev_u)
            out_stats[i].copy_(self.stats, non_blocking=True)
            out_r[i].copy_(self.t["rewards"], non_blocking=True)
            out_d[i].copy_(self.t["dones"], non_blocking=True)
        e1.record(s)
        torch.cuda.synchronize()
        h2d = T * E * 4
        d2h = self.stats.numel() * 4 + T * E * 4 + T * E
        return e0.elapsed_time(e1), h2d, d2h

    def time_raycast(self, steps: int):
        """Ray-cast launches of `steps` env steps run outside the collect graph, with the
        library's event timer on the render kernel: (ms, launches, output bytes)."""
        t = self.t
        E = self.E
        act = torch.randint(1, 4, (steps, E), dtype=torch.int32, device="cuda")
        obs = torch.empty_like(t["obs"][0])
        goal = torch.empty_like(t["goal"][0])
        r = torch.empty(E, device="cuda")
        d = torch.empty(E, dtype=torch.uint8, device="cuda")
        B.ddppo_timing_enable(self.h, True)
        for i in range(steps):
            B.ddppo_env_step(self.h, act[i], obs, goal, r, d)
        out = B.ddppo_timing_read(self.h, 1)
        B.ddppo_timing_enable(self.h, False)
        return out

    def launches_per_step(self) -> int:
        return B.ddppo_count_kernels(self.h, self.view, self.hp, self.gamma, self.lam)

    def tensor_core_gemm(self) -> bool:
        ms, n, flops = B.ddppo_timing_read(self.h, 2)
        return n > 0
