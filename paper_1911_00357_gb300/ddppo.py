"""DD-PPO's distributed pieces (Sec. 3): the gradient AllReduce of Eq. 4 and the preemption
threshold of the collection stage.

A worker is one library context: its own envs (its own world seed), rollout buffers,
parameter copy and CUDA stream. Workers either share one GPU (VirtualWorkers: the
AllReduce is ddppo_grad_mean over their gradient buffers and the "finished" counter is a
host integer) or own one GPU each in separate processes (DistributedWorker: the
AllReduce is torch.distributed.all_reduce, NCCL on GPUs, and the counter lives in a
torch.distributed store, the paper's TCPStore). In both, one iteration is:

  collect  every worker steps its envs; once ceil(p N) workers have finished their T
           steps, a worker that has taken at least T/4 steps stops (Sec. 3: stragglers are
           preempted, with a minimum of one quarter of the rollout); its rollout is then
           T_valid < T steps long;
  GAE      over each worker's own T_valid steps (bootstrapped at slot T_valid);
  update   for every epoch and minibatch: each worker's gradient over its own minibatch
           (the mean over its own samples: every worker weighs equally), the mean over
           workers, and the same clipped Adam step on every worker, so all parameter
           copies stay equal (Eq. 4).

Every step of the arithmetic runs in the CUDA library; this module orders the calls and
moves the gradient buffers between workers.
"""
from __future__ import annotations

import math
import time

import torch

from . import binding as B
from .worker import Worker


def min_steps(T: int) -> int:
    """The fewest steps a preempted worker collects: one quarter of the rollout (Sec. 3)."""
    return max(1, T // 4)


class PreemptionCounter:
    """How many workers have finished collecting this round, and the stop rule: a worker
    stops once ceil(p N) workers have finished their T steps, provided it has taken at
    least T/4 (p = 1: nobody is preempted). With `store` (a torch.distributed Store shared
    by the processes) the count is global; without, it counts the workers of this
    process."""

    def __init__(self, n_workers: int, p: float, T: int, store=None, prefix: str = "ddppo_done"):
        if not 0.0 < p <= 1.0:
            raise ValueError("preemption threshold p must be in (0, 1]")
        self.N, self.p, self.T = n_workers, p, T
        self.need = math.ceil(p * n_workers - 1e-9)
        self.store, self.prefix = store, prefix
        self.round = 0
        self.local = 0

    def new_round(self):
        self.round += 1
        self.local = 0

    def _key(self) -> str:
        return "%s/%d" % (self.prefix, self.round)

    def mark_finished(self):
        if self.store is None:
            self.local += 1
        else:
            self.store.add(self._key(), 1)

    def finished(self) -> int:
        return self.local if self.store is None else int(self.store.add(self._key(), 0))

    def should_stop(self, steps: int) -> bool:
        if steps >= self.T:
            return True
        return steps >= min_steps(self.T) and self.finished() >= self.need


def preempted_collection(step, T: int, counter: PreemptionCounter, wait=None) -> int:
    """One worker's collection under the preemption threshold: step(t) enqueues step t,
    wait() blocks until it has run. Returns the steps taken (T_valid)."""
    t = 0
    while not counter.should_stop(t):
        step(t)
        if wait is not None:
            wait()
        t += 1
        if t == T:
            counter.mark_finished()
    return t


def exchange_update(epochs: int, minibatches: int, grad, allreduce, apply):
    """Eq. 4 for one worker: for every epoch and minibatch, its gradient (grad(e, k) returns
    the buffer), the AllReduce across workers (in place), then the optimizer step."""
    for e in range(epochs):
        for k in range(minibatches):
            g = grad(e, k)
            allreduce(g)
            apply(g)


class VirtualWorkers:
    """N DD-PPO workers sharing one GPU, each on its own CUDA stream, so a straggler's
    steps (larger worlds to render and to reset) run beside the others'. worker w uses
    world seed `seed + w` and, with `grid_sides`, square grids of side grid_sides[w] (the
    heterogeneous workload: some workers' scenes cost more to simulate)."""

    def __init__(self, preset: str, n: int, p: float = 1.0, seed: int = 0, grid_sides=None,
                 hparams: dict | None = None, tune: bool = False, **overrides):
        self.n = n
        self.workers = []
        for w in range(n):
            kw = dict(overrides)
            if grid_sides is not None:
                kw.update(grid_min=grid_sides[w], grid_max=grid_sides[w])
            self.workers.append(Worker(preset, seed=seed + w, hparams=hparams, **kw))
        w0 = self.workers[0]
        self.T = w0.T
        self.P = B.ddppo_num_params(w0.h)
        if tune and w0.cfg.precision >= 1:
            # the GEMM autotuner times its candidates on worker 0 alone (every worker has
            # the same network shapes), then the table is frozen and shared: preempted
            # rollouts' new shapes take the fixed heuristic instead of timing trials
            # disturbed by the other workers' streams
            w0.iterate()
            table = B.ddppo_autotune_export(w0.h)
            for w in self.workers:
                if w is not w0:
                    B.ddppo_autotune_import(w.h, table)
                B.ddppo_autotune(w.h, False)
        else:
            for w in self.workers:
                B.ddppo_autotune(w.h, False)
        flat = torch.empty(self.P, device="cuda")
        B.ddppo_get_params(w0.h, flat)
        for w in self.workers:
            B.ddppo_set_params(w.h, flat)
        torch.cuda.synchronize()
        self.streams = [torch.cuda.Stream() for _ in range(n)]
        self.grads = [torch.zeros(self.P, device="cuda") for _ in range(n)]
        self.mean = torch.zeros(self.P, device="cuda")
        self.stats = [torch.zeros(B.NSTATS, device="cuda") for _ in range(n)]
        self.counter = PreemptionCounter(n, p, self.T)
        self.T_valid = [self.T] * n
        self.updates = 0

    def close(self):
        for w in self.workers:
            w.close()

    def set_threshold(self, p: float):
        """Change the preemption threshold (the next collection uses it)."""
        self.counter = PreemptionCounter(self.n, p, self.T)

    def collect(self) -> list[int]:
        """Every worker collects on its own stream, at most one step in flight each; the
        preemption rule decides when each stops. Returns the workers' T_valid."""
        c = self.counter
        c.new_round()
        cur = torch.cuda.current_stream()
        for w, s in zip(self.workers, self.streams):
            s.wait_stream(cur)
            with torch.cuda.stream(s):
                w.t["uniforms"].copy_(w._pool[w._k % w._pool.shape[0]], non_blocking=True)
                w._k += 1
                B.ddppo_collect_begin(w.h, w.view, s)
        steps = [0] * self.n
        marked = [False] * self.n
        stopped = [False] * self.n
        events = [None] * self.n
        while not all(stopped):
            for i, (w, s) in enumerate(zip(self.workers, self.streams)):
                if stopped[i] or (events[i] is not None and not events[i].query()):
                    continue
                if steps[i] == self.T and not marked[i]:
                    c.mark_finished()
                    marked[i] = True
                if c.should_stop(steps[i]):
                    stopped[i] = True
                    continue
                B.ddppo_collect_step(w.h, w.view, steps[i], s)
                ev = torch.cuda.Event()
                ev.record(s)
                events[i] = ev
                steps[i] += 1
        for w, s, tv in zip(self.workers, self.streams, steps):
            with torch.cuda.stream(s):
                B.ddppo_collect_end(w.h, w.view, tv, s)
                t = w.t
                B.ddppo_gae(t["rewards"], t["dones"], t["values"], tv, w.E, w.gamma, w.lam,
                            t["adv"], t["ret"])
        self.T_valid = steps
        return steps

    def update(self):
        """Eq. 4 over the workers: per minibatch, each worker's gradient on its stream, their
        mean on the current stream, and the same Adam step on every worker."""
        cur = torch.cuda.current_stream()
        hp0 = self.workers[0].hp
        for w in self.workers:
            w.hp.update_index = self.updates
        for e in range(hp0.epochs):
            for k in range(hp0.minibatches):
                for w, s, g, st, tv in zip(self.workers, self.streams, self.grads, self.stats,
                                           self.T_valid):
                    B.ddppo_ppo_grad(w.h, w.view, w.hp, tv, e, k, g, st, s)
                    cur.wait_stream(s)
                B.ddppo_grad_mean(self.grads, self.mean, cur)
                for w, s, st in zip(self.workers, self.streams, self.stats):
                    s.wait_stream(cur)
                    B.ddppo_apply_grad(w.h, self.mean, 1.0, w.hp, st, s)
                    cur.wait_stream(s)
        for w in self.workers:
            w.updates += 1
        self.updates += 1

    def iterate(self) -> list[int]:
        tv = self.collect()
        self.update()
        return tv

    def frames(self) -> int:
        """Frames collected by the last collection: sum over workers of T_valid x envs."""
        return sum(tv * w.E for tv, w in zip(self.T_valid, self.workers))


class DistributedWorker:
    """One DD-PPO worker per process and GPU (torch.distributed initialised, NCCL on GPUs):
    the preemption counter in `store` (a torch.distributed Store shared by all ranks, e.g.
    a TCPStore), the gradient mean by all_reduce. Parameters start equal: rank 0's are
    broadcast."""

    def __init__(self, preset: str, store, p: float = 1.0, seed: int = 0, **overrides):
        import torch.distributed as dist
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.w = Worker(preset, seed=seed + self.rank, **overrides)
        self.T = self.w.T
        self.P = B.ddppo_num_params(self.w.h)
        flat = torch.empty(self.P, device="cuda")
        B.ddppo_get_params(self.w.h, flat)
        dist.broadcast(flat, 0)
        B.ddppo_set_params(self.w.h, flat)
        self.grad = torch.zeros(self.P, device="cuda")
        self.stats = torch.zeros(B.NSTATS, device="cuda")
        self.counter = PreemptionCounter(self.world, p, self.T, store=store)
        self.T_valid = self.T

    def close(self):
        self.w.close()

    def collect(self) -> int:
        w = self.w
        self.counter.new_round()
        w.t["uniforms"].copy_(w._pool[w._k % w._pool.shape[0]], non_blocking=True)
        w._k += 1
        B.ddppo_collect_begin(w.h, w.view)
        s = torch.cuda.current_stream()
        tv = preempted_collection(lambda t: B.ddppo_collect_step(w.h, w.view, t), self.T,
                                  self.counter, wait=s.synchronize)
        B.ddppo_collect_end(w.h, w.view, tv)
        t = w.t
        B.ddppo_gae(t["rewards"], t["dones"], t["values"], tv, w.E, w.gamma, w.lam, t["adv"],
                    t["ret"])
        self.T_valid = tv
        return tv

    def update(self):
        w = self.w
        w.hp.update_index = w.updates

        def grad(e, k):
            B.ddppo_ppo_grad(w.h, w.view, w.hp, self.T_valid, e, k, self.grad, self.stats)
            return self.grad

        exchange_update(w.hp.epochs, w.hp.minibatches, grad, self.dist.all_reduce,
                        lambda g: B.ddppo_apply_grad(w.h, g, 1.0 / self.world, w.hp, self.stats))
        w.updates += 1


def timed_iterations(vw: VirtualWorkers, iters: int, warmup: int = 1) -> dict:
    """Frames per second of `iters` iterations after `warmup` (device-synchronised wall
    clock: the workers' streams overlap, so no single stream's events bracket them)."""
    for _ in range(warmup):
        vw.iterate()
    torch.cuda.synchronize()
    frames, tvs = 0, []
    t0 = time.perf_counter()
    for _ in range(iters):
        tvs.append(vw.iterate())
        frames += vw.frames()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return {"frames_per_s": frames / dt, "s_per_iter": dt / iters, "T_valid": tvs}
