"""Multi-worker aggregation of the benchmark on CPU ranks (gloo, world size 2)."""
import os

import torch.distributed as dist
import torch.multiprocessing as mp


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1911_00357_gb300.dist import aggregate
    frames = 8192.0
    ms = 1000.0 if rank == 0 else 2000.0     # rank 1 is the straggler
    v, tmax, ftot = aggregate(frames, ms)
    out[rank] = (v, tmax, ftot)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29531
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        v, tmax, ftot = out[r]
        assert tmax == 2000.0 and ftot == 16384.0
        assert abs(v - 16384.0 / 2.0) < 1e-9      # all frames over the slowest rank's time


def test_aggregate_single_process():
    from paper_1911_00357_gb300.dist import aggregate
    v, tmax, ftot = aggregate(100.0, 500.0)
    assert v == 200.0 and tmax == 500.0 and ftot == 100.0


# ---------------------------------------------------------------- DD-PPO across processes
def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _preempt_worker(rank, world, port, p, out):
    import time
    _init(rank, world, port)
    from paper_1911_00357_gb300.ddppo import PreemptionCounter, preempted_collection
    store = dist.TCPStore("127.0.0.1", port + 1, world, is_master=rank == 0)
    T = 40
    counter = PreemptionCounter(world, p, T, store=store)
    res = []
    for _ in range(2):  # two rounds: the counter keys are per round
        counter.new_round()
        dist.barrier()
        delay = 0.0 if rank == 0 else 0.01  # rank 1 simulates a slower world
        res.append(preempted_collection(lambda t: time.sleep(delay), T, counter))
        dist.barrier()
    out[rank] = res
    dist.destroy_process_group()


def _run(fn, world, *args):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=fn, args=(r, world) + args + (out,)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    return dict(out)


def test_preemption_threshold_across_two_ranks():
    """Sec. 3: with p = 50% the slow rank's collection ends once the fast one has finished
    its T = 40 steps, after at least T/4 = 10 steps; with p = 100% nobody is preempted."""
    out = _run(_preempt_worker, 2, 29541, 0.5)
    for r0, r1 in zip(out[0], out[1]):
        assert r0 == 40 and 10 <= r1 < 40
    out = _run(_preempt_worker, 2, 29545, 1.0)
    assert out[0] == [40, 40] and out[1] == [40, 40]


def _dd_worker(rank, world, port, out):
    _init(rank, world, port)
    import torch
    from oracle import rl as OR
    from oracle import sim as OS
    from paper_1911_00357_gb300.ddppo import exchange_update
    from tests import inputs as I
    cfg = I.net_config("tiny")
    hp = OR.PPOHParams(epochs=2, minibatches=2)
    flat = I.params(cfg, seed=31)
    ro = I.minibatch(cfg, T=3, E=4, seed=40 + rank)
    seed, update = 100 + rank, 1
    state = {"flat": flat, "m": torch.zeros_like(flat), "v": torch.zeros_like(flat), "step": 0}

    def grad(e, k):
        perm = torch.from_numpy(OS.env_permutation(seed, update, e, 4).astype("int64"))
        idx = perm[k * 2:(k + 1) * 2]
        mb = {key: ro[key][:, idx] for key in ro}
        _, _, g = OR.minibatch_loss_and_grad(state["flat"], mb, cfg, hp)
        return g

    def apply(g):
        g, _ = OR.clip_grad_norm(g / world, hp.max_grad_norm)
        state["step"] += 1
        state["flat"], state["m"], state["v"] = OR.adam_step(state["flat"], g, state["m"],
                                                             state["v"], state["step"], hp)

    exchange_update(hp.epochs, hp.minibatches, grad, dist.all_reduce, apply)
    out[rank] = state["flat"].numpy().tobytes()
    dist.destroy_process_group()


def test_gradient_allreduce_update_matches_the_oracle():
    """Eq. 4 over two gloo ranks: each rank's minibatch gradient, all_reduce (sum) / 2, the
    clipped Adam step; both ranks end with the parameters of oracle.rl.dd_ppo_update run in
    one process over both ranks' rollouts."""
    import numpy as np
    import torch
    from oracle import rl as OR
    from tests import inputs as I
    out = _run(_dd_worker, 2, 29551)
    cfg = I.net_config("tiny")
    hp = OR.PPOHParams(epochs=2, minibatches=2)
    flat = I.params(cfg, seed=31)
    ros = [I.minibatch(cfg, T=3, E=4, seed=40 + r) for r in range(2)]
    z = torch.zeros_like(flat)
    f, _, _, step, _, _ = OR.dd_ppo_update(flat, z, z.clone(), 0, ros, cfg, hp, [100, 101], update=1)
    assert step == 4
    got0 = np.frombuffer(out[0], np.float64)
    got1 = np.frombuffer(out[1], np.float64)
    assert (got0 == got1).all()
    assert np.allclose(got0, f.numpy(), rtol=1e-12, atol=1e-14)
