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
