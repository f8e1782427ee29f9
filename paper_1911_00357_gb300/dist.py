"""Whole-job aggregation of a multi-worker benchmark (one worker process per GPU).

Workers run independent replicas (no data-path collective): the job's time is the
slowest worker's and its throughput is all frames over that time.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def aggregate(frames_local: float, ms_local: float, device=None) -> tuple[float, float, float]:
    """Returns (frames per second of the whole job, max ms over ranks, total frames)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return frames_local / (ms_local / 1e3), ms_local, frames_local
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    f = torch.tensor([frames_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    return f.item() / (t.item() / 1e3), t.item(), f.item()
