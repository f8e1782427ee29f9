"""Launch overlap changes when a kernel's blocks become resident, never what they compute:
each kernel waits for its predecessor's completion before it touches global memory. Three
rollout-then-update iterations (captured collect and update graphs, plus the uncaptured
first act and update) with the overlap on and off give bit-identical parameters, Adam
moments, statistics and rollouts."""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker

pytestmark = pytest.mark.gpu

SMALL = dict(num_envs=8, rollout_T=8, minibatches=2)


def _run(preset, on, precision=None):
    B.ddppo_set_launch_overlap(on)
    kw = dict(SMALL)
    if precision is not None:
        kw["precision"] = precision
    w = Worker(preset, seed=11, **kw)
    try:
        B.ddppo_autotune(w.h, False)  # the same contraction configurations in both runs
        rec = []
        for _ in range(3):
            w.iterate()
            torch.cuda.synchronize()
            rec.append((w.stats.cpu().clone(), w.t["actions"].cpu().clone(), w.t["rewards"].cpu().clone()))
        P = B.ddppo_num_params(w.h)
        p = torch.zeros(P, device="cuda")
        m = torch.zeros(P, device="cuda")
        v = torch.zeros(P, device="cuda")
        B.ddppo_get_params(w.h, p)
        B.ddppo_get_adam(w.h, m, v)
        torch.cuda.synchronize()
        assert B.ddppo_device_status(w.h) == 0
        return rec, p.cpu(), m.cpu(), v.cpu()
    finally:
        w.close()


@pytest.mark.parametrize("preset,precision", [("resnet", None), ("resnet", 0), ("nature_fp32", None), ("blind", None)])
def test_overlap_on_and_off_are_bit_identical(preset, precision):
    before = B.ddppo_launch_overlap()
    try:
        ra, pa, ma, va = _run(preset, True, precision)
        rb, pb, mb, vb = _run(preset, False, precision)
    finally:
        B.ddppo_set_launch_overlap(before)
    for it, (a, b) in enumerate(zip(ra, rb)):
        for x, y in zip(a, b):
            assert torch.equal(x, y), it
    assert torch.equal(pa, pb) and torch.equal(ma, mb) and torch.equal(va, vb)
