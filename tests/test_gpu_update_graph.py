"""The PPO update replays as one CUDA graph after its first (uncaptured) run. The captured
and the directly launched update run the same kernels in the same order, so three
rollout-then-update iterations give bit-identical parameters, Adam moments, statistics
and rollouts; a changed hyper-parameter re-captures. GEMM timing recorded inside the
graph reports one record per contraction launch."""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker

pytestmark = pytest.mark.gpu

SMALL = dict(num_envs=8, rollout_T=8, minibatches=2)


def _state(w):
    P = B.ddppo_num_params(w.h)
    p = torch.zeros(P, device="cuda")
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    B.ddppo_get_params(w.h, p)
    step = B.ddppo_get_adam(w.h, m, v)
    torch.cuda.synchronize()
    return p.cpu(), m.cpu(), v.cpu(), step


def test_captured_update_matches_direct_launches():
    wa = Worker("resnet", seed=7, **SMALL)
    wb = Worker("resnet", seed=7, **SMALL)
    try:
        for w in (wa, wb):
            B.ddppo_autotune(w.h, False)   # same contraction configurations on both
        B.ddppo_update_graph(wb.h, False)  # wb launches every update directly
        for it in range(3):
            wa.iterate()
            wb.iterate()
            torch.cuda.synchronize()
            assert torch.equal(wa.stats.cpu(), wb.stats.cpu()), it
            assert torch.equal(wa.t["actions"].cpu(), wb.t["actions"].cpu()), it
        pa, ma, va, sa = _state(wa)
        pb, mb, vb, sb = _state(wb)
        assert sa == sb == 3 * 2 * 2
        assert torch.equal(pa, pb) and torch.equal(ma, mb) and torch.equal(va, vb)
        # a different learning rate is a different graph: it must take effect
        before = pa.clone()
        wa.hp.lr = 0.0
        wa.iterate()
        after, _, _, _ = _state(wa)
        assert torch.equal(before, after)       # lr = 0: Adam leaves the parameters unchanged
        # per-launch timing inside the captured update: same launch count as the direct path
        for w in (wa, wb):
            B.ddppo_timing_enable(w.h, True)
            w.iterate()
            torch.cuda.synchronize()
        na = B.ddppo_timing_read(wa.h, 0)
        nb = B.ddppo_timing_read(wb.h, 0)
        assert na[1] == nb[1] > 0 and na[0] > 0
        ms_a, _, _ = B.ddppo_timing_launches(wa.h, 0)
        assert len(ms_a) == nb[1] and min(ms_a) > 0
        for w in (wa, wb):
            B.ddppo_timing_enable(w.h, False)
        assert B.ddppo_device_status(wa.h) == 0 and B.ddppo_device_status(wb.h) == 0
    finally:
        wa.close()
        wb.close()
