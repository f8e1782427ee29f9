"""The blind agent (GPS+Compass only, Sec. 5): no visual encoder and no visual FC, the
LSTM input is [goal FC, action embedding]. Parity of its forward and backward against the
float64 oracle is in test_gpu_policy.py (blind_small / blind_full); here: its act does not
read the observation, and a full collect + update iteration runs on it."""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.presets import make_config
from tests import inputs as I
from tests.gpu_util import net_config_from, obs_dtype

pytestmark = pytest.mark.gpu


def test_blind_act_ignores_the_observation():
    E = 5
    cfg = make_config("blind", num_envs=E, rollout_T=4, minibatches=1)
    h_ = B.ddppo_create(cfg)
    try:
        ncfg = net_config_from(cfg)
        B.ddppo_set_params(h_, I.params(ncfg, 7).float().cuda())
        mb = I.minibatch(ncfg, T=1, E=E, seed=8)
        oh = cfg.depth_h >> cfg.pool2x2
        outs = []
        for fill in (0.0, float("nan")):
            obs = torch.full((E, 1, oh, oh), fill, dtype=obs_dtype(cfg), device="cuda")
            h = mb["h0"].float().cuda()
            c = mb["c0"].float().cuda()
            act = torch.zeros(E, dtype=torch.int32, device="cuda")
            logp = torch.zeros(E, device="cuda")
            val = torch.zeros(E, device="cuda")
            u = torch.full((E,), 0.5, device="cuda")
            B.ddppo_policy_act(h_, obs, mb["goal"][0].float().cuda(), mb["prev_a"][0].int().cuda(),
                               mb["masks"][0].cuda(), h, c, u, act, logp, val)
            torch.cuda.synchronize()
            outs.append([t.cpu() for t in (act, logp, val, h, c)])
        for a, b in zip(*outs):
            assert torch.equal(a, b)
        assert torch.isfinite(outs[1][2]).all()
    finally:
        B.ddppo_destroy(h_)


def test_blind_worker_iteration():
    from paper_1911_00357_gb300.worker import Worker
    w = Worker("blind", seed=5, num_envs=16, rollout_T=16, minibatches=2)
    try:
        for _ in range(2):
            w.iterate()
        torch.cuda.synchronize()
        assert B.ddppo_device_status(w.h) == 0
        assert torch.isfinite(w.stats.cpu()).all()
        assert torch.isfinite(w.t["values"].cpu()).all()
    finally:
        w.close()
