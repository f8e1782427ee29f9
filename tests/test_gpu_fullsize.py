"""Parity at the benchmark's full size, in the benchmark's launch configuration.

The paper-shaped workload (64 envs, 128x128 rooms-and-doors grids at 0.1 m, 256x256
depth pooled to 128x128, ResNet-18/32 GroupNorm encoder, 2-layer LSTM 512, T = 128,
BF16 GEMMs), driven through the same Worker the benchmark times (graph-captured collect,
GAE, 2 x 2 PPO update). Checked on outputs the oracle can compute one by one:
  * the whole trajectory: the oracle world re-stepped with the collected actions gives
    bit-identical rewards and dones for every (t, env);
  * the observation of sampled frames: oracle depth, pooled and normalised;
  * the policy on sampled envs: over each env's full 128-step sequence, the stored
    log-probabilities and values are within twice the distance of a float64 emulation of
    the BF16 roundings (tests/bf16_emu.py) to the float64 oracle, plus 1e-2: the BF16
    ResNet is chaotic at fp32 noise level, so its distance to float64 is set by the bf16
    roundings themselves, which the emulation measures;
  * GAE on the stored rewards/values: float64 recursion within 1e-5 relative.
"""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from oracle import rl as OR
from oracle import sim as OS
from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker
from tests import bf16_emu as EMU
from tests.gpu_util import net_config_from, sim_config_from

pytestmark = pytest.mark.gpu


def test_full_size_sampled_parity():
    w = Worker("resnet", seed=5)
    try:
        cfg = w.cfg
        E, T = w.E, w.T
        flat = torch.zeros(B.ddppo_num_params(w.h), device="cuda")
        B.ddppo_get_params(w.h, flat)
        w.iterate()   # first iteration: collect with the initial parameters, then update
        torch.cuda.synchronize()
        t = {k: v.cpu() for k, v in w.t.items()}
        # 1. trajectory: oracle world stepped with the collected actions
        sim = OS.BatchSim(sim_config_from(cfg))
        sim.reset()
        acts = t["actions"].numpy()
        sample_frames = {0: None, 64: None, 127: None}
        for s in range(T):
            if s in sample_frames:
                sample_frames[s] = sim.render()
            r, d, _, _ = sim.step(acts[s])
            assert (t["rewards"][s].numpy().view(np.uint32) == r.view(np.uint32)).all(), s
            assert (t["dones"][s].numpy() == d).all(), s
        # 2. sampled observations (the obs of step s is the frame the policy acted on)
        for s, (depth, goal) in sample_frames.items():
            o_ref = OS.pool_obs(depth, True, 10.0)
            o = t["obs"][s, :, 0].float().numpy()
            ok = np.abs(o - o_ref) <= (2.0 ** -8) * np.abs(o_ref) + 2e-5
            assert ok.mean() >= 0.9999
            assert np.allclose(t["goal"][s].numpy(), goal, rtol=2e-6, atol=2e-5)
        # 3. the policy over whole sequences of sampled envs (parameters of this rollout)
        ncfg = net_config_from(cfg)
        p = OP.unflatten(flat.cpu().double(), ncfg)
        envs = [0, 37]
        args = (p, t["obs"][:T, envs].double(), t["goal"][:T, envs].double(), t["prev_a"][:T, envs],
                t["masks"][:T, envs], t["h0"][:, envs].double(), t["c0"][:, envs].double(), ncfg)
        act = t["actions"][:, envs].long().unsqueeze(2)
        with torch.no_grad():
            lg, v, _, _ = OP.sequence_forward(*args)
            lg_e, v_e, _, _ = EMU.sequence_forward(*args)
        lp = torch.log_softmax(lg, -1).gather(2, act)[..., 0]
        lp_e = torch.log_softmax(lg_e, -1).gather(2, act)[..., 0]
        lp_g, v_g = t["logp"][:, envs].double(), t["values"][:T, envs].double()
        scale_lp = max(1.0, lp.abs().max().item())
        scale_v = max(v.abs().max().item(), 1e-3)
        err_lp = (lp_g - lp).abs().max().item() / scale_lp
        err_v = (v_g - v).abs().max().item() / scale_v
        cost_lp = (lp_e - lp).abs().max().item() / scale_lp
        cost_v = (v_e - v).abs().max().item() / scale_v
        print("full size: logp err %.3g (bf16 emulation %.3g), value err %.3g (emulation %.3g)"
              % (err_lp, cost_lp, err_v, cost_v))
        assert err_lp <= 2 * cost_lp + 1e-2, (err_lp, cost_lp)
        assert err_v <= 2 * cost_v + 1e-2, (err_v, cost_v)
        # 4. GAE of this rollout
        A_ref, R_ref = OR.gae(t["rewards"].numpy(), t["dones"].numpy(), t["values"].numpy(), 0.99, 0.95)
        assert np.all(np.abs(t["adv"].numpy() - A_ref) <= 1e-5 * np.maximum(1.0, np.abs(A_ref)))
        # the update moved the parameters, and the device status is clean
        after = torch.zeros_like(flat)
        B.ddppo_get_params(w.h, after)
        assert (after - flat).abs().max().item() > 0
        assert torch.isfinite(after).all()
        assert B.ddppo_device_status(w.h) == 0
    finally:
        w.close()
