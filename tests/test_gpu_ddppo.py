"""DD-PPO's worker pieces on the GPU (Sec. 3, Eq. 4): step-wise collection with the
preemption threshold, per-minibatch gradients exchanged between workers, the shared
optimizer step.

  * begin + T collect_steps + end produce exactly ddppo_collect's rollout (two
    iterations: the second starts from the carried slot);
  * ppo_grad + apply_grad (scale 1) for every epoch and minibatch produce exactly
    ddppo_ppo_update's parameters;
  * two virtual workers sharing the GPU (own envs, seeds, streams): their mean-gradient
    update of seeded synthetic rollouts matches oracle.rl.dd_ppo_update (FP32 form,
    within the update tolerance of the single-worker parity test), and both parameter
    copies stay bit-identical;
  * preemption on a heterogeneous mix (two workers on 32x32 worlds, two on 256x256): every
    T_valid is at least T/4, at least ceil(p N) workers finished all T steps, the
    trajectories of the preempted workers continue correctly into the next iteration
    (the oracle world re-stepped with the collected actions gives the same rewards and
    dones across both iterations), and the parameter copies stay equal.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rl as OR
from oracle import sim as OS
from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.ddppo import VirtualWorkers, min_steps
from paper_1911_00357_gb300.worker import Worker
from tests import inputs as I
from tests.gpu_util import net_config_from, sim_config_from

pytestmark = pytest.mark.gpu
SMALL = dict(num_envs=4, rollout_T=6, minibatches=2, hidden=16, lstm_layers=2, max_steps=9)


def _params(h):
    p = torch.empty(B.ddppo_num_params(h), device="cuda")
    B.ddppo_get_params(h, p)
    torch.cuda.synchronize()
    return p.cpu()


@pytest.mark.parametrize("preset", ["nature_fp32", "resnet"])
def test_stepwise_collection_equals_collect(preset):
    kw = dict(SMALL, precision=1) if preset == "resnet" else dict(SMALL)
    if preset == "resnet":
        kw.update(base_ch=8, depth_h=128, depth_w=128, pool2x2=0)
    a = Worker(preset, seed=4, **kw)
    b = Worker(preset, seed=4, **kw)
    try:
        B.ddppo_autotune(a.h, False)
        B.ddppo_autotune(b.h, False)
        for it in range(2):
            u = a._pool[it]
            a.t["uniforms"].copy_(u)
            b.t["uniforms"].copy_(u)
            B.ddppo_collect(a.h, a.view, True)
            B.ddppo_collect_begin(b.h, b.view)
            for t in range(b.T):
                B.ddppo_collect_step(b.h, b.view, t)
            B.ddppo_collect_end(b.h, b.view, b.T)
            torch.cuda.synchronize()
            for k in ("obs", "goal", "prev_a", "masks", "actions", "logp", "values", "rewards",
                      "dones", "h0", "c0", "h", "c"):
                assert torch.equal(a.t[k].cpu().view(torch.uint8), b.t[k].cpu().view(torch.uint8)), (it, k)
        with pytest.raises(B.DDPPOError):
            B.ddppo_collect_step(b.h, b.view, 3)  # not begun
    finally:
        a.close()
        b.close()


def test_grad_and_apply_equal_the_update():
    a = Worker("nature_fp32", seed=6, **SMALL)
    b = Worker("nature_fp32", seed=6, **SMALL)
    try:
        for w in (a, b):
            B.ddppo_update_graph(w.h, False)
        a.iterate()  # a rollout and one update
        for k in ("obs", "goal", "prev_a", "masks", "actions", "logp", "values", "adv", "ret",
                  "h0", "c0"):
            b.t[k].copy_(a.t[k])
        p = torch.empty(B.ddppo_num_params(a.h), device="cuda")
        B.ddppo_get_params(a.h, p)
        B.ddppo_set_params(b.h, p)
        # Adam moments differ (set_params clears them): start both from a fresh state
        B.ddppo_set_params(a.h, p)
        hp = a.hp
        hp.update_index = 5
        B.ddppo_ppo_update(a.h, a.view, hp, a.stats)
        g = torch.empty_like(p)
        for e in range(hp.epochs):
            for k in range(hp.minibatches):
                B.ddppo_ppo_grad(b.h, b.view, hp, b.T, e, k, g)
                B.ddppo_apply_grad(b.h, g, 1.0, hp)
        assert torch.equal(_params(a.h), _params(b.h))
        m1, m2 = torch.empty_like(p), torch.empty_like(p)
        assert B.ddppo_get_adam(a.h, m1, None) == B.ddppo_get_adam(b.h, m2, None)
        assert torch.equal(m1, m2)
    finally:
        a.close()
        b.close()


def test_two_virtual_workers_match_the_oracle_dd_update():
    T, E = 5, 4
    vw = VirtualWorkers("nature_fp32", 2, seed=8, num_envs=E, rollout_T=T, minibatches=2,
                        hidden=16, lstm_layers=2)
    try:
        ncfg = net_config_from(vw.workers[0].cfg)
        f0 = _params(vw.workers[0].h).double()
        ros = []
        for r, w in enumerate(vw.workers):
            mb = I.minibatch(ncfg, T=T, E=E, seed=60 + r)
            t = w.t
            t["obs"][:T].copy_(mb["obs"].float())
            t["goal"][:T].copy_(mb["goal"].float())
            t["prev_a"][:T].copy_(mb["prev_a"].int())
            t["masks"][:T].copy_(mb["masks"])
            t["actions"].copy_(mb["actions"].int())
            t["logp"].copy_(mb["logp_old"].float())
            t["adv"].copy_(mb["adv"].float())
            t["ret"].copy_(mb["ret"].float())
            t["h0"].copy_(mb["h0"].float())
            t["c0"].copy_(mb["c0"].float())
            ros.append({"obs": t["obs"][:T].cpu().double(), "goal": t["goal"][:T].cpu().double(),
                        "prev_a": mb["prev_a"], "masks": mb["masks"], "actions": mb["actions"],
                        "logp_old": t["logp"].cpu().double(), "adv": t["adv"].cpu().double(),
                        "ret": t["ret"].cpu().double(), "h0": t["h0"].cpu().double(),
                        "c0": t["c0"].cpu().double()})
        vw.T_valid = [T, T]
        vw.updates = 2
        vw.update()
        p0, p1 = _params(vw.workers[0].h), _params(vw.workers[1].h)
        assert torch.equal(p0, p1)
        hp = OR.PPOHParams(minibatches=2)
        z = torch.zeros_like(f0)
        seeds = [w.cfg.seed for w in vw.workers]
        f, _, _, step, _, _ = OR.dd_ppo_update(f0, z, z.clone(), 0, ros, ncfg, hp, seeds, update=2)
        err = (p0.double() - f).abs().max().item()
        assert err <= 0.02 * hp.lr * step, err
        assert all(B.ddppo_device_status(w.h) == 0 for w in vw.workers)
    finally:
        vw.close()


def test_preemption_on_a_heterogeneous_mix():
    T, p = 16, 0.5
    vw = VirtualWorkers("nature_fp32", 4, p=p, seed=12, grid_sides=[32, 32, 256, 256],
                        num_envs=8, rollout_T=T, minibatches=2, hidden=16, lstm_layers=1,
                        max_steps=40)
    try:
        sims = []
        for w in vw.workers:
            s = OS.BatchSim(sim_config_from(w.cfg))
            s.reset()
            sims.append(s)
        for it in range(2):
            tv = vw.iterate()
            torch.cuda.synchronize()
            assert all(min_steps(T) <= v <= T for v in tv), tv
            assert sum(v == T for v in tv) >= math.ceil(p * 4), tv
            for w, s, v in zip(vw.workers, sims, tv):
                acts = w.t["actions"][:v].cpu().numpy()
                for t in range(v):
                    r, d, _, _ = s.step(acts[t])
                    assert (w.t["rewards"][t].cpu().numpy().view(np.uint32) == r.view(np.uint32)).all()
                    assert (w.t["dones"][t].cpu().numpy() == d).all()
            assert vw.frames() == sum(v * 8 for v in tv)
        ps = [_params(w.h) for w in vw.workers]
        assert all(torch.equal(ps[0], q) for q in ps[1:])
        assert all(B.ddppo_device_status(w.h) == 0 for w in vw.workers)
    finally:
        vw.close()
