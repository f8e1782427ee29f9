"""Closed-form pins of the PPO loss terms, its statistics and the observation pool.

Each case builds inputs whose loss terms, statistics or pooled values are known by
hand, independent of the oracle's formulas:
  - the value term alone (Sec. 4 "Training" leaves c_v and the 0.5 factor open; the
    reading is 0.5 c_v mean((R - V)^2)),
  - the entropy bonus at uniform logits (ln 4) and at one dominant logit (-> 0), with
    its sign in the loss (-c_e H),
  - the clipped surrogate of Eq. 2, the clip fraction and the approximate KL on
    hand-picked probability ratios,
  - the 2x2 average pool of App. "Visual Encoder" and the 1 / max_depth scaling.
A dropped 0.5, a flipped entropy sign, a clip test on rho instead of |rho - 1|, a KL of
the wrong sign or a pool over the wrong axes fails one of them.
"""
import math

import numpy as np
import pytest
import torch

from oracle import rl as R
from oracle import sim as S

DT = torch.float64


def _uniform_case(n, V, Rt, clip=0.2, cv=0.5, ce=0.01):
    """n samples at uniform logits with logp_old = log 1/4 (rho = 1) and A = 0."""
    logits = torch.zeros(n, 4, dtype=DT)
    values = torch.full((n,), V, dtype=DT)
    actions = torch.arange(n, dtype=torch.int32) % 4
    logp_old = torch.full((n,), math.log(0.25), dtype=DT)
    adv = torch.zeros(n, dtype=DT)
    ret = torch.full((n,), Rt, dtype=DT)
    hp = R.PPOHParams(clip=clip, value_coef=cv, entropy_coef=ce)
    return logits, values, actions, logp_old, adv, ret, hp


def test_value_term_alone_is_half_mean_squared_error():
    """V = 0, R = 2, c_e = 0, rho = 1, A = 0: L = c_v * 0.5 * 4."""
    lg, v, a, lo, A, Rt, hp = _uniform_case(6, 0.0, 2.0, cv=0.5, ce=0.0)
    v = v.clone().requires_grad_(True)
    loss, st = R.ppo_loss(lg, v, a, lo, A, Rt, hp)
    assert st["value_loss"].item() == 2.0
    assert st["policy_loss"].item() == 0.0
    assert loss.item() == 0.5 * 2.0
    (g,) = torch.autograd.grad(loss, v)
    # d/dV_i of c_v 0.5 mean((R - V)^2) = -c_v (R - V_i) / n
    assert torch.allclose(g, torch.full((6,), -0.5 * 2.0 / 6, dtype=DT), atol=1e-15)


def test_value_term_scales_with_coefficient_and_mixed_errors():
    lg, v, a, lo, A, Rt, hp = _uniform_case(4, 0.0, 0.0, cv=0.25, ce=0.0)
    v = torch.tensor([1.0, -1.0, 3.0, 0.0], dtype=DT)
    Rt = torch.tensor([0.0, 1.0, 0.0, 0.0], dtype=DT)
    loss, st = R.ppo_loss(lg, v, a, lo, A, Rt, hp)
    # squared errors 1, 4, 9, 0 -> mean 3.5 -> 0.5 * 3.5 = 1.75
    assert st["value_loss"].item() == 1.75
    assert abs(loss.item() - 0.25 * 1.75) < 1e-15


def test_entropy_at_uniform_logits_is_ln4_with_negative_sign_in_loss():
    lg, v, a, lo, A, Rt, hp = _uniform_case(5, 1.0, 1.0, cv=0.5, ce=0.01)
    loss, st = R.ppo_loss(lg, v, a, lo, A, Rt, hp)
    assert abs(st["entropy"].item() - math.log(4.0)) < 1e-15
    assert abs(loss.item() - (-0.01 * math.log(4.0))) < 1e-15


@pytest.mark.parametrize("L", [1.0, 5.0, 30.0])
def test_entropy_with_one_dominant_logit(L):
    """logits (L, 0, 0, 0): p0 = e^L / (e^L + 3), p = 1 / (e^L + 3);
    H = -p0 ln p0 - 3 p ln p, which tends to 0 as L grows."""
    n = 3
    logits = torch.tensor([[L, 0.0, 0.0, 0.0]] * n, dtype=DT)
    actions = torch.zeros(n, dtype=torch.int32)
    p0 = math.exp(L) / (math.exp(L) + 3.0)
    p = 1.0 / (math.exp(L) + 3.0)
    H = -p0 * math.log(p0) - 3.0 * p * math.log(p)
    hp = R.PPOHParams(value_coef=0.0, entropy_coef=1.0)
    lp0 = torch.full((n,), math.log(p0), dtype=DT)
    loss, st = R.ppo_loss(logits, torch.zeros(n, dtype=DT), actions, lp0, torch.zeros(n, dtype=DT),
                          torch.zeros(n, dtype=DT), hp)
    assert abs(st["entropy"].item() - H) < 1e-13
    assert abs(loss.item() + H) < 1e-13
    if L >= 30.0:
        assert st["entropy"].item() < 1e-10


# rho, A, and whether |rho - 1| > 0.2
RATIOS = [(0.5, 1.0), (0.9, -2.0), (1.0, 0.5), (1.1, 3.0), (1.25, 1.0), (2.0, -1.0), (0.75, -1.5)]


def _ratio_case(clip=0.2):
    n = len(RATIOS)
    logits = torch.zeros(n, 4, dtype=DT)  # log pi(a) = log 1/4 for every action
    actions = torch.tensor([i % 4 for i in range(n)], dtype=torch.int32)
    rho = torch.tensor([r for r, _ in RATIOS], dtype=DT)
    adv = torch.tensor([a for _, a in RATIOS], dtype=DT)
    logp_old = math.log(0.25) - torch.log(rho)
    hp = R.PPOHParams(clip=clip, value_coef=0.0, entropy_coef=0.0)
    return logits, actions, logp_old, adv, rho, hp


def test_clip_fraction_and_approx_kl_on_hand_ratios():
    logits, actions, lo, adv, rho, hp = _ratio_case()
    n = len(RATIOS)
    _, st = R.ppo_loss(logits, torch.zeros(n, dtype=DT), actions, lo, adv, torch.zeros(n, dtype=DT), hp)
    # |rho - 1| > 0.2 for 0.5, 1.25, 2.0, 0.75 (0.75 is 0.25 away): 4 of 7
    assert st["clip_frac"].item() == 4.0 / 7.0
    # approx KL = mean(logp_old - logp) = mean(-ln rho)
    kl = -sum(math.log(r) for r, _ in RATIOS) / n
    assert abs(st["approx_kl"].item() - kl) < 1e-15


def test_clipped_surrogate_on_hand_ratios():
    """Eq. 2 sample by sample: min(rho A, clip(rho, 0.8, 1.2) A)."""
    logits, actions, lo, adv, rho, hp = _ratio_case()
    terms = {
        (0.5, 1.0): min(0.5, 0.8),      # 0.5
        (0.9, -2.0): min(-1.8, -1.8),   # inside the band
        (1.0, 0.5): 0.5,
        (1.1, 3.0): min(3.3, 3.3),
        (1.25, 1.0): min(1.25, 1.2),    # 1.2: clipped from above, A > 0
        (2.0, -1.0): min(-2.0, -1.2),   # -2.0: unclipped is smaller, A < 0
        (0.75, -1.5): min(-1.125, -1.2),  # -1.2: clipped from below, A < 0
    }
    want = -sum(terms[k] for k in RATIOS) / len(RATIOS)
    n = len(RATIOS)
    loss, st = R.ppo_loss(logits, torch.zeros(n, dtype=DT), actions, lo, adv, torch.zeros(n, dtype=DT), hp)
    assert abs(st["policy_loss"].item() - want) < 1e-14
    assert abs(loss.item() - want) < 1e-14


def test_loss_is_the_sum_of_its_three_terms():
    logits, actions, lo, adv, rho, _ = _ratio_case()
    n = len(RATIOS)
    hp = R.PPOHParams(clip=0.2, value_coef=0.5, entropy_coef=0.01)
    values = torch.linspace(-1, 1, n, dtype=DT)
    ret = torch.zeros(n, dtype=DT)
    loss, st = R.ppo_loss(logits, values, actions, lo, adv, ret, hp)
    vl = 0.5 * float((values ** 2).mean())
    assert abs(st["value_loss"].item() - vl) < 1e-15
    assert abs(loss.item() - (st["policy_loss"].item() + 0.5 * vl - 0.01 * math.log(4.0))) < 1e-14


# ---------------------------------------------------------------- observation pool
def test_pool_obs_constant_image():
    d = np.full((2, 8, 6), 3.5)
    o = S.pool_obs(d, True, 10.0)
    assert o.shape == (2, 4, 3) and (o == 0.35).all()
    o = S.pool_obs(d, False, 10.0)
    assert o.shape == (2, 8, 6) and (o == 0.35).all()


def test_pool_obs_checkerboard_averages_to_midpoint():
    """A 1-pixel checkerboard of a and b: every 2x2 window holds two of each."""
    H, W = 6, 10
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = np.where((ii + jj) % 2 == 0, 1.0, 7.0)
    o = S.pool_obs(d, True, 2.0)
    assert o.shape == (3, 5) and np.all(o == 2.0)


def test_pool_obs_ramp_on_a_non_square_image():
    """d[i, j] = 100 i + j on a 4x6 image: the window at (p, q) holds rows 2p, 2p+1 and
    columns 2q, 2q+1, so its mean is 100 (2p + 0.5) + 2q + 0.5 (a transposed or
    mis-strided window gives other values)."""
    H, W = 4, 6
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    d = 100.0 * ii + jj
    o = S.pool_obs(d, True, 5.0)
    assert o.shape == (2, 3)
    for p in range(2):
        for q in range(3):
            assert o[p, q] == (100.0 * (2 * p + 0.5) + 2 * q + 0.5) / 5.0


def test_pool_obs_odd_valued_pixels_are_not_truncated():
    d = np.array([[1.0, 2.0], [4.0, 8.0]])
    o = S.pool_obs(d, True, 1.0)
    assert o.shape == (1, 1) and o[0, 0] == 3.75


# ---------------------------------------------------------------- minibatch permutation
def test_env_permutation_is_uniform_over_small_permutations():
    """Fisher-Yates with unbiased draws gives each of the 3! orders probability 1/6; the
    classic off-by-one (Sattolo's cycle, or swapping with any index) does not."""
    counts = {}
    n = 3000
    for u in range(n):
        key = tuple(int(x) for x in S.env_permutation(11, u, 0, 3))
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 6
    chi2 = sum((c - n / 6) ** 2 / (n / 6) for c in counts.values())
    assert chi2 < 20.5  # 5 degrees of freedom, p ~ 0.001


# ---------------------------------------------------------------- LSTM input layout
def test_policy_inputs_concatenate_visual_goal_action_in_that_order():
    """The header's flat layout gives layer 0 the input [visual FC (H) | goal FC (32) |
    action embedding (32)]. With the visual FC bias at 3, the goal FC bias at 1 and the
    embedding rows at 2 (all weights 0), the input is 3s, then 1s, then 2s."""
    from oracle import policy as P
    from tests import inputs as I
    cfg = I.net_config("tiny")
    p = P.unflatten(torch.zeros(P.num_params(cfg), dtype=DT), cfg)
    p["vis.b"] += 3.0
    p["goal.b"] += 1.0
    p["act.emb"] += 2.0
    obs = torch.rand(2, 1, cfg.in_h, cfg.in_w, dtype=DT)
    goal = torch.rand(2, 3, dtype=DT)
    x = P.policy_inputs(p, obs, goal, torch.tensor([0, 4]), cfg)
    H = cfg.hidden
    assert x.shape == (2, H + 64)
    assert (x[:, :H] == 3).all() and (x[:, H:H + 32] == 1).all() and (x[:, H + 32:] == 2).all()


# ---------------------------------------------------------------- DD-PPO's gradient AllReduce
def _rollout(cfg, T, E, seed):
    from tests import inputs as I
    return I.minibatch(cfg, T=T, E=E, seed=seed)


def test_dd_update_with_one_worker_is_ppo_update():
    from tests import inputs as I
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(epochs=2, minibatches=2)
    flat = I.params(cfg, seed=21)
    ro = _rollout(cfg, 3, 4, 22)
    z = torch.zeros_like(flat)
    f1, m1, v1, s1, _ = R.ppo_update(flat, z, z.clone(), 0, ro, cfg, hp, seed=5, update=2)
    f2, m2, v2, s2, _, _ = R.dd_ppo_update(flat, z, z.clone(), 0, [ro], cfg, hp, [5], update=2)
    assert s1 == s2 == 4
    assert torch.equal(f1, f2) and torch.equal(m1, m2) and torch.equal(v1, v2)


def test_dd_mean_gradient_is_the_gradient_of_the_union_minibatch():
    """Eq. 4 with equal minibatch sizes: the mean of the workers' mean losses is the mean
    loss over the union of their samples, so the averaged gradient equals the gradient of
    one minibatch holding both workers' sequences (a second restatement, through
    minibatch_loss_and_grad on concatenated inputs, not through the averaging code)."""
    from tests import inputs as I
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(epochs=1, minibatches=1)
    flat = I.params(cfg, seed=23)
    ros = [_rollout(cfg, 3, 2, 24), _rollout(cfg, 3, 2, 25)]
    z = torch.zeros_like(flat)
    _, _, _, _, _, grads = R.dd_ppo_update(flat, z, z.clone(), 0, ros, cfg, hp, [7, 8], update=0)
    union = {}
    for key in ("obs", "goal", "prev_a", "masks", "actions", "logp_old", "adv", "ret"):
        union[key] = torch.cat([ros[0][key], ros[1][key]], dim=1)
    for key in ("h0", "c0"):
        union[key] = torch.cat([ros[0][key], ros[1][key]], dim=1)
    _, _, g_union = R.minibatch_loss_and_grad(flat, union, cfg, hp)
    # one minibatch per epoch: every env of each worker, in any order (the loss is a mean)
    assert torch.allclose(grads[0], g_union, rtol=1e-10, atol=1e-13)


def test_dd_short_rollout_weighs_its_worker_equally():
    """A preempted worker (T_valid < T) contributes the mean over its own samples with the
    same weight 1/N as a full one (Sec. 3): the averaged gradient is the plain mean of the
    two workers' gradients, each over its own steps."""
    from tests import inputs as I
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(epochs=1, minibatches=1)
    flat = I.params(cfg, seed=26)
    ros = [_rollout(cfg, 4, 2, 27), _rollout(cfg, 4, 2, 28)]
    z = torch.zeros_like(flat)
    _, _, _, _, _, grads = R.dd_ppo_update(flat, z, z.clone(), 0, ros, cfg, hp, [1, 2], update=0,
                                           T_valid=[4, 2])
    mb1 = {k: ros[1][k][:2] for k in ("obs", "goal", "prev_a", "masks", "actions", "logp_old", "adv", "ret")}
    mb1["h0"], mb1["c0"] = ros[1]["h0"], ros[1]["c0"]
    _, _, g0 = R.minibatch_loss_and_grad(flat, ros[0], cfg, hp)
    _, _, g1 = R.minibatch_loss_and_grad(flat, mb1, cfg, hp)
    assert torch.allclose(grads[0], 0.5 * (g0 + g1), rtol=1e-10, atol=1e-13)
