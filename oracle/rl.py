"""FP64 CPU oracle of the learning step of DD-PPO (Sec. 2 Eq. 1-2; Sec. 4 "Training").

TEST INFRASTRUCTURE ONLY. GAE by its backward recursion, the PPO clipped
surrogate by definition, its gradient by float64 autograd (pinned against
central finite differences in the tests), global-norm clipping and Adam by the
published update (Kingma & Ba 2015, Algorithm 1).

Loss (Eq. 2 plus the value and entropy terms the paper leaves unstated):
    L = -mean(min(rho*A, clip(rho, 1-eps, 1+eps)*A)) + c_v*0.5*mean((R - V)^2) - c_e*mean(H)
with rho = exp(logpi - logpi_old); advantages are not normalised by default
(Sec. 4 "Training"); the optional normalisation uses the mean and the
(population) standard deviation over the whole rollout with eps 1e-5 added.

Pins (independent of the formulas here; a plausible mistake fails the named test):
  gae                 direct discounted sum at lambda = 1, TD error at lambda = 0, done cuts
                      (tests/test_oracle_rl.py)
  ppo_loss            value term alone = 0.5 c_v mean((R - V)^2) with its gradient; entropy
                      ln 4 at uniform logits and the closed form at one dominant logit, with
                      its sign; the clipped surrogate, clip fraction and approximate KL on
                      hand-picked ratios (tests/test_oracle_pins_loss.py)
  minibatch_loss_and_grad  central finite differences on four nets; -A grad log pi at
                      theta_old; zero policy gradient when every sample is clipped
  clip_grad_norm      3-4-5 closed form; below-threshold identity
  adam_step           first two bias-corrected steps in closed form; a quadratic's minimum
  ppo_update          one minibatch = one clipped Adam step on the permuted envs
  dd_ppo_update       one worker = ppo_update; the mean of equal-sized workers' gradients =
                      the gradient of the loss over the union of their minibatches
                      (tests/test_oracle_pins_loss.py)
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import policy as P
from . import sim as S

DT = torch.float64


@dataclasses.dataclass
class PPOHParams:
    clip: float = 0.2
    epochs: int = 2
    minibatches: int = 2
    lr: float = 2.5e-4
    value_coef: float = 0.5
    entropy_coef: float = 0.01
    max_grad_norm: float = 0.5
    beta1: float = 0.9
    beta2: float = 0.999
    adam_eps: float = 1e-5
    gamma: float = 0.99
    lam: float = 0.95
    norm_adv: bool = False


def gae(rewards, dones, values, gamma, lam):
    """Generalised advantage estimation (Schulman et al. 2016), Sec. 4 "Training".

    rewards, dones [T, E]; values [T+1, E] (the last row bootstraps).
    delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t ;  A_t = delta_t + gamma lam (1 - d_t) A_{t+1}
    Returns (A, R = A + V[:T]) as float64 arrays.
    """
    r = np.asarray(rewards, np.float64)
    d = np.asarray(dones, np.float64)
    v = np.asarray(values, np.float64)
    T, E = r.shape
    adv = np.zeros((T, E), np.float64)
    nxt = np.zeros(E, np.float64)
    for t in range(T - 1, -1, -1):
        nd = 1.0 - d[t]
        delta = r[t] + gamma * nd * v[t + 1] - v[t]
        nxt = delta + gamma * lam * nd * nxt
        adv[t] = nxt
    return adv, adv + v[:T]


def ppo_loss(logits, values, actions, logp_old, adv, ret, hp: PPOHParams):
    """Scalar PPO loss and its statistics for one minibatch (Eq. 2)."""
    logp_all = torch.log_softmax(logits, dim=-1)
    logp = logp_all.gather(-1, actions.long().unsqueeze(-1)).squeeze(-1)
    ratio = torch.exp(logp - logp_old)
    surr1 = ratio * adv
    surr2 = torch.clamp(ratio, 1.0 - hp.clip, 1.0 + hp.clip) * adv
    pol = -torch.minimum(surr1, surr2).mean()
    vloss = 0.5 * ((ret - values) ** 2).mean()
    ent = -(logp_all.exp() * logp_all).sum(-1).mean()
    loss = pol + hp.value_coef * vloss - hp.entropy_coef * ent
    with torch.no_grad():
        clipfrac = ((ratio - 1.0).abs() > hp.clip).to(DT).mean()
        approx_kl = (logp_old - logp).mean()
    stats = {"loss": loss.detach(), "policy_loss": pol.detach(), "value_loss": vloss.detach(),
             "entropy": ent.detach(), "clip_frac": clipfrac, "approx_kl": approx_kl}
    return loss, stats


def clip_grad_norm(g: torch.Tensor, max_norm: float):
    """Scale g by min(1, max_norm / (||g||_2 + 1e-6)); returns (g', ||g||)."""
    n = torch.linalg.vector_norm(g)
    coef = torch.clamp(max_norm / (n + 1e-6), max=1.0)
    return g * coef, n


def adam_step(theta, g, m, v, t, hp: PPOHParams):
    """Adam (Kingma & Ba 2015, Alg. 1) with step count t >= 1, float64."""
    m = hp.beta1 * m + (1 - hp.beta1) * g
    v = hp.beta2 * v + (1 - hp.beta2) * g * g
    mh = m / (1 - hp.beta1 ** t)
    vh = v / (1 - hp.beta2 ** t)
    theta = theta - hp.lr * mh / (torch.sqrt(vh) + hp.adam_eps)
    return theta, m, v


def minibatch_loss_and_grad(flat, mb, ncfg, hp):
    """Loss, stats and d loss / d flat for a minibatch dict of float64 tensors."""
    flat = flat.detach().clone().requires_grad_(True)
    p = P.unflatten(flat, ncfg)
    logits, values, _, _ = P.sequence_forward(p, mb["obs"], mb["goal"], mb["prev_a"], mb["masks"],
                                              mb["h0"], mb["c0"], ncfg)
    loss, stats = ppo_loss(logits, values, mb["actions"], mb["logp_old"], mb["adv"], mb["ret"], hp)
    (g,) = torch.autograd.grad(loss, flat)
    return loss.detach(), stats, g


def ppo_update(flat, m, v, step, ro, ncfg, hp: PPOHParams, seed: int, update: int):
    """epochs x minibatches of PPO on a rollout (Sec. 4 "Training").

    ro: dict of float64/int tensors with time-major [T, E, ...] entries obs, goal,
    prev_a, masks, actions, logp_old, adv, ret, and h0/c0 [L, E, Hd].
    Minibatch k of epoch e holds the envs perm[k*E_mb:(k+1)*E_mb] with
    perm = oracle.sim.env_permutation(seed, update, e, E), full T sequences.
    Returns new (flat, m, v, step) and a list of per-minibatch stats.
    """
    E = ro["actions"].shape[1]
    Emb = E // hp.minibatches
    adv = ro["adv"]
    if hp.norm_adv:
        adv = (adv - adv.mean()) / (adv.std(unbiased=False) + 1e-5)
    all_stats = []
    for e in range(hp.epochs):
        perm = torch.from_numpy(S.env_permutation(seed, update, e, E).astype(np.int64))
        for k in range(hp.minibatches):
            idx = perm[k * Emb:(k + 1) * Emb]
            mb = {key: ro[key][:, idx] for key in ("obs", "goal", "prev_a", "masks", "actions",
                                                     "logp_old", "ret")}
            mb["adv"] = adv[:, idx]
            mb["h0"] = ro["h0"][:, idx]
            mb["c0"] = ro["c0"][:, idx]
            _, stats, g = minibatch_loss_and_grad(flat, mb, ncfg, hp)
            g, gn = clip_grad_norm(g, hp.max_grad_norm)
            stats["grad_norm"] = gn
            step += 1
            flat, m, v = adam_step(flat.detach(), g, m, v, step, hp)
            all_stats.append(stats)
    return flat, m, v, step, all_stats


def dd_ppo_update(flat, m, v, step, rollouts, ncfg, hp: PPOHParams, seeds, update: int,
                  T_valid=None):
    """DD-PPO's update across N workers (Sec. 3, Eq. 4): at every minibatch step each worker
    n computes the PPO gradient of its own minibatch (its own envs, permuted by its own
    seed), the gradients are averaged (AllReduce with the mean), and every worker applies
    the same clipped Adam step, so all parameter copies stay equal.

    rollouts: one dict per worker as for ppo_update; seeds: the workers' seeds; T_valid:
    per worker, the steps of its rollout that count (a preempted straggler's shorter
    rollout: its loss is the mean over its own samples, each worker weighing equally).
    Returns (flat, m, v, step, per-step list of per-worker stats, per-step mean gradients).
    """
    N = len(rollouts)
    Tv = [ro["actions"].shape[0] for ro in rollouts] if T_valid is None else list(T_valid)
    all_stats, grads_out = [], []
    for e in range(hp.epochs):
        perms = [torch.from_numpy(S.env_permutation(seeds[n], update, e, rollouts[n]["actions"].shape[1])
                                  .astype(np.int64)) for n in range(N)]
        for k in range(hp.minibatches):
            grads, stats = [], []
            for n, ro in enumerate(rollouts):
                E = ro["actions"].shape[1]
                Emb = E // hp.minibatches
                idx = perms[n][k * Emb:(k + 1) * Emb]
                T = Tv[n]
                adv = ro["adv"][:T]
                if hp.norm_adv:
                    adv = (adv - adv.mean()) / (adv.std(unbiased=False) + 1e-5)
                mb = {key: ro[key][:T, idx] for key in ("obs", "goal", "prev_a", "masks", "actions",
                                                        "logp_old", "ret")}
                mb["adv"] = adv[:, idx]
                mb["h0"] = ro["h0"][:, idx]
                mb["c0"] = ro["c0"][:, idx]
                _, st, g = minibatch_loss_and_grad(flat, mb, ncfg, hp)
                grads.append(g)
                stats.append(st)
            g = sum(grads) / N                 # AllReduce(mean)
            grads_out.append(g)
            g, gn = clip_grad_norm(g, hp.max_grad_norm)
            for st in stats:
                st["grad_norm"] = gn
            step += 1
            flat, m, v = adam_step(flat.detach(), g, m, v, step, hp)
            all_stats.append(stats)
    return flat, m, v, step, all_stats, grads_out
