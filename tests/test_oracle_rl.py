"""Pins of the network / learning oracle (``oracle.policy``, ``oracle.rl``).

Each check compares the oracle with something independent of it: a direct
sum instead of the GAE recursion, central finite differences instead of
autograd, the closed form of Adam's first steps, loop restatements of
convolution and GroupNorm, torch.nn.LSTM for the gate equations.
"""
import math

import numpy as np
import pytest
import torch

from oracle import policy as P
from oracle import rl as R
from tests import inputs as I

DT = torch.float64


# ---------------------------------------------------------------- GAE (Sec. 4 "Training")
def _discounted_return_minus_v(r, d, v, gamma):
    """lambda = 1: A_t = sum_{i>=t} gamma^{i-t} r_i (stopping at a done, else bootstrapping
    with gamma^{T-t} V_T) - V_t, written as a direct sum (Eq. 1)."""
    T, E = r.shape
    out = np.zeros((T, E))
    for e in range(E):
        for t in range(T):
            acc, disc = 0.0, 1.0
            i = t
            while True:
                acc += disc * r[i, e]
                if d[i, e]:
                    break
                disc *= gamma
                i += 1
                if i == T:
                    acc += disc * v[T, e]
                    break
            out[t, e] = acc - v[t, e]
    return out


def test_gae_lambda_one_is_discounted_return_minus_value():
    rng = np.random.default_rng(0)
    T, E = 17, 5
    r = rng.normal(size=(T, E))
    d = (rng.random((T, E)) < 0.15).astype(np.uint8)
    v = rng.normal(size=(T + 1, E))
    A, Rt = R.gae(r, d, v, 0.99, 1.0)
    assert np.allclose(A, _discounted_return_minus_v(r, d, v, 0.99), atol=1e-12)
    assert np.allclose(Rt, A + v[:T])


def test_gae_lambda_zero_is_td_error():
    rng = np.random.default_rng(1)
    T, E = 9, 4
    r = rng.normal(size=(T, E))
    d = (rng.random((T, E)) < 0.3).astype(np.uint8)
    v = rng.normal(size=(T + 1, E))
    A, _ = R.gae(r, d, v, 0.9, 0.0)
    td = r + 0.9 * (1 - d) * v[1:] - v[:T]
    assert np.allclose(A, td, atol=1e-14)


def test_gae_done_cuts_the_recursion():
    T, E = 6, 1
    r = np.zeros((T, E))
    r[4, 0] = 1.0
    d = np.zeros((T, E), np.uint8)
    d[2, 0] = 1
    v = np.zeros((T + 1, E))
    A, _ = R.gae(r, d, v, 0.5, 1.0)
    assert A[0, 0] == 0 and A[1, 0] == 0 and A[2, 0] == 0
    assert A[3, 0] == 0.5 and A[4, 0] == 1.0


# ---------------------------------------------------------------- network building blocks
def _conv_loops(x, w, b, s, p):
    N, C, H, W = x.shape
    O, _, kh, kw = w.shape
    Ho, Wo = (H + 2 * p - kh) // s + 1, (W + 2 * p - kw) // s + 1
    out = np.zeros((N, O, Ho, Wo))
    xn, wn = x.numpy(), w.numpy()
    for n in range(N):
        for o in range(O):
            for i in range(Ho):
                for j in range(Wo):
                    acc = 0.0 if b is None else float(b[o])
                    for c in range(C):
                        for u in range(kh):
                            for v in range(kw):
                                y, xx = i * s - p + u, j * s - p + v
                                if 0 <= y < H and 0 <= xx < W:
                                    acc += xn[n, c, y, xx] * wn[o, c, u, v]
                    out[n, o, i, j] = acc
    return out


@pytest.mark.parametrize("k,s,p", [(3, 1, 1), (3, 2, 1), (7, 2, 3), (1, 2, 0), (8, 4, 0)])
def test_conv_matches_loop_definition(k, s, p):
    g = torch.Generator().manual_seed(k * 10 + s)
    x = torch.randn(2, 3, 11, 12, generator=g, dtype=DT)
    w = torch.randn(4, 3, k, k, generator=g, dtype=DT)
    b = torch.randn(4, generator=g, dtype=DT)
    ref = _conv_loops(x, w, b, s, p)
    got = torch.nn.functional.conv2d(x, w, b, stride=s, padding=p).numpy()
    assert np.allclose(got, ref, atol=1e-10)


def test_group_norm_matches_definition():
    g = torch.Generator().manual_seed(3)
    x = torch.randn(3, 8, 5, 6, generator=g, dtype=DT)
    gam = torch.randn(8, generator=g, dtype=DT)
    bet = torch.randn(8, generator=g, dtype=DT)
    got = P._gn(x, gam, bet, 1e-5).numpy()
    xn = x.numpy()
    ref = np.zeros_like(xn)
    G = 4  # C / 2 groups of 2 channels
    for n in range(3):
        for gi in range(G):
            blk = xn[n, 2 * gi:2 * gi + 2]
            mu = blk.mean()
            var = ((blk - mu) ** 2).mean()  # biased variance
            for c in (2 * gi, 2 * gi + 1):
                ref[n, c] = (xn[n, c] - mu) / math.sqrt(var + 1e-5) * gam[c].item() + bet[c].item()
    assert np.allclose(got, ref, atol=1e-12)


def test_lstm_cell_matches_torch_lstm():
    torch.manual_seed(0)
    In, Hd, E, T = 7, 5, 3, 6
    ref = torch.nn.LSTM(In, Hd, num_layers=2, dtype=DT)
    x = torch.randn(T, E, In, dtype=DT)
    h0 = torch.randn(2, E, Hd, dtype=DT)
    c0 = torch.randn(2, E, Hd, dtype=DT)
    y_ref, (hT, cT) = ref(x, (h0, c0))
    h = [h0[0], h0[1]]
    c = [c0[0], c0[1]]
    ys = []
    for t in range(T):
        z = x[t]
        for l in range(2):
            h[l], c[l] = P.lstm_cell(z, h[l], c[l], getattr(ref, f"weight_ih_l{l}"),
                                     getattr(ref, f"weight_hh_l{l}"), getattr(ref, f"bias_ih_l{l}"),
                                     getattr(ref, f"bias_hh_l{l}"))
            z = h[l]
        ys.append(z)
    assert torch.allclose(torch.stack(ys), y_ref, atol=1e-12)
    assert torch.allclose(h[1], hT[1], atol=1e-12) and torch.allclose(c[0], cT[0], atol=1e-12)


def test_resnet_feature_shape_is_128x4x4():
    """App. "Visual Encoder": 128x128 effective input -> 128x4x4 = 2048-d."""
    cfg = I.net_config("resnet_b32")
    assert P.feature_dim(cfg) == 2048
    cfg1 = I.net_config("nature")
    assert P.feature_dim(cfg1) == 512


def test_sampling_inverse_cdf():
    probs = torch.tensor([[0.1, 0.2, 0.3, 0.4]], dtype=DT)
    lg = probs.log()
    for u, a in [(0.0, 0), (0.05, 0), (0.15, 1), (0.35, 2), (0.61, 3), (0.999999, 3)]:
        assert P.sample_action(lg, torch.tensor([u], dtype=DT)).item() == a


def test_masks_reset_recurrent_state():
    cfg = I.net_config("tiny")
    flat = I.params(cfg, seed=0)
    p = P.unflatten(flat, cfg)
    ro = I.rollout_inputs(cfg, T=3, E=2, seed=1)
    h0 = torch.randn(cfg.lstm_layers, 2, cfg.hidden, dtype=DT)
    c0 = torch.randn(cfg.lstm_layers, 2, cfg.hidden, dtype=DT)
    m = torch.zeros(3, 2, dtype=torch.uint8)
    lg1, v1, _, _ = P.sequence_forward(p, ro["obs"], ro["goal"], ro["prev_a"], m, h0, c0, cfg)
    lg2, v2, _, _ = P.sequence_forward(p, ro["obs"], ro["goal"], ro["prev_a"], m, 0 * h0, 0 * c0, cfg)
    assert torch.allclose(lg1, lg2) and torch.allclose(v1, v2)


# ---------------------------------------------------------------- PPO loss and its gradient
def _mb(cfg, T, E, seed):
    return I.minibatch(cfg, T=T, E=E, seed=seed)


@pytest.mark.parametrize("net", ["tiny", "tiny_resnet", "tiny_blind", "tiny_sx"])
def test_ppo_gradient_matches_central_differences(net):
    cfg = I.net_config(net)
    hp = R.PPOHParams()
    flat = I.params(cfg, seed=2)
    mb = _mb(cfg, T=4, E=2, seed=3)
    loss, _, g = R.minibatch_loss_and_grad(flat, mb, cfg, hp)
    rng = np.random.default_rng(4)
    idx = rng.choice(flat.numel(), 40, replace=False)
    h = 1e-6
    for i in idx:
        fp = flat.clone(); fp[i] += h
        fm = flat.clone(); fm[i] -= h
        lp, _, _ = R.minibatch_loss_and_grad(fp, mb, cfg, hp)
        lm, _, _ = R.minibatch_loss_and_grad(fm, mb, cfg, hp)
        fd = (lp - lm).item() / (2 * h)
        assert abs(fd - g[i].item()) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i].item())


def test_ppo_gradient_at_old_policy_is_minus_adv_grad_logpi():
    """At theta = theta_old the ratio is 1 and d/dtheta of the surrogate term is
    -mean(A * grad log pi(a))."""
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(value_coef=0.0, entropy_coef=0.0)
    flat = I.params(cfg, seed=5)
    mb = _mb(cfg, T=3, E=2, seed=6)
    p = P.unflatten(flat, cfg)
    with torch.no_grad():
        lg, _, _, _ = P.sequence_forward(p, mb["obs"], mb["goal"], mb["prev_a"], mb["masks"],
                                         mb["h0"], mb["c0"], cfg)
        mb["logp_old"] = torch.log_softmax(lg, -1).gather(-1, mb["actions"].long().unsqueeze(-1))[..., 0]
    _, stats, g = R.minibatch_loss_and_grad(flat, mb, cfg, hp)
    assert abs(stats["clip_frac"].item()) == 0.0
    fl = flat.clone().requires_grad_(True)
    p2 = P.unflatten(fl, cfg)
    lg2, _, _, _ = P.sequence_forward(p2, mb["obs"], mb["goal"], mb["prev_a"], mb["masks"],
                                      mb["h0"], mb["c0"], cfg)
    lp = torch.log_softmax(lg2, -1).gather(-1, mb["actions"].long().unsqueeze(-1))[..., 0]
    (g_ref,) = torch.autograd.grad(-(mb["adv"] * lp).mean(), fl)
    assert torch.allclose(g, g_ref, atol=1e-13, rtol=1e-10)


def test_clipped_samples_have_no_policy_gradient():
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(value_coef=0.0, entropy_coef=0.0)
    flat = I.params(cfg, seed=7)
    mb = _mb(cfg, T=2, E=2, seed=8)
    # ratio = e^{1} > 1.2 with A > 0: min picks the clipped (constant) term everywhere
    p = P.unflatten(flat, cfg)
    with torch.no_grad():
        lg, _, _, _ = P.sequence_forward(p, mb["obs"], mb["goal"], mb["prev_a"], mb["masks"],
                                         mb["h0"], mb["c0"], cfg)
        lp = torch.log_softmax(lg, -1).gather(-1, mb["actions"].long().unsqueeze(-1))[..., 0]
    mb["logp_old"] = lp - 1.0
    mb["adv"] = mb["adv"].abs() + 0.1
    loss, stats, g = R.minibatch_loss_and_grad(flat, mb, cfg, hp)
    assert stats["clip_frac"].item() == 1.0
    assert torch.count_nonzero(g).item() == 0
    assert abs(loss.item() + 1.2 * mb["adv"].mean().item()) < 1e-12


# ---------------------------------------------------------------- Adam and clipping
def test_adam_first_steps_closed_form():
    """Kingma & Ba 2015: the first bias-corrected step is -lr * g / (|g| + eps)."""
    hp = R.PPOHParams(lr=0.1)
    th = torch.tensor([1.0, -2.0, 0.5], dtype=DT)
    g1 = torch.tensor([0.3, -4.0, 0.0], dtype=DT)
    m = torch.zeros(3, dtype=DT)
    v = torch.zeros(3, dtype=DT)
    th1, m, v = R.adam_step(th, g1, m, v, 1, hp)
    assert torch.allclose(th1, th - 0.1 * g1 / (g1.abs() + 1e-5), atol=1e-15)
    # second step with g2: m = 0.9*0.1*g1 + 0.1*g2 ... closed form with bias corrections
    g2 = torch.tensor([0.1, 1.0, 2.0], dtype=DT)
    th2, _, _ = R.adam_step(th1, g2, m, v, 2, hp)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert torch.allclose(th2, th1 - 0.1 * mh / (vh.sqrt() + 1e-5), atol=1e-14)


def test_adam_minimises_a_quadratic():
    hp = R.PPOHParams(lr=0.05)
    th = torch.tensor([3.0, -1.0], dtype=DT)
    m = torch.zeros(2, dtype=DT)
    v = torch.zeros(2, dtype=DT)
    for t in range(1, 2001):
        th, m, v = R.adam_step(th, 2 * (th - torch.tensor([0.5, 0.25], dtype=DT)), m, v, t, hp)
    assert torch.allclose(th, torch.tensor([0.5, 0.25], dtype=DT), atol=1e-3)


def test_grad_norm_clip():
    g = torch.tensor([3.0, 4.0], dtype=DT)
    g2, n = R.clip_grad_norm(g, 0.5)
    assert n.item() == 5.0 and abs(torch.linalg.vector_norm(g2).item() - 0.5) < 1e-6
    g3, _ = R.clip_grad_norm(torch.tensor([0.1, 0.0], dtype=DT), 0.5)
    assert g3[0].item() == 0.1


def test_ppo_update_single_minibatch_is_one_clipped_adam_step():
    cfg = I.net_config("tiny")
    hp = R.PPOHParams(epochs=1, minibatches=1)
    flat = I.params(cfg, seed=9)
    ro = I.minibatch(cfg, T=3, E=2, seed=10)
    ro["logp_old"] = ro["logp_old"]
    m = torch.zeros_like(flat)
    v = torch.zeros_like(flat)
    f2, m2, v2, step, stats = R.ppo_update(flat, m, v, 0, ro, cfg, hp, seed=0, update=0)
    perm = torch.from_numpy(np.asarray(__import__("oracle.sim", fromlist=["x"]).env_permutation(0, 0, 0, 2), np.int64))
    mb = {k: (ro[k][:, perm] if k not in ("h0", "c0") else ro[k][:, perm]) for k in ro}
    _, _, g = R.minibatch_loss_and_grad(flat, mb, cfg, hp)
    g, _ = R.clip_grad_norm(g, hp.max_grad_norm)
    f_ref, _, _ = R.adam_step(flat, g, torch.zeros_like(flat), torch.zeros_like(flat), 1, hp)
    assert step == 1 and torch.allclose(f2, f_ref, atol=1e-14)
