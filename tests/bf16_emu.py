"""Float64 emulation of the BF16 form of the agent network, for the GPU parity tests.

The BF16 form (precision 1) rounds values to bfloat16 at fixed places and computes
everything else in fp32:
  - every contraction reads bf16 operands: the layer input (the bf16 copy the GroupNorm /
    max-pool / LSTM kernels write, or the cast encoder features) and the weight, and
    accumulates in fp32;
  - in the backward, the gradient with respect to a contraction's output is stored in
    bf16 before the two contractions that consume it (input and weight gradients); the
    bias / GroupNorm-affine gradients read the fp32 value;
  - the LSTM input pieces written by the visual FC, the goal FC and the action embedding
    are stored in bf16, and so is the masked recurrent state h * m entering each step
    and the layer output feeding the next layer; cell states, gates, heads and the loss
    stay fp32.
This module restates the oracle's network (``oracle.policy``, same parameter names and
layout) in float64 with exactly those roundings: operands rounded in the forward and the
output gradient rounded in the backward, by custom autograd functions. What remains
between it and the GPU is fp32 arithmetic and the rare ReLU / max-pool decision that it
flips. With rounding switched off it is the oracle's network (a CPU test checks that),
so it shares the oracle's definition and adds only the rounding points above.
"""
from __future__ import annotations

import contextlib

import torch
import torch.nn.functional as F

from oracle import policy as OP

DT = torch.float64
_ON = [True]


@contextlib.contextmanager
def rounding(on: bool):
    """Switch the bf16 rounding points on or off (off: the plain float64 network)."""
    old = _ON[0]
    _ON[0] = on
    try:
        yield
    finally:
        _ON[0] = old


def R(x: torch.Tensor) -> torch.Tensor:
    """bfloat16 value of x (round to nearest even), back in float64."""
    if not _ON[0]:
        return x
    return x.to(torch.float32).to(torch.bfloat16).to(DT)


class _Store(torch.autograd.Function):
    """A value stored in bf16; its gradient passes unchanged (the backward reads fp32)."""

    @staticmethod
    def forward(ctx, x):
        return R(x)

    @staticmethod
    def backward(ctx, g):
        return g


class _Linear(torch.autograd.Function):
    """y = R(A) R(W)^T; backward: dA = R(g) R(W), dW = R(g)^T R(A)."""

    @staticmethod
    def forward(ctx, A, W):
        a, w = R(A), R(W)
        ctx.save_for_backward(a, w)
        return a @ w.T

    @staticmethod
    def backward(ctx, g):
        a, w = ctx.saved_tensors
        gr = R(g)
        return gr @ w, gr.T @ a


class _Conv(torch.autograd.Function):
    """y = conv(R(x), R(w)) (optionally grouped); backward from R(dy)."""

    @staticmethod
    def forward(ctx, x, w, stride, padding, groups):
        xr, wr = R(x), R(w)
        ctx.save_for_backward(xr, wr)
        ctx.cfg = (stride, padding, groups, x.shape, w.shape)
        return F.conv2d(xr, wr, stride=stride, padding=padding, groups=groups)

    @staticmethod
    def backward(ctx, g):
        xr, wr = ctx.saved_tensors
        stride, padding, groups, xs, ws = ctx.cfg
        gr = R(g)
        dx = torch.nn.grad.conv2d_input(xs, wr, gr, stride=stride, padding=padding, groups=groups)
        dw = torch.nn.grad.conv2d_weight(xr, ws, gr, stride=stride, padding=padding, groups=groups)
        return dx, dw, None, None, None


def linear(A, W):
    return _Linear.apply(A, W)


def conv(x, w, stride=1, padding=0, groups=1):
    return _Conv.apply(x, w, stride, padding, groups)


def store(x):
    return _Store.apply(x)


def _gn(x, g, b, eps):
    return F.group_norm(x, x.shape[1] // 2, g, b, eps)


def encoder(p, obs, cfg):
    """obs [N, 1, h, w] -> features [N, F] (NCHW flatten), as oracle.policy.encoder."""
    x = obs
    if cfg.net_kind == 0:
        x = F.relu(conv(x, p["c1.w"], 4) + p["c1.b"][:, None, None])
        x = F.relu(conv(x, p["c2.w"], 2) + p["c2.b"][:, None, None])
        x = F.relu(conv(x, p["c3.w"], 1) + p["c3.b"][:, None, None])
        return x.flatten(1)
    e = cfg.gn_eps
    x = F.relu(_gn(conv(x, p["stem.w"], 2, 3), p["stem.g"], p["stem.b"], e))
    x = F.max_pool2d(x, 3, stride=2, padding=1)
    if cfg.net_kind == 3:
        # SE-ResNeXt: the three convolutions read bf16 copies; the squeeze-excite FCs, the
        # GroupNorms and the shortcut stay fp32
        for i, (_, _, _, s) in enumerate(OP._sx_blocks(cfg)):
            q = f"x{i}."
            y = F.relu(_gn(conv(x, p[q + "c1.w"]), p[q + "n1.g"], p[q + "n1.b"], e))
            y = F.relu(_gn(conv(y, p[q + "c2.w"], s, 1, cfg.cardinality), p[q + "n2.g"],
                           p[q + "n2.b"], e))
            y = _gn(conv(y, p[q + "c3.w"]), p[q + "n3.g"], p[q + "n3.b"], e)
            y = OP.squeeze_excite(p, q, y)
            if q + "d.w" in p:
                sc = _gn(conv(x, p[q + "d.w"], s), p[q + "nd.g"], p[q + "nd.b"], e)
            else:
                sc = x
            x = F.relu(y + sc)
        x = F.relu(_gn(conv(x, p["cmp.w"], 1, 1), p["cmp.g"], p["cmp.b"], e))
        return x.flatten(1)
    for i, (cin, cout, s) in enumerate(OP._resnet_blocks(cfg.base_ch)):
        q = f"b{i}."
        y = F.relu(_gn(conv(x, p[q + "c1.w"], s, 1), p[q + "n1.g"], p[q + "n1.b"], e))
        y = _gn(conv(y, p[q + "c2.w"], 1, 1), p[q + "n2.g"], p[q + "n2.b"], e)
        if q + "d.w" in p:
            sc = _gn(conv(x, p[q + "d.w"], s, 0), p[q + "nd.g"], p[q + "nd.b"], e)
        else:
            sc = x
        x = F.relu(y + sc)
    x = F.relu(_gn(conv(x, p["cmp.w"], 1, 1), p["cmp.g"], p["cmp.b"], e))
    return x.flatten(1)


def policy_inputs(p, obs, goal, prev_a, cfg):
    gvec = store(goal @ p["goal.w"].T + p["goal.b"])
    avec = store(p["act.emb"][prev_a.long()])
    if cfg.net_kind == 2:
        return torch.cat([gvec, avec], dim=1)
    v = store(F.relu(linear(encoder(p, obs, cfg), p["vis.w"]) + p["vis.b"]))
    return torch.cat([v, gvec, avec], dim=1)


def sequence_forward(p, obs, goal, prev_a, masks, h0, c0, cfg):
    """The oracle's sequence_forward with the BF16 form's rounding points."""
    T, E = prev_a.shape
    x_all = policy_inputs(p, obs.reshape(T * E, *obs.shape[2:]), goal.reshape(T * E, 3),
                          prev_a.reshape(T * E), cfg).reshape(T, E, -1)
    L, Hd = cfg.lstm_layers, cfg.hidden
    h = [h0[l] for l in range(L)]
    c = [c0[l] for l in range(L)]
    logits, values = [], []
    for t in range(T):
        m = masks[t].to(DT).unsqueeze(1)
        x = x_all[t]
        for l in range(L):
            z = (linear(x, p[f"lstm{l}.w_ih"]) + linear(store(h[l] * m), p[f"lstm{l}.w_hh"])
                 + p[f"lstm{l}.b_ih"] + p[f"lstm{l}.b_hh"])
            i = torch.sigmoid(z[:, 0:Hd])
            f = torch.sigmoid(z[:, Hd:2 * Hd])
            g = torch.tanh(z[:, 2 * Hd:3 * Hd])
            o = torch.sigmoid(z[:, 3 * Hd:4 * Hd])
            c[l] = f * (c[l] * m) + i * g
            h[l] = o * torch.tanh(c[l])
            x = h[l]  # the next layer's linear() reads it as its bf16 copy
        logits.append(x @ p["actor.w"].T + p["actor.b"])
        values.append((x @ p["critic.w"].T + p["critic.b"])[:, 0])
    return torch.stack(logits), torch.stack(values), torch.stack(h), torch.stack(c)


@contextlib.contextmanager
def in_oracle():
    """Route oracle.policy.sequence_forward (used by oracle.rl's loss, gradient and PPO
    update) through this emulation while the context is open."""
    orig = OP.sequence_forward
    OP.sequence_forward = sequence_forward
    try:
        yield
    finally:
        OP.sequence_forward = orig
