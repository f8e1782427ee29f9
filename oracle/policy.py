"""FP64 CPU oracle of the DD-PPO PointGoal agent (Sec. 4 "Agent"; App. "Agent Design").

TEST INFRASTRUCTURE ONLY. Plain float64 PyTorch CPU ops (conv2d, group_norm,
matmul as library primitives); the LSTM, heads and action sampling are written
out by their definitions, one time step at a time.

Architecture (the paper's agent with the widths of the synthetic workloads):
  visual encoder -> flatten -> FC to hidden + ReLU          (App. "Navigation Policy")
  goal [r, cos, sin] -> FC -> 32                             (App. "Goal encoder")
  previous action (4 = start token) -> 32-d embedding        (App. "Navigation Policy")
  concat -> L-layer LSTM (gates i, f, g, o) -> actor (4) + critic (1)
Encoders:
  kind 0 ("nature"): conv 8x8/4 -> 32, 4x4/2 -> 64, 3x3/1 -> 32, ReLU after each, biases.
  kind 1 ("resnet18"): ResNet-18 BasicBlocks with base width c (c, 2c, 4c, 8c), stem
     7x7/2 + maxpool 3x3/2, GroupNorm (C/2 groups) in place of BatchNorm (App. "Visual
     Encoder"), then a 3x3 conv to 128 channels + GroupNorm + ReLU (128x4x4 = 2048-d).
  kind 2 ("blind"): no visual input at all, the agent trained with only the GPS+Compass
     sensor (Sec. 5): the LSTM input is [goal FC, action embedding].
  kind 3 ("se_resnext"): SE-ResNeXt (App. "Visual Encoder": SE-ResNeXt50/101 with every
     layer's channels halved, GroupNorm for BatchNorm, 1024x4x4 output). Bottleneck
     blocks [3, 4, 6, 3] (50) or [3, 4, 23, 3] (101): 1x1 conv to the inner width 2c 2^i,
     3x3 grouped conv (cardinality groups, stride here), 1x1 conv to 4c 2^i, each with
     GroupNorm, ReLU after the first two; squeeze-excite on the branch (global mean, FC to
     C/r + ReLU, FC back + sigmoid, channel scale) before the residual addition; 1x1 conv
     + GroupNorm shortcut when the shape changes. Stem, max pool and the 3x3 compression
     conv to 128 channels as in kind 1.
The 2x2 average pool of App. "Visual Encoder" is applied when the observation is
produced (``oracle.sim.pool_obs``), so the encoder input is already [1, 128, 128].

The flat parameter vector is the concatenation, in ``param_spec`` order, of each
tensor in PyTorch's natural layout (conv [Cout, Cin, kh, kw], linear [out, in]).

Pins (tests/test_oracle_rl.py, tests/test_oracle_sx.py, tests/test_oracle_pins_loss.py):
  conv2d / _gn        loop definitions of convolution and GroupNorm (biased variance, C/2
                      groups)
  lstm_cell           torch.nn.LSTM on the same weights (gate order i, f, g, o)
  feature_dim / encoder  128x4x4 = 2048 at 128x128 (App. "Visual Encoder"); SE-ResNeXt's
                      1024x4x4 backbone, block counts, closed and open squeeze-excite gates
  policy_inputs       concatenation order [visual, goal, action] on hand-set weights
  sequence_forward    masks zero the state before the step (h0 has no effect at mask 0)
  sample_action       inverse-CDF closed form
  all of the above, through the PPO loss: central finite differences of the gradient
"""
from __future__ import annotations

import dataclasses

import torch
import torch.nn.functional as F

DT = torch.float64
START_TOKEN = 4
NUM_ACTIONS = 4


@dataclasses.dataclass
class NetConfig:
    net_kind: int = 0          # 0 nature, 1 resnet18, 2 blind
    base_ch: int = 32
    hidden: int = 128
    lstm_layers: int = 1
    in_h: int = 64             # encoder input (after the optional 2x2 pool)
    in_w: int = 64
    goal_dim: int = 32
    act_dim: int = 32
    gn_eps: float = 1e-5
    # kind 3 only
    sx_blocks: tuple = (3, 4, 6, 3)   # bottleneck blocks per stage (50 layers)
    cardinality: int = 32             # groups of the 3x3 convolution
    se_reduction: int = 16            # squeeze-excite bottleneck ratio


def _resnet_blocks(c):
    """(cin, cout, stride) of the 8 BasicBlocks."""
    out = []
    cin = c
    for li, w in enumerate([c, 2 * c, 4 * c, 8 * c]):
        for b in range(2):
            s = 2 if (li > 0 and b == 0) else 1
            out.append((cin, w, s))
            cin = w
    return out


def _sx_blocks(cfg):
    """(cin, inner, cout, stride) of the SE-ResNeXt bottleneck blocks."""
    out = []
    c = cfg.base_ch
    cin = c
    for i, n in enumerate(cfg.sx_blocks):
        for b in range(n):
            s = 2 if (i > 0 and b == 0) else 1
            out.append((cin, 2 * c * 2 ** i, 4 * c * 2 ** i, s))
            cin = 4 * c * 2 ** i
    return out


def _conv_out(n, k, s, p):
    return (n + 2 * p - k) // s + 1


def feature_dim(cfg: NetConfig) -> int:
    if cfg.net_kind == 2:
        return 0
    if cfg.net_kind == 0:
        h = _conv_out(_conv_out(_conv_out(cfg.in_h, 8, 4, 0), 4, 2, 0), 3, 1, 0)
        w = _conv_out(_conv_out(_conv_out(cfg.in_w, 8, 4, 0), 4, 2, 0), 3, 1, 0)
        return 32 * h * w
    h, w = cfg.in_h, cfg.in_w
    h, w = _conv_out(h, 7, 2, 3), _conv_out(w, 7, 2, 3)
    h, w = _conv_out(h, 3, 2, 1), _conv_out(w, 3, 2, 1)
    strides = [s for (_, _, s) in _resnet_blocks(cfg.base_ch)] if cfg.net_kind == 1 else \
        [s for (_, _, _, s) in _sx_blocks(cfg)]
    for s in strides:
        h, w = _conv_out(h, 3, s, 1), _conv_out(w, 3, s, 1)
    return 128 * h * w


def param_spec(cfg: NetConfig) -> list[tuple[str, tuple[int, ...]]]:
    spec: list[tuple[str, tuple[int, ...]]] = []
    if cfg.net_kind == 0:
        spec += [("c1.w", (32, 1, 8, 8)), ("c1.b", (32,)), ("c2.w", (64, 32, 4, 4)),
                 ("c2.b", (64,)), ("c3.w", (32, 64, 3, 3)), ("c3.b", (32,))]
    elif cfg.net_kind == 1:
        c = cfg.base_ch
        spec += [("stem.w", (c, 1, 7, 7)), ("stem.g", (c,)), ("stem.b", (c,))]
        for i, (cin, cout, s) in enumerate(_resnet_blocks(c)):
            spec += [(f"b{i}.c1.w", (cout, cin, 3, 3)), (f"b{i}.n1.g", (cout,)), (f"b{i}.n1.b", (cout,)),
                     (f"b{i}.c2.w", (cout, cout, 3, 3)), (f"b{i}.n2.g", (cout,)), (f"b{i}.n2.b", (cout,))]
            if s != 1 or cin != cout:
                spec += [(f"b{i}.d.w", (cout, cin, 1, 1)), (f"b{i}.nd.g", (cout,)), (f"b{i}.nd.b", (cout,))]
        spec += [("cmp.w", (128, 8 * c, 3, 3)), ("cmp.g", (128,)), ("cmp.b", (128,))]
    elif cfg.net_kind == 3:
        c, G, r = cfg.base_ch, cfg.cardinality, cfg.se_reduction
        spec += [("stem.w", (c, 1, 7, 7)), ("stem.g", (c,)), ("stem.b", (c,))]
        for i, (cin, mid, cout, s) in enumerate(_sx_blocks(cfg)):
            q = f"x{i}."
            spec += [(q + "c1.w", (mid, cin, 1, 1)), (q + "n1.g", (mid,)), (q + "n1.b", (mid,)),
                     (q + "c2.w", (mid, mid // G, 3, 3)), (q + "n2.g", (mid,)), (q + "n2.b", (mid,)),
                     (q + "c3.w", (cout, mid, 1, 1)), (q + "n3.g", (cout,)), (q + "n3.b", (cout,)),
                     (q + "se1.w", (cout // r, cout)), (q + "se1.b", (cout // r,)),
                     (q + "se2.w", (cout, cout // r)), (q + "se2.b", (cout,))]
            if s != 1 or cin != cout:
                spec += [(q + "d.w", (cout, cin, 1, 1)), (q + "nd.g", (cout,)), (q + "nd.b", (cout,))]
        last = _sx_blocks(cfg)[-1][2]
        spec += [("cmp.w", (128, last, 3, 3)), ("cmp.g", (128,)), ("cmp.b", (128,))]
    Hd = cfg.hidden
    if cfg.net_kind != 2:
        spec += [("vis.w", (Hd, feature_dim(cfg))), ("vis.b", (Hd,))]
    spec += [("goal.w", (cfg.goal_dim, 3)), ("goal.b", (cfg.goal_dim,)),
             ("act.emb", (NUM_ACTIONS + 1, cfg.act_dim))]
    vis = 0 if cfg.net_kind == 2 else Hd
    for l in range(cfg.lstm_layers):
        In = vis + cfg.goal_dim + cfg.act_dim if l == 0 else Hd
        spec += [(f"lstm{l}.w_ih", (4 * Hd, In)), (f"lstm{l}.w_hh", (4 * Hd, Hd)),
                 (f"lstm{l}.b_ih", (4 * Hd,)), (f"lstm{l}.b_hh", (4 * Hd,))]
    spec += [("actor.w", (NUM_ACTIONS, Hd)), ("actor.b", (NUM_ACTIONS,)),
             ("critic.w", (1, Hd)), ("critic.b", (1,))]
    return spec


def num_params(cfg: NetConfig) -> int:
    n = 0
    for _, shp in param_spec(cfg):
        k = 1
        for s in shp:
            k *= s
        n += k
    return n


def unflatten(flat: torch.Tensor, cfg: NetConfig) -> dict[str, torch.Tensor]:
    out = {}
    off = 0
    for name, shp in param_spec(cfg):
        k = 1
        for s in shp:
            k *= s
        out[name] = flat[off:off + k].view(shp)
        off += k
    assert off == flat.numel(), (off, flat.numel())
    return out


def _gn(x, g, b, eps):
    return F.group_norm(x, x.shape[1] // 2, g, b, eps)


def encoder(p: dict, obs: torch.Tensor, cfg: NetConfig) -> torch.Tensor:
    """obs [N, 1, h, w] float64 -> visual features [N, F] (NCHW flatten order)."""
    x = obs
    if cfg.net_kind == 0:
        x = F.relu(F.conv2d(x, p["c1.w"], p["c1.b"], stride=4))
        x = F.relu(F.conv2d(x, p["c2.w"], p["c2.b"], stride=2))
        x = F.relu(F.conv2d(x, p["c3.w"], p["c3.b"], stride=1))
        return x.flatten(1)
    e = cfg.gn_eps
    x = F.relu(_gn(F.conv2d(x, p["stem.w"], stride=2, padding=3), p["stem.g"], p["stem.b"], e))
    x = F.max_pool2d(x, 3, stride=2, padding=1)
    if cfg.net_kind == 3:
        for i, (_, _, _, s) in enumerate(_sx_blocks(cfg)):
            x = sx_block(p, f"x{i}.", x, s, cfg)
        x = F.relu(_gn(F.conv2d(x, p["cmp.w"], padding=1), p["cmp.g"], p["cmp.b"], e))
        return x.flatten(1)
    for i, (cin, cout, s) in enumerate(_resnet_blocks(cfg.base_ch)):
        y = F.relu(_gn(F.conv2d(x, p[f"b{i}.c1.w"], stride=s, padding=1), p[f"b{i}.n1.g"], p[f"b{i}.n1.b"], e))
        y = _gn(F.conv2d(y, p[f"b{i}.c2.w"], stride=1, padding=1), p[f"b{i}.n2.g"], p[f"b{i}.n2.b"], e)
        if f"b{i}.d.w" in p:
            sc = _gn(F.conv2d(x, p[f"b{i}.d.w"], stride=s), p[f"b{i}.nd.g"], p[f"b{i}.nd.b"], e)
        else:
            sc = x
        x = F.relu(y + sc)
    x = F.relu(_gn(F.conv2d(x, p["cmp.w"], padding=1), p["cmp.g"], p["cmp.b"], e))
    return x.flatten(1)


def squeeze_excite(p: dict, q: str, y: torch.Tensor) -> torch.Tensor:
    """y * sigmoid(W2 relu(W1 mean_hw(y) + b1) + b2), per image and channel."""
    z = y.mean(dim=(2, 3))
    a = F.relu(z @ p[q + "se1.w"].T + p[q + "se1.b"])
    w = torch.sigmoid(a @ p[q + "se2.w"].T + p[q + "se2.b"])
    return y * w[:, :, None, None]


def sx_block(p: dict, q: str, x: torch.Tensor, stride: int, cfg: NetConfig) -> torch.Tensor:
    """One SE-ResNeXt bottleneck block (parameter prefix q)."""
    e = cfg.gn_eps
    y = F.relu(_gn(F.conv2d(x, p[q + "c1.w"]), p[q + "n1.g"], p[q + "n1.b"], e))
    y = F.relu(_gn(F.conv2d(y, p[q + "c2.w"], stride=stride, padding=1, groups=cfg.cardinality),
                   p[q + "n2.g"], p[q + "n2.b"], e))
    y = _gn(F.conv2d(y, p[q + "c3.w"]), p[q + "n3.g"], p[q + "n3.b"], e)
    y = squeeze_excite(p, q, y)
    if q + "d.w" in p:
        sc = _gn(F.conv2d(x, p[q + "d.w"], stride=stride), p[q + "nd.g"], p[q + "nd.b"], e)
    else:
        sc = x
    return F.relu(y + sc)


def lstm_cell(x, h, c, w_ih, w_hh, b_ih, b_hh):
    """One LSTM step by definition (gate order i, f, g, o)."""
    z = x @ w_ih.T + b_ih + h @ w_hh.T + b_hh
    Hd = h.shape[-1]
    i = torch.sigmoid(z[:, 0:Hd])
    f = torch.sigmoid(z[:, Hd:2 * Hd])
    g = torch.tanh(z[:, 2 * Hd:3 * Hd])
    o = torch.sigmoid(z[:, 3 * Hd:4 * Hd])
    c2 = f * c + i * g
    h2 = o * torch.tanh(c2)
    return h2, c2


def policy_inputs(p, obs, goal, prev_a, cfg):
    """Concatenated LSTM input for a batch of N frames."""
    gvec = goal @ p["goal.w"].T + p["goal.b"]
    avec = p["act.emb"][prev_a.long()]
    if cfg.net_kind == 2:
        return torch.cat([gvec, avec], dim=1)
    v = F.relu(encoder(p, obs, cfg) @ p["vis.w"].T + p["vis.b"])
    return torch.cat([v, gvec, avec], dim=1)


def sequence_forward(p, obs, goal, prev_a, masks, h0, c0, cfg):
    """Forward over a rollout segment (Sec. 4 "Training").

    obs [T, E, 1, h, w], goal [T, E, 3], prev_a [T, E] int, masks [T, E] (1 = keep
    the recurrent state, 0 = episode start: h, c <- 0 before the step), h0/c0 [L, E, Hd].
    Returns logits [T, E, 4], values [T, E], hT, cT.
    """
    T, E = prev_a.shape
    x_all = policy_inputs(p, obs.reshape(T * E, *obs.shape[2:]), goal.reshape(T * E, 3),
                          prev_a.reshape(T * E), cfg).reshape(T, E, -1)
    L = cfg.lstm_layers
    h = [h0[l] for l in range(L)]
    c = [c0[l] for l in range(L)]
    logits, values = [], []
    for t in range(T):
        m = masks[t].to(h0.dtype).unsqueeze(1)  # float64 here; a float32 state in the tests' fp32 floor
        x = x_all[t]
        for l in range(L):
            h[l], c[l] = lstm_cell(x, h[l] * m, c[l] * m, p[f"lstm{l}.w_ih"], p[f"lstm{l}.w_hh"],
                                   p[f"lstm{l}.b_ih"], p[f"lstm{l}.b_hh"])
            x = h[l]
        logits.append(x @ p["actor.w"].T + p["actor.b"])
        values.append((x @ p["critic.w"].T + p["critic.b"])[:, 0])
    return torch.stack(logits), torch.stack(values), torch.stack(h), torch.stack(c)


def sample_action(logits: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """a = min{k : CDF_k > u} for a caller-supplied uniform u in [0, 1)."""
    cdf = torch.cumsum(torch.softmax(logits, dim=-1), dim=-1)
    a = (cdf <= u.unsqueeze(-1)).sum(dim=-1)
    return a.clamp(max=NUM_ACTIONS - 1)


def act(p, obs, goal, prev_a, masks, h, c, u, cfg):
    """One inference step for E envs: returns action, log pi(a), V, h', c', logits."""
    lg, v, h2, c2 = sequence_forward(p, obs.unsqueeze(0), goal.unsqueeze(0), prev_a.unsqueeze(0),
                                     masks.unsqueeze(0), h, c, cfg)
    lg, v = lg[0], v[0]
    a = sample_action(lg, u)
    logp = torch.log_softmax(lg, dim=-1).gather(1, a.unsqueeze(1))[:, 0]
    return a, logp, v, h2, c2, lg
