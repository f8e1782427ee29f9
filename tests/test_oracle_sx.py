"""Pins of the SE-ResNeXt encoder of the oracle (App. "Visual Encoder": SE-ResNeXt50 with
every layer's channels halved, GroupNorm for BatchNorm). Its gradient is pinned by central
differences in test_oracle_rl.py (tiny_sx); here: the feature-map shape the paper states,
and the two limits of the squeeze-excite gate, which fix where the gate sits."""
import torch
import torch.nn.functional as F

from oracle import policy as OP
from tests import inputs as I


def test_halved_se_resnext50_backbone_is_1024x4x4_at_128x128():
    # "each backbone produces a 1024x4x4 feature map" for the 128x128 effective input
    cfg = OP.NetConfig(net_kind=3, base_ch=32, hidden=512, lstm_layers=2, in_h=128, in_w=128)
    p = OP.unflatten(I.params(cfg, seed=1), cfg)
    x = torch.rand(1, 1, 128, 128, dtype=torch.float64)
    e = cfg.gn_eps
    x = F.relu(OP._gn(F.conv2d(x, p["stem.w"], stride=2, padding=3), p["stem.g"], p["stem.b"], e))
    x = F.max_pool2d(x, 3, stride=2, padding=1)
    for i, (_, _, _, s) in enumerate(OP._sx_blocks(cfg)):
        x = OP.sx_block(p, f"x{i}.", x, s, cfg)
    assert tuple(x.shape) == (1, 1024, 4, 4)
    assert OP.feature_dim(cfg) == 128 * 4 * 4
    assert len(OP._sx_blocks(cfg)) == 16      # 3 + 4 + 6 + 3 bottlenecks: 50 layers
    cfg101 = OP.NetConfig(net_kind=3, base_ch=32, sx_blocks=(3, 4, 23, 3))
    assert len(OP._sx_blocks(cfg101)) == 33   # 101 layers


def _identity_block_params(seed):
    cfg = OP.NetConfig(net_kind=3, base_ch=4, sx_blocks=(2, 1, 1, 1), cardinality=2, se_reduction=4)
    p = dict(OP.unflatten(I.params(cfg, seed=seed), cfg))
    return cfg, p, "x1."   # block 1 of stage 1: 16 -> 16 channels, stride 1, identity shortcut


def test_closed_squeeze_excite_gate_makes_the_block_an_identity():
    # gate = sigmoid(-60) ~ 1e-26: the branch is switched off, and relu(0 + x) = x for the
    # non-negative input every block receives
    cfg, p, q = _identity_block_params(3)
    p[q + "se2.w"] = torch.zeros_like(p[q + "se2.w"])
    p[q + "se2.b"] = torch.full_like(p[q + "se2.b"], -60.0)
    x = torch.relu(torch.randn(2, 16, 8, 8, dtype=torch.float64))
    y = OP.sx_block(p, q, x, 1, cfg)
    assert torch.allclose(y, x, rtol=0, atol=1e-20)


def test_open_squeeze_excite_gate_leaves_the_bottleneck():
    # gate = sigmoid(60) = 1 in float64: the block is the plain ResNeXt bottleneck
    # relu(GN(conv1x1(relu(GN(gconv3x3(relu(GN(conv1x1 x)))))) + x), written out here
    cfg, p, q = _identity_block_params(4)
    p[q + "se2.w"] = torch.zeros_like(p[q + "se2.w"])
    p[q + "se2.b"] = torch.full_like(p[q + "se2.b"], 60.0)
    x = torch.relu(torch.randn(2, 16, 8, 8, dtype=torch.float64))
    gn = lambda t, n: F.group_norm(t, t.shape[1] // 2, p[q + n + ".g"], p[q + n + ".b"], 1e-5)
    b = F.relu(gn(F.conv2d(x, p[q + "c1.w"]), "n1"))
    b = F.relu(gn(F.conv2d(b, p[q + "c2.w"], padding=1, groups=2), "n2"))
    b = gn(F.conv2d(b, p[q + "c3.w"]), "n3")
    want = F.relu(b + x)
    assert torch.allclose(OP.sx_block(p, q, x, 1, cfg), want, rtol=1e-15, atol=1e-15)
