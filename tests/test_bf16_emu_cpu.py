"""The BF16 emulation used by the GPU parity tests (tests/bf16_emu.py) is the oracle's
network plus rounding points: with rounding off it reproduces oracle.policy's outputs and
float64 autograd gradients to the last bits; with rounding on it moves them by a bf16-
sized amount (checked against the unit roundoff 2^-8)."""
import pytest
import torch

from oracle import policy as OP
from oracle import rl as OR
from tests import bf16_emu as EMU
from tests import inputs as I


def _grads(fwd, cfg, flat, mb):
    f = flat.clone().requires_grad_(True)
    p = OP.unflatten(f, cfg)
    lg, v, h, c = fwd(p, mb["obs"], mb["goal"], mb["prev_a"], mb["masks"], mb["h0"], mb["c0"], cfg)
    g = torch.Generator().manual_seed(9)
    wl = torch.randn(lg.shape, generator=g, dtype=torch.float64)
    wv = torch.randn(v.shape, generator=g, dtype=torch.float64)
    (gr,) = torch.autograd.grad((lg * wl).sum() + (v * wv).sum(), f)
    return lg.detach(), v.detach(), h.detach(), gr


@pytest.mark.parametrize("net", ["tiny", "tiny_resnet", "tiny_blind", "tiny_sx"])
def test_emulation_without_rounding_is_the_oracle(net):
    cfg = I.net_config(net)
    flat = I.params(cfg, seed=1)
    mb = I.minibatch(cfg, T=3, E=2, seed=2)
    ref = _grads(OP.sequence_forward, cfg, flat, mb)
    with EMU.rounding(False):
        got = _grads(EMU.sequence_forward, cfg, flat, mb)
    for a, b in zip(got, ref):
        assert torch.allclose(a, b, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("net", ["tiny", "tiny_resnet"])
def test_emulation_with_rounding_moves_results_by_bf16_amounts(net):
    cfg = I.net_config(net)
    flat = I.params(cfg, seed=1)
    mb = I.minibatch(cfg, T=3, E=2, seed=2)
    ref = _grads(OP.sequence_forward, cfg, flat, mb)
    got = _grads(EMU.sequence_forward, cfg, flat, mb)
    u = 2.0 ** -8
    for a, b in zip(got[:3], ref[:3]):
        rel = ((a - b).abs().max() / b.abs().max()).item()
        assert 1e-3 * u < rel < 20 * u, rel


def test_in_oracle_routes_the_ppo_gradient_through_the_emulation():
    cfg = I.net_config("tiny")
    flat = I.params(cfg, seed=3)
    mb = I.minibatch(cfg, T=3, E=2, seed=4)
    hp = OR.PPOHParams()
    _, _, g64 = OR.minibatch_loss_and_grad(flat, mb, cfg, hp)
    with EMU.in_oracle():
        _, _, gb = OR.minibatch_loss_and_grad(flat, mb, cfg, hp)
    assert OP.sequence_forward is not EMU.sequence_forward
    rel = (torch.linalg.vector_norm(gb - g64) / torch.linalg.vector_norm(g64)).item()
    assert 0 < rel < 0.1, rel


def test_rounding_is_round_to_nearest_even():
    x = torch.tensor([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -9), 3.0],
                     dtype=torch.float64)
    assert EMU.R(x).tolist() == [1.0, 1.0 + 2.0 ** -6, -1.0, 3.0]
