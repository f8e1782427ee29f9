"""The encoder's GroupNorm in one launch (statistics and normalisation in one cooperative
grid, the blocks of an image meeting at a bounded barrier) against the two-launch form
(a statistics kernel, then a normalise kernel). Both split an image over the same number
of blocks and add the per-block sums in the same order, so every output -- logits,
values, LSTM states, every gradient, the parameters after a whole PPO update -- is
bit-identical between the two forms."""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from tests import inputs as I
from tests.test_gpu_policy import Net, _cfg, _dev_inputs, _rollout_tensors, _view
from tests.test_gpu_sx import _sx_cfg

pytestmark = pytest.mark.gpu


def _cfg_of(name, E, T, precision=0, mb=1):
    if name == "sx50_16":
        return _sx_cfg(3, 16, E, T, precision, mb=mb)
    return _cfg(name, E, T, precision, mb=mb)


def _run(net, T, E, one):
    B.ddppo_group_norm_one_launch(net.h, one)
    mb = I.minibatch(net.ncfg, T=T, E=E, seed=2)
    dev, _ = _dev_inputs(net.cfg, mb)
    logits = torch.zeros(T, E, 4, device="cuda")
    values = torch.zeros(T, E, device="cuda")
    B.ddppo_policy_evaluate(net.h, T, E, dev["obs"], dev["goal"], dev["prev_a"], dev["masks"],
                            dev["h0"], dev["c0"], logits, values)
    g = torch.Generator().manual_seed(3)
    dl = torch.randn(T, E, 4, generator=g).cuda()
    dv = torch.randn(T, E, generator=g).cuda()
    grad = torch.zeros(net.P, device="cuda")
    B.ddppo_policy_backward(net.h, dl, dv, grad)
    h, c = dev["h0"].clone(), dev["c0"].clone()
    act = torch.zeros(E, dtype=torch.int32, device="cuda")
    logp = torch.zeros(E, device="cuda")
    val = torch.zeros(E, device="cuda")
    u = torch.from_numpy(I.uniforms(1, E, seed=6)[0]).cuda()
    B.ddppo_policy_act(net.h, dev["obs"][0], dev["goal"][0], dev["prev_a"][0], dev["masks"][0],
                       h, c, u, act, logp, val)
    torch.cuda.synchronize()
    assert B.ddppo_device_status(net.h) == 0
    return [x.cpu().double() for x in (logits, values, grad, h, c, logp, val)]


@pytest.mark.parametrize("name,T,E,precision", [("resnet_small", 4, 6, 0), ("resnet_full", 3, 8, 0),
                                                ("resnet_full", 3, 8, 1), ("sx50_16", 2, 3, 0),
                                                ("resnet_small", 16, 64, 1)])
def test_one_launch_matches_two_launches(name, T, E, precision):
    cfg = _cfg_of(name, E, T, precision)
    net = Net(cfg, seed=1)
    try:
        a = _run(net, T, E, True)
        b = _run(net, T, E, False)
        for nm, x, y in zip(["logits", "values", "grad", "h", "c", "logp", "value"], a, b):
            assert torch.equal(x, y), (nm, (x - y).abs().max().item())
    finally:
        net.close()


def test_one_launch_update_matches_two_launches():
    T, E, mb = 8, 4, 2
    outs = []
    for one in (True, False):
        cfg = _cfg("resnet_small", E, T, 0, mb=mb)
        net = Net(cfg, seed=7)
        try:
            B.ddppo_group_norm_one_launch(net.h, one)
            ro_t, _ = _rollout_tensors(cfg, net, T, E, seed=8)
            B.ddppo_ppo_update(net.h, _view(ro_t), B.default_hparams(minibatches=mb, update_index=3))
            out = torch.zeros(net.P, device="cuda")
            B.ddppo_get_params(net.h, out)
            torch.cuda.synchronize()
            assert B.ddppo_device_status(net.h) == 0
            outs.append((out.cpu().double(), net.flat64()))
        finally:
            net.close()
    (a, _), (b, _) = outs
    assert torch.equal(a, b)
