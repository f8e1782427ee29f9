"""The encoder's GroupNorm in one launch (statistics and normalisation in one cooperative
grid, the blocks of an image meeting at a bounded barrier) against the two-launch form
(a statistics kernel, then a normalise kernel). The arithmetic is the same; the one-launch
form may split an image over fewer blocks, which changes only the fp32 order in which the
per-block sums are added. So in FP32 the logits, values, LSTM states and gradients agree
to fp32 accuracy (1e-5 relative; 1e-4 for per-tensor gradients), and a whole PPO update
agrees within 2% of lr x steps per coordinate."""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from paper_1911_00357_gb300 import binding as B
from tests import inputs as I
from tests.test_gpu_policy import Net, _cfg, _dev_inputs, _rollout_tensors, _view
from tests.test_gpu_sx import _sx_cfg

pytestmark = pytest.mark.gpu


def _cfg_of(name, E, T, mb=1):
    if name == "sx50_16":
        return _sx_cfg(3, 16, E, T, 0, mb=mb)
    return _cfg(name, E, T, 0, mb=mb)


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


@pytest.mark.parametrize("name,T,E", [("resnet_small", 4, 6), ("resnet_full", 3, 8),
                                      ("sx50_16", 2, 3)])
def test_one_launch_matches_two_launches(name, T, E):
    cfg = _cfg_of(name, E, T)
    net = Net(cfg, seed=1)
    try:
        a = _run(net, T, E, True)
        b = _run(net, T, E, False)
        for nm, x, y in zip(["logits", "values", "grad", "h", "c", "logp", "value"], a, b):
            if nm == "grad":
                off, err = 0, 0.0
                for _, shp in OP.param_spec(net.ncfg):
                    k = int(np.prod(shp))
                    gy = y[off:off + k]
                    ny = torch.linalg.vector_norm(gy).item()
                    if ny > 1e-8:
                        err = max(err, torch.linalg.vector_norm(x[off:off + k] - gy).item() / ny)
                    off += k
                lim = 1e-4
            else:
                err = (x - y).abs().max().item() / max(y.abs().max().item(), 1e-6)
                lim = 1e-5
            assert err <= lim, (nm, err)
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
    (a, f0), (b, _) = outs
    assert ((a - f0) - (b - f0)).abs().max().item() <= 0.02 * 2.5e-4 * 4
