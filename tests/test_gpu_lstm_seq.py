"""The whole-segment LSTM kernels (one cooperative launch per layer for the T-step forward
and for its back-propagation through time) against the step-by-step path (a recurrent
contraction and a cell kernel per step). Both compute the same arithmetic; only the
recurrent contraction's fp32 summation order differs, so results agree to fp32 accuracy:
logits, values, LSTM states and every gradient tensor within 1e-5 relative (1e-4 for the
gradients, which sum over the segment), and a whole 2 x 2 PPO update within 2% of
lr x steps per coordinate. The float64 oracle parity of the default (step-by-step) path
is covered by the policy and update parity tests.
"""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from paper_1911_00357_gb300 import binding as B
from tests import inputs as I
from tests.test_gpu_policy import Net, _cfg, _dev_inputs, _rollout_tensors, _view

pytestmark = pytest.mark.gpu


def _cfg2(name, E, T, precision, mb=1):
    # hidden sizes whose units split unevenly over the SMs (U = 2 units per CTA for H = 32)
    extra = {"nature_h32": dict(hidden=32), "nature_h64": dict(hidden=64)}
    if name in extra:
        from paper_1911_00357_gb300.presets import make_config
        return make_config("nature_fp32", num_envs=E, rollout_T=T, minibatches=mb,
                           precision=precision, lstm_layers=2, **extra[name])
    return _cfg(name, E, T, precision, mb=mb)


def _run(net, cfg, T, E, whole):
    B.ddppo_lstm_whole_segment(net.h, whole)
    mb = I.minibatch(net.ncfg, T=T, E=E, seed=2)
    dev, _ = _dev_inputs(cfg, mb)
    logits = torch.zeros(T, E, 4, device="cuda")
    values = torch.zeros(T, E, device="cuda")
    B.ddppo_policy_evaluate(net.h, T, E, dev["obs"], dev["goal"], dev["prev_a"], dev["masks"],
                            dev["h0"], dev["c0"], logits, values)
    g = torch.Generator().manual_seed(3)
    dl = torch.randn(T, E, 4, generator=g).cuda()
    dv = torch.randn(T, E, generator=g).cuda()
    grad = torch.zeros(net.P, device="cuda")
    B.ddppo_policy_backward(net.h, dl, dv, grad)
    # one act step (T = 1: the same kernel without a barrier)
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


@pytest.mark.parametrize("name,T,E,precision", [("nature_small", 7, 5, 0), ("resnet_small", 6, 4, 0),
                                                ("nature_h32", 5, 3, 0), ("nature_h64", 5, 64, 0),
                                                ("blind_full", 9, 6, 0), ("nature_full", 8, 33, 0),
                                                ("blind_full", 9, 6, 1), ("resnet_full", 4, 3, 1)])
def test_whole_segment_matches_step_by_step(name, T, E, precision):
    cfg = _cfg2(name, E, T, precision)
    net = Net(cfg, seed=1)
    try:
        a = _run(net, cfg, T, E, True)
        b = _run(net, cfg, T, E, False)
        names = ["logits", "values", "grad", "h", "c", "logp", "value"]
        tol = {"grad": 1e-4}
        for nm, x, y in zip(names, a, b):
            if nm == "grad":
                off, worst = 0, 0.0
                for pname, shp in OP.param_spec(net.ncfg):
                    k = int(np.prod(shp))
                    gy = y[off:off + k]
                    ny = torch.linalg.vector_norm(gy).item()
                    if ny > 1e-8:
                        worst = max(worst, torch.linalg.vector_norm(x[off:off + k] - gy).item() / ny)
                    off += k
                err = worst
            else:
                err = (x - y).abs().max().item() / max(y.abs().max().item(), 1e-6)
            # BF16 operands: an fp32 summation difference can flip a bf16 rounding of the
            # recurrent state (a 2^-9 step) -- bounded by a few bf16 units
            lim = tol.get(nm, 1e-5) if precision == 0 else 2e-2
            assert err <= lim, (nm, err)
    finally:
        net.close()


def test_whole_segment_update_matches_step_by_step():
    T, E, mb = 8, 4, 2
    outs = []
    for whole in (True, False):
        cfg = _cfg("resnet_small", E, T, 0, mb=mb)
        net = Net(cfg, seed=7)
        try:
            B.ddppo_lstm_whole_segment(net.h, whole)
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
