"""The torch.autograd.Function wrappers (paper_1911_00357_gb300/autograd.py) on the FP32
form, at the differentiation workload's check size: a 4-env slice (T = 8) of the
ResNet-18/32 agent with the 2-layer LSTM 512, and the 3-layer conv agent.

Each wrapper's gradient is checked two ways:
  - against float64 autograd of the oracle's definition of the same piece (encoder,
    LSTM layers, whole agent + PPO loss), within the FP32 form's tolerances;
  - by central finite differences of the FP32 forward along random directions in
    parameter space: (L(theta + h v) - L(theta - h v)) / 2h against grad . v, within 2%
    (FP32 forwards and ReLU kinks limit the differences' accuracy).
"""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from oracle import rl as OR
from paper_1911_00357_gb300 import autograd as AG
from paper_1911_00357_gb300 import binding as B
from tests import inputs as I
from tests.test_gpu_policy import Net, _cfg, _dev_inputs

pytestmark = pytest.mark.gpu
DT = torch.float64


def _slices(ncfg, prefixes):
    """Boolean mask over the flat parameters of the tensors whose names start with one
    of the prefixes."""
    mask, off = [], 0
    for name, shp in OP.param_spec(ncfg):
        k = int(np.prod(shp))
        mask.append(torch.full((k,), name.startswith(prefixes), dtype=torch.bool))
        off += k
    return torch.cat(mask)


def _directional_fd(loss_of, theta, g, mask, loss64=None, n_dirs=3, rel=1e-3, seed=0):
    """Central differences (L(theta + h v) - L(theta - h v)) / 2h of the FP32 forward along
    directions v supported on mask: the gradient's own direction, then mixtures of it with
    random directions. Returns (fd, g . v, fd of the float64 oracle forward or None)."""
    gen = torch.Generator().manual_seed(seed)
    gm = g.double() * mask
    out = []
    for i in range(n_dirs):
        v = gm / torch.linalg.vector_norm(gm)
        if i:
            r = torch.randn(theta.numel(), generator=gen, dtype=DT) * mask
            v = v + r / torch.linalg.vector_norm(r)
            v = v / torch.linalg.vector_norm(v)
        h = rel * torch.linalg.vector_norm(theta.double()[mask]).item()
        tp, tm = (theta.double() + h * v).float(), (theta.double() - h * v).float()
        # the step actually taken, after rounding the perturbed parameters to fp32
        hv = (tp.double() - tm.double()) / 2
        fd = (loss_of(tp) - loss_of(tm)) / 2
        fd64 = (loss64(tp.double()) - loss64(tm.double())) / 2 if loss64 is not None else None
        out.append((fd, float(g.double() @ hv), fd64))
    return out


ENC = ("c1.", "c2.", "c3.", "stem.", "b", "cmp.")


@pytest.mark.parametrize("name", ["resnet_full", "nature_full"])
def test_encoder_function(name):
    T, E = 8, 4
    cfg = _cfg(name, E, T, 0)
    net = Net(cfg, seed=11)
    try:
        nc = net.ncfg
        F = OP.feature_dim(nc)
        mb = I.minibatch(nc, T=T, E=E, seed=12)
        obs = mb["obs"].reshape(T * E, 1, nc.in_h, nc.in_w).float().cuda()
        w = torch.randn(T * E, F, generator=torch.Generator().manual_seed(13), dtype=DT)
        wd = w.float().cuda()
        params = net.flat32.cuda().requires_grad_(True)
        feat = AG.EncoderFunction.apply(params, obs, net.h, F)
        (feat * wd).sum().backward()
        g = params.grad.cpu()
        # float64 oracle
        f64 = net.flat64().clone().requires_grad_(True)
        feat_r = OP.encoder(OP.unflatten(f64, nc), obs.cpu().double(), nc)
        (g_r,) = torch.autograd.grad((feat_r * w).sum(), f64)
        assert (feat.detach().cpu().double() - feat_r.detach()).abs().max() <= 1e-4 * feat_r.abs().max()
        mask = _slices(nc, ENC)
        assert torch.count_nonzero(g[~mask]) == 0  # only encoder tensors get a gradient
        err = torch.linalg.vector_norm(g.double() - g_r) / torch.linalg.vector_norm(g_r)
        assert err <= (3e-2 if name == "resnet_full" else 1e-3), err.item()

        def loss_of(theta):
            with torch.no_grad():
                f = AG.EncoderFunction.apply(theta.cuda(), obs, net.h, F)
                return float((f.double() * w.cuda()).sum())

        def loss64(theta):
            with torch.no_grad():
                return float((OP.encoder(OP.unflatten(theta, nc), obs.cpu().double(), nc) * w).sum())
        # the GroupNorm ResNet is piecewise smooth (ReLU, max pool): differences over a finite
        # step carry its kinks, in float64 as well; the FP32 forward's differences must track
        # the oracle's, and the gradient the differences within the kink error
        # (a step of 2e-5 of the parameter norm keeps the kinks' share of the difference small)
        rel = 2e-5 if name == "resnet_full" else 2e-4
        for fd, gv, fd64 in _directional_fd(loss_of, net.flat32, g, mask, loss64, rel=rel):
            assert abs(fd - fd64) <= 1e-2 * abs(fd64) + 1e-6, (fd, fd64)
            assert abs(fd - gv) <= 5e-2 * abs(gv) + 1e-6, (fd, gv)
    finally:
        AG.sync_params.forget(net.h)
        net.close()


def _oracle_lstm(p, x, masks, h0, c0, ncfg):
    T = x.shape[0]
    h = [h0[l] for l in range(ncfg.lstm_layers)]
    c = [c0[l] for l in range(ncfg.lstm_layers)]
    ys = []
    for t in range(T):
        m = masks[t].to(DT).unsqueeze(1)
        z = x[t]
        for l in range(ncfg.lstm_layers):
            h[l], c[l] = OP.lstm_cell(z, h[l] * m, c[l] * m, p[f"lstm{l}.w_ih"], p[f"lstm{l}.w_hh"],
                                      p[f"lstm{l}.b_ih"], p[f"lstm{l}.b_hh"])
            z = h[l]
        ys.append(z)
    return torch.stack(ys)


def test_lstm_function():
    T, E = 8, 4
    cfg = _cfg("resnet_full", E, T, 0)
    net = Net(cfg, seed=14)
    try:
        nc = net.ncfg
        In0 = nc.hidden + 64
        gen = torch.Generator().manual_seed(15)
        x = torch.randn(T, E, In0, generator=gen, dtype=DT)
        mb = I.minibatch(nc, T=T, E=E, seed=16)
        dev, ref = _dev_inputs(cfg, mb)
        w = torch.randn(T, E, nc.hidden, generator=gen, dtype=DT)
        params = net.flat32.cuda().requires_grad_(True)
        xd = x.float().cuda().requires_grad_(True)
        y = AG.LSTMFunction.apply(params, xd, dev["masks"], dev["h0"], dev["c0"], net.h, nc.hidden)
        (y * w.float().cuda()).sum().backward()
        g, gx = params.grad.cpu(), xd.grad.cpu()
        f64 = net.flat64().clone().requires_grad_(True)
        x64 = xd.detach().cpu().double().requires_grad_(True)
        y_r = _oracle_lstm(OP.unflatten(f64, nc), x64, ref["masks"], ref["h0"], ref["c0"], nc)
        g_r, gx_r = torch.autograd.grad((y_r * w).sum(), (f64, x64))
        assert (y.detach().cpu().double() - y_r.detach()).abs().max() <= 1e-4 * y_r.abs().max()
        mask = _slices(nc, ("lstm",))
        assert torch.count_nonzero(g[~mask]) == 0
        assert torch.linalg.vector_norm(g.double() - g_r) <= 1e-3 * torch.linalg.vector_norm(g_r)
        assert torch.linalg.vector_norm(gx.double() - gx_r) <= 1e-3 * torch.linalg.vector_norm(gx_r)

        def loss_of(theta):
            with torch.no_grad():
                yy = AG.LSTMFunction.apply(theta.cuda(), xd.detach(), dev["masks"], dev["h0"],
                                           dev["c0"], net.h, nc.hidden)
                return float((yy.double() * w.cuda()).sum())
        for fd, gv, _ in _directional_fd(loss_of, net.flat32, g, mask):
            assert abs(fd - gv) <= 2e-2 * abs(gv) + 1e-6, (fd, gv)
    finally:
        AG.sync_params.forget(net.h)
        net.close()


@pytest.mark.parametrize("name", ["resnet_full", "nature_full"])
def test_policy_and_ppo_loss_functions(name):
    T, E = 8, 4
    cfg = _cfg(name, E, T, 0)
    net = Net(cfg, seed=17)
    try:
        nc = net.ncfg
        mb = I.minibatch(nc, T=T, E=E, seed=18)
        dev, ref = _dev_inputs(cfg, mb)
        hp = OR.PPOHParams()
        act = mb["actions"].int().cuda()
        lo, adv, ret = (mb[k].float().cuda() for k in ("logp_old", "adv", "ret"))
        params = net.flat32.cuda().requires_grad_(True)
        stats = torch.zeros(B.NSTATS, device="cuda")

        def loss_fn(theta, st=None):
            lg, vv = AG.PolicyFunction.apply(theta, dev["obs"], dev["goal"], dev["prev_a"],
                                             dev["masks"], dev["h0"], dev["c0"], net.h)
            return AG.PPOLossFunction.apply(lg, vv, act, lo, adv, ret, hp.clip, hp.value_coef,
                                            hp.entropy_coef, st)
        loss = loss_fn(params, stats)
        loss.backward()
        g = params.grad.cpu()
        mbr = dict(ref)
        mbr.update(actions=mb["actions"], logp_old=lo.cpu().double(), adv=adv.cpu().double(),
                   ret=ret.cpu().double())
        l_r, st_r, g_r = OR.minibatch_loss_and_grad(net.flat64(), mbr, nc, hp)
        assert abs(loss.item() - l_r.item()) <= 1e-4 * max(1.0, abs(l_r.item()))
        assert abs(stats[0].item() - loss.item()) == 0.0
        err = torch.linalg.vector_norm(g.double() - g_r) / torch.linalg.vector_norm(g_r)
        assert err <= (3e-2 if name == "resnet_full" else 1e-3), err.item()
        # a loss scaled by 3 scales the gradient by 3 (the upstream factor)
        params.grad = None
        (3.0 * loss_fn(params)).backward()
        g3 = params.grad.cpu().double()
        assert torch.linalg.vector_norm(g3 - 3 * g.double()) <= 1e-5 * torch.linalg.vector_norm(3 * g.double())

        def loss_of(theta):
            with torch.no_grad():
                return float(loss_fn(theta.cuda()))
        mask = torch.ones(net.P, dtype=torch.bool)
        tol = 5e-2 if name == "resnet_full" else 2e-2
        rel = 2e-5 if name == "resnet_full" else 2e-4
        for fd, gv, _ in _directional_fd(loss_of, net.flat32, g, mask, rel=rel):
            assert abs(fd - gv) <= tol * abs(gv) + 1e-6, (fd, gv)
    finally:
        AG.sync_params.forget(net.h)
        net.close()
