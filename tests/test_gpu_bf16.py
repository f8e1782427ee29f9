"""GPU parity of the BF16 form against a float64 emulation of the same bf16 roundings.

The BF16 form rounds the operands of every contraction, and the output gradients that
feed the backward contractions, to bfloat16 (8 significant bits); everything else is
fp32. tests/bf16_emu.py is the oracle's network with exactly those roundings, in
float64. Against it:

  - the 3-layer conv agent and the blind agent: the GPU reproduces the emulation to fp32
    accuracy (outputs within 1e-5, gradients within 1e-5 / 3e-4 relative L2), so any
    rounding added, dropped or moved in the contraction, FC, LSTM or head paths fails;
  - the GroupNorm ResNet-18: a deep stack of bf16 roundings is a chaotic function of
    fp32-level noise. Perturbing the emulation's parameters by one fp32 unit roundoff
    (2^-24, relative) moves its logits by ~2e-3 and its encoder gradients by up to ~0.3
    relative L2: every bf16 rounding an fp32 difference flips injects a 2^-9 jump, and
    after a few layers the roundings of two computations that differ at fp32 level are
    independent. No implementation can be closer to the emulation than that floor. The
    test measures the floor (the emulation against itself under 2^-24, 2^-23 and 2^-22
    perturbations) and bounds the GPU's distance to the emulation by 2.5 times it, with
    the gradients pooled over the encoder's tensors and over the others.
Against float64 the GPU must stay within twice the emulation's own distance (the cost of
the bf16 roundings) plus 1e-2.

Checked: evaluate + backward on small and full-width nets (logits, values and every
parameter tensor's gradient), and a whole ddppo_ppo_update (2 epochs x 2 minibatches of
T-step sequences: gather, replay, loss, BPTT, encoder backward, clip, Adam, captured
graph) against oracle.rl.ppo_update run through the emulation.
"""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from oracle import rl as OR
from paper_1911_00357_gb300 import binding as B
from tests import bf16_emu as EMU
from tests import inputs as I
from tests.test_gpu_policy import Net, _cfg, _dev_inputs, _rollout_tensors, _view

pytestmark = pytest.mark.gpu
DT = torch.float64

# non-chaotic nets (3-layer conv, blind): GPU vs emulation
TOL_OUT = 1e-5       # logits and values, relative to the tensor's largest magnitude
TOL_GRAD = 1e-5      # relative L2 of every non-encoder parameter gradient
TOL_GRAD_ENC = 3e-4  # relative L2 of every encoder parameter gradient
CHAOS_EPS = (2.0 ** -24, 2.0 ** -22)


def _rel(a, b):
    a = torch.as_tensor(a, dtype=DT)
    b = torch.as_tensor(b, dtype=DT)
    return ((a - b).abs().max() / max(b.abs().max().item(), 1e-6)).item()


def _rel_l2(a, b):
    nb = torch.linalg.vector_norm(b).item()
    return torch.linalg.vector_norm(a - b).item() / max(nb, 1e-12)


def _forward_grad(fwd, flat64, ref, ncfg, dl, dv):
    f = flat64.clone().requires_grad_(True)
    p = OP.unflatten(f, ncfg)
    lg, vv, _, _ = fwd(p, ref["obs"], ref["goal"], ref["prev_a"], ref["masks"], ref["h0"],
                       ref["c0"], ncfg)
    (g,) = torch.autograd.grad((lg * dl).sum() + (vv * dv).sum(), f)
    return lg.detach(), vv.detach(), g


def _per_tensor(ncfg, g):
    out, off = {}, 0
    for name, shp in OP.param_spec(ncfg):
        k = int(np.prod(shp))
        out[name] = g[off:off + k]
        off += k
    return out


ENC_PREFIX = ("c1.", "c2.", "c3.", "stem.", "b", "cmp.")
HEAD_PREFIX = ("vis", "goal", "act", "lstm", "actor", "critic")


@pytest.mark.parametrize("name,T,E,chunk", [("nature_small", 5, 3, 0), ("resnet_small", 4, 5, 0),
                                            ("nature_full", 3, 4, 0), ("resnet_full", 2, 3, 0),
                                            ("resnet_small", 4, 5, 6), ("blind_small", 5, 3, 0)])
def test_bf16_evaluate_backward_vs_emulation(name, T, E, chunk):
    cfg = _cfg(name, E, T, 1, encoder_chunk=chunk)
    net = Net(cfg, seed=1)
    try:
        mb = I.minibatch(net.ncfg, T=T, E=E, seed=2)
        dev, ref = _dev_inputs(cfg, mb)
        logits = torch.zeros(T, E, 4, device="cuda")
        values = torch.zeros(T, E, device="cuda")
        B.ddppo_policy_evaluate(net.h, T, E, dev["obs"], dev["goal"], dev["prev_a"], dev["masks"],
                                dev["h0"], dev["c0"], logits, values)
        g = torch.Generator().manual_seed(3)
        dl = torch.randn(T, E, 4, generator=g, dtype=DT).float()
        dv = torch.randn(T, E, generator=g, dtype=DT).float()
        grad = torch.zeros(net.P, device="cuda")
        B.ddppo_policy_backward(net.h, dl.cuda(), dv.cuda(), grad)
        torch.cuda.synchronize()
        assert B.ddppo_device_status(net.h) == 0
        f64 = net.flat64()
        lg_e, v_e, g_e = _forward_grad(EMU.sequence_forward, f64, ref, net.ncfg, dl.double(), dv.double())
        lg_r, v_r, g_r = _forward_grad(OP.sequence_forward, f64, ref, net.ncfg, dl.double(), dv.double())
        gg = grad.cpu().double()
        err = {"logits": _rel(logits.cpu(), lg_e), "values": _rel(values.cpu(), v_e)}
        cost = {"logits": _rel(lg_e, lg_r), "values": _rel(v_e, v_r)}
        gpu64 = {"logits": _rel(logits.cpu(), lg_r), "values": _rel(values.cpu(), v_r)}
        ge, gr, gp = _per_tensor(net.ncfg, g_e), _per_tensor(net.ncfg, g_r), _per_tensor(net.ncfg, gg)
        enc, rest = {}, {}
        for k in ge:
            if torch.linalg.vector_norm(ge[k]).item() < 1e-8:
                assert torch.linalg.vector_norm(gp[k]).item() < 1e-6, k
                continue
            e = _rel_l2(gp[k], ge[k])
            (rest if k.startswith(HEAD_PREFIX) else enc)[k] = e
            cost[k] = _rel_l2(ge[k], gr[k])
            gpu64[k] = _rel_l2(gp[k], gr[k])
        fmt = lambda d: {k: "%.2g" % v for k, v in d.items()}
        print("\n%s GPU vs emulation: out %s\n  encoder %s\n  rest %s" % (name, fmt(err), fmt(enc), fmt(rest)))
        print("  emulation vs float64 (bf16 cost): %s" % fmt(cost))
        if net.ncfg.net_kind == 1:
            # the chaos floor: the emulation against itself under fp32-level perturbations of
            # its parameters; the gradients compared pooled over the encoder's tensors and over
            # the others (a few ReLU decisions of a narrow layer make single tensors noisy)
            def pooled(g):
                gq = _per_tensor(net.ncfg, g)
                return (torch.cat([gq[k] for k in enc]) if enc else None,
                        torch.cat([gq[k] for k in rest]))
            pe, pr = pooled(g_e)
            pg_enc, pg_rest = pooled(gg)
            got = {"logits": err["logits"], "values": err["values"],
                   "encoder": _rel_l2(pg_enc, pe) if enc else 0.0, "rest": _rel_l2(pg_rest, pr)}
            floor = {k: 0.0 for k in got}
            for i, eps in enumerate(CHAOS_EPS + (2.0 ** -23,)):
                noise = torch.randn(f64.shape, generator=torch.Generator().manual_seed(40 + i), dtype=DT)
                lg_p, v_p, g_p = _forward_grad(EMU.sequence_forward, f64 * (1 + eps * noise), ref,
                                               net.ncfg, dl.double(), dv.double())
                qe, qr = pooled(g_p)
                cand = {"logits": _rel(lg_p, lg_e), "values": _rel(v_p, v_e),
                        "encoder": _rel_l2(qe, pe) if enc else 0.0, "rest": _rel_l2(qr, pr)}
                floor = {k: max(floor[k], cand[k]) for k in floor}
            print("  pooled GPU vs emulation: %s; chaos floor: %s" % (fmt(got), fmt(floor)))
            for k in got:
                assert got[k] <= 2.5 * floor[k] + 1e-4, (k, got[k], floor[k])
        else:
            assert err["logits"] <= TOL_OUT and err["values"] <= TOL_OUT, err
            worst = max(rest, key=rest.get)
            assert rest[worst] <= TOL_GRAD, (worst, rest[worst])
            if enc:
                worst = max(enc, key=enc.get)
                assert enc[worst] <= TOL_GRAD_ENC, (worst, enc[worst])
        for k in gpu64:
            assert gpu64[k] <= 2 * cost[k] + 1e-2, (k, gpu64[k], cost[k])
    finally:
        net.close()


@pytest.mark.parametrize("name,T,E", [("nature_small", 8, 4), ("resnet_small", 8, 4),
                                      ("resnet_full", 8, 4)])
def test_bf16_ppo_update_vs_emulation(name, T, E):
    """The whole BF16 update against oracle.rl.ppo_update through the emulation.
    3-layer conv agent: every parameter's change (Adam moves each coordinate by about lr
    per step) within 5% of lr x steps, the per-minibatch loss within 1e-4 of its
    magnitude, the gradient norm (before clipping) within 1e-3. ResNet agents (chaotic in
    BF16, see above): the parameter change vector, the losses and the gradient norms
    within 2.5 times the larger of the emulated update's chaos floor (its distance to the
    same update from parameters perturbed by 2^-24) and its distance to the float64
    update, plus a small absolute term."""
    mb = 2
    cfg = _cfg(name, E, T, 1, mb=mb)
    net = Net(cfg, seed=7)
    try:
        ro_t, ref = _rollout_tensors(cfg, net, T, E, seed=8)
        hpb = B.default_hparams(minibatches=mb, update_index=3)
        stats = torch.zeros(2 * mb, 8, device="cuda")
        B.ddppo_ppo_update(net.h, _view(ro_t), hpb, stats)
        out = torch.zeros(net.P, device="cuda")
        B.ddppo_get_params(net.h, out)
        step = B.ddppo_get_adam(net.h, torch.zeros(net.P, device="cuda"), torch.zeros(net.P, device="cuda"))
        torch.cuda.synchronize()
        assert B.ddppo_device_status(net.h) == 0
        hp = OR.PPOHParams(minibatches=mb)
        ro = {k: ref[k] for k in ("obs", "goal", "prev_a", "masks", "actions", "logp_old", "adv",
                                   "ret", "h0", "c0")}
        f0 = net.flat64()
        z = torch.zeros_like(f0)
        with EMU.in_oracle():
            f_e, _, _, st_e, sts_e = OR.ppo_update(f0, z, z.clone(), 0, ro, net.ncfg, hp,
                                                   seed=cfg.seed, update=3)
        f_r, _, _, _, sts_r = OR.ppo_update(f0, z, z.clone(), 0, ro, net.ncfg, hp, seed=cfg.seed,
                                            update=3)
        assert step == st_e == 2 * mb
        d_gpu, d_emu, d_64 = out.cpu().double() - f0, f_e - f0, f_r - f0
        unit = hp.lr * st_e
        e_par = (d_gpu - d_emu).abs().max().item() / unit
        c_par = (d_emu - d_64).abs().max().item() / unit
        e_l2 = _rel_l2(d_gpu, d_emu)
        c_l2 = _rel_l2(d_emu, d_64)
        s = stats.cpu().double()
        rl = lambda a, b: abs(a - b) / max(1.0, abs(b))
        e_loss = max(rl(s[k, 0].item(), st["loss"].item()) for k, st in enumerate(sts_e))
        c_loss = max(rl(a["loss"].item(), b["loss"].item()) for a, b in zip(sts_e, sts_r))
        e_gn = max(abs(s[k, 6].item() - st["grad_norm"].item()) / st["grad_norm"].item()
                   for k, st in enumerate(sts_e))
        c_gn = max(abs(a["grad_norm"].item() - b["grad_norm"].item()) / b["grad_norm"].item()
                   for a, b in zip(sts_e, sts_r))
        print("\n%s BF16 update vs emulation: param change max %.3g of lr*steps, rel L2 %.3g, loss "
              "%.2g, grad norm %.2g; emulation vs float64: max %.3g, rel L2 %.3g, loss %.2g, grad "
              "norm %.2g" % (name, e_par, e_l2, e_loss, e_gn, c_par, c_l2, c_loss, c_gn))
        if net.ncfg.net_kind == 1:
            # the update's chaos floor: the emulated update from parameters perturbed at fp32
            # level, against the unperturbed one
            noise = torch.randn(f0.shape, generator=torch.Generator().manual_seed(50), dtype=DT)
            with EMU.in_oracle():
                f_p, _, _, _, sts_p = OR.ppo_update(f0 * (1 + 2.0 ** -24 * noise), z, z.clone(), 0,
                                                    ro, net.ncfg, hp, seed=cfg.seed, update=3)
            p_l2 = _rel_l2(f_p - f0, d_emu)
            p_loss = max(rl(a["loss"].item(), b["loss"].item()) for a, b in zip(sts_p, sts_e))
            p_gn = max(abs(a["grad_norm"].item() - b["grad_norm"].item()) / b["grad_norm"].item()
                       for a, b in zip(sts_p, sts_e))
            print("  chaos floor of the emulated update: rel L2 %.3g, loss %.2g, grad norm %.2g"
                  % (p_l2, p_loss, p_gn))
            assert e_l2 <= 2.5 * max(p_l2, c_l2) + 1e-2, (e_l2, p_l2, c_l2)
            assert e_loss <= 2.5 * max(p_loss, c_loss) + 1e-4, (e_loss, p_loss, c_loss)
            assert e_gn <= 2.5 * max(p_gn, c_gn) + 1e-3, (e_gn, p_gn, c_gn)
        else:
            assert e_par <= 0.05, e_par
            assert e_loss <= 1e-4, e_loss
            assert e_gn <= 1e-3, e_gn
        # and against float64 itself: within twice the bf16 cost
        assert _rel_l2(d_gpu, d_64) <= 2 * c_l2 + 1e-2
    finally:
        net.close()
