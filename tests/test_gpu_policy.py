"""GPU parity of the agent network and the learning step against the float64 oracle.

FP32 form: logits/values within 1e-4 (relative to the tensor's scale) of the float64
forward; every gradient tensor within 1e-3 relative L2 of float64 autograd, except the
encoder of the full-width ResNet (3e-2): its gradient passes through ReLU masks and
max-pool argmax choices that flip under any float32 rounding (a plain float32 PyTorch
evaluation of the same network differs from float64 by 1.4e-2 there). The PPO loss and
its logit/value gradients: within 1e-5 relative.

BF16 form (bf16 GEMM operands, fp32 accumulation and everything else fp32): logits and
values within 5e-2; gradients of non-encoder tensors within 0.25 relative L2; encoder
gradients within 0.1 (3-layer conv) and, for the GroupNorm ResNet, max 0.8 / median 0.45
relative L2. For comparison a plain bfloat16 PyTorch evaluation of the same networks
measures 0.047 (3-layer conv) and max 0.62-0.79 / median 0.39 (ResNet) against float64.
"""
import numpy as np
import pytest
import torch

from oracle import policy as OP
from oracle import rl as OR
from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.presets import make_config
from tests import inputs as I
from tests.gpu_util import net_config_from, obs_dtype

pytestmark = pytest.mark.gpu
DT = torch.float64

NETS = {
    # small nets (few-tile GEMMs, ragged tails) and the full-size encoders
    "nature_small": dict(preset="nature_fp32", hidden=16, lstm_layers=2),
    # 128x128 input keeps the last feature map at 4x4, as in the full encoder: GroupNorm
    # over 2-element groups (a 1x1 map) is ill-conditioned and makes a poor parity case
    "resnet_small": dict(preset="resnet", base_ch=8, hidden=16, lstm_layers=2, depth_h=128,
                         depth_w=128, pool2x2=0),
    "nature_full": dict(preset="nature_fp32"),
    "resnet_full": dict(preset="resnet"),
    # the blind agent (GPS+Compass only): no encoder, no visual FC
    "blind_small": dict(preset="nature_fp32", net_kind=2, hidden=16, lstm_layers=2),
    "blind_full": dict(preset="resnet", net_kind=2),
}


def _cfg(name, E, T, precision, mb=1, **kw):
    d = dict(NETS[name])
    d.update(kw)
    pre = d.pop("preset")
    return make_config(pre, num_envs=E, rollout_T=T, minibatches=mb, precision=precision, **d)


class Net:
    def __init__(self, cfg, seed=0):
        self.cfg = cfg
        self.h = B.ddppo_create(cfg)
        self.ncfg = net_config_from(cfg)
        self.P = B.ddppo_num_params(self.h)
        assert self.P == OP.num_params(self.ncfg)
        self.flat32 = I.params(self.ncfg, seed).float()
        B.ddppo_set_params(self.h, self.flat32.cuda())

    def close(self):
        B.ddppo_destroy(self.h)

    def flat64(self):
        return self.flat32.double()


def _dev_inputs(cfg, mb):
    """Cast the seeded float64 inputs to what the kernels read; return (device, oracle)."""
    od = obs_dtype(cfg)
    dev = {
        "obs": mb["obs"].to(od).cuda().contiguous(),
        "goal": mb["goal"].float().cuda(),
        "prev_a": mb["prev_a"].int().cuda(),
        "masks": mb["masks"].cuda(),
        "h0": mb["h0"].float().cuda(),
        "c0": mb["c0"].float().cuda(),
    }
    ref = {
        "obs": dev["obs"].cpu().double(),
        "goal": dev["goal"].cpu().double(),
        "prev_a": mb["prev_a"],
        "masks": mb["masks"],
        "h0": dev["h0"].cpu().double(),
        "c0": dev["c0"].cpu().double(),
    }
    return dev, ref


def _rel_close(a, b, rtol, name=""):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.abs(b).max(), 1e-6)
    err = np.abs(a - b).max() / scale
    assert err <= rtol, "%s: max err %.3g of scale %.3g > %.3g" % (name, err, scale, rtol)
    return err


@pytest.mark.parametrize("name,T,E,chunk", [("nature_small", 5, 3, 0), ("resnet_small", 4, 5, 0),
                                            ("nature_full", 3, 4, 0), ("resnet_full", 2, 3, 0),
                                            ("resnet_small", 4, 5, 6), ("nature_small", 5, 3, 4),
                                            ("blind_small", 5, 3, 0), ("blind_full", 4, 6, 0)])
@pytest.mark.parametrize("precision", [0, 1])
def test_evaluate_and_backward_parity(name, T, E, chunk, precision):
    """chunk > 0 runs the encoder in chunks of that many frames (ragged last chunk); the
    backward then recomputes every chunk but the last before back-propagating it."""
    cfg = _cfg(name, E, T, precision, encoder_chunk=chunk)
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
        # oracle
        flat = net.flat64().clone().requires_grad_(True)
        p = OP.unflatten(flat, net.ncfg)
        lg, vv, _, _ = OP.sequence_forward(p, ref["obs"], ref["goal"], ref["prev_a"], ref["masks"],
                                           ref["h0"], ref["c0"], net.ncfg)
        (g_ref,) = torch.autograd.grad((lg * dl.double()).sum() + (vv * dv.double()).sum(), flat)
        tol_f = 1e-4 if precision == 0 else 5e-2
        _rel_close(logits.cpu(), lg.detach(), tol_f, "logits")
        _rel_close(values.cpu(), vv.detach(), tol_f, "values")
        gg = grad.cpu().double()
        off = 0
        errs = {}
        for pname, shp in OP.param_spec(net.ncfg):
            k = int(np.prod(shp))
            a, b = gg[off:off + k], g_ref[off:off + k]
            off += k
            nb = torch.linalg.vector_norm(b).item()
            if nb < 1e-8:
                assert torch.linalg.vector_norm(a).item() < 1e-6, pname
                continue
            errs[pname] = torch.linalg.vector_norm(a - b).item() / nb
        print("gradient relative L2 errors (precision %d):" % precision,
              {k: "%.2g" % v for k, v in errs.items()})
        head = ("vis", "goal", "act", "lstm", "actor", "critic")
        enc = {k: v for k, v in errs.items() if not k.startswith(head)}
        rest = {k: v for k, v in errs.items() if k.startswith(head)}
        resnet = net.ncfg.net_kind == 1
        if precision == 0:
            tol_enc = 3e-2 if (resnet and name == "resnet_full") else 1e-3
            tol_rest, tol_med = 1e-3, 1.0
        else:
            tol_enc, tol_med = (0.8, 0.45) if resnet else (0.1, 1.0)
            tol_rest = 0.25
        if enc:  # the blind agent has no encoder
            worst = max(enc, key=enc.get)
            assert enc[worst] <= tol_enc, "%s: relative L2 error %.3g > %.3g" % (worst, enc[worst], tol_enc)
            assert np.median(list(enc.values())) <= tol_med
        worst = max(rest, key=rest.get)
        assert rest[worst] <= tol_rest, "%s: relative L2 error %.3g > %.3g" % (worst, rest[worst], tol_rest)
    finally:
        net.close()


@pytest.mark.parametrize("name,E", [("nature_small", 7), ("resnet_full", 6), ("blind_small", 7),
                                    ("blind_full", 6)])
@pytest.mark.parametrize("precision", [0, 1])
def test_act_parity(name, E, precision):
    cfg = _cfg(name, E, 4, precision)
    net = Net(cfg, seed=4)
    try:
        mb = I.minibatch(net.ncfg, T=1, E=E, seed=5)
        dev, ref = _dev_inputs(cfg, mb)
        u = torch.from_numpy(I.uniforms(1, E, seed=6)[0]).cuda()
        h = dev["h0"].clone()
        c = dev["c0"].clone()
        act = torch.zeros(E, dtype=torch.int32, device="cuda")
        logp = torch.zeros(E, device="cuda")
        val = torch.zeros(E, device="cuda")
        B.ddppo_policy_act(net.h, dev["obs"][0], dev["goal"][0], dev["prev_a"][0], dev["masks"][0], h,
                           c, u, act, logp, val)
        torch.cuda.synchronize()
        p = OP.unflatten(net.flat64(), net.ncfg)
        a_r, lp_r, v_r, h_r, c_r, lg_r = OP.act(p, ref["obs"][0], ref["goal"][0], ref["prev_a"][0],
                                                ref["masks"][0], ref["h0"], ref["c0"],
                                                u.cpu().double(), net.ncfg)
        tol = 1e-4 if precision == 0 else 5e-2
        cdf = torch.cumsum(torch.softmax(lg_r, -1), -1)
        decided = ((cdf - u.cpu().double().unsqueeze(1)).abs() > (1e-4 if precision == 0 else 3e-2)).all(1)
        assert (act.cpu().long()[decided] == a_r[decided]).all()
        assert decided.float().mean() > 0.5
        lp_g = logp.cpu().double()
        lp_at = torch.log_softmax(lg_r, -1).gather(1, act.cpu().long().unsqueeze(1))[:, 0]
        _rel_close(lp_g, lp_at, tol, "logp")
        _rel_close(val.cpu(), v_r, tol, "value")
        _rel_close(h.cpu(), h_r, tol, "h")
        _rel_close(c.cpu(), c_r, tol, "c")
    finally:
        net.close()


@pytest.mark.parametrize("n", [1, 37, 256, 4097])
def test_ppo_loss_parity(n):
    g = torch.Generator().manual_seed(n)
    logits = torch.randn(n, 4, generator=g, dtype=DT).float()
    values = torch.randn(n, generator=g, dtype=DT).float()
    actions = torch.randint(0, 4, (n,), generator=g, dtype=torch.int32)
    lp_now = torch.log_softmax(logits.double(), -1).gather(1, actions.long().unsqueeze(1))[:, 0]
    logp_old = (lp_now + 0.3 * torch.randn(n, generator=g, dtype=DT)).float()
    adv = torch.randn(n, generator=g, dtype=DT).float()
    ret = torch.randn(n, generator=g, dtype=DT).float()
    hp = OR.PPOHParams()
    stats = torch.zeros(8, device="cuda")
    dl = torch.zeros(n, 4, device="cuda")
    dv = torch.zeros(n, device="cuda")
    B.ddppo_ppo_loss(n, logits.cuda(), values.cuda(), actions.cuda(), logp_old.cuda(), adv.cuda(),
                     ret.cuda(), hp.clip, hp.value_coef, hp.entropy_coef, stats, dl, dv)
    torch.cuda.synchronize()
    L = logits.double().requires_grad_(True)
    V = values.double().requires_grad_(True)
    loss, st = OR.ppo_loss(L, V, actions, logp_old.double(), adv.double(), ret.double(), hp)
    gl, gv = torch.autograd.grad(loss, (L, V))
    s = stats.cpu().double()
    for i, key in enumerate(["loss", "policy_loss", "value_loss", "entropy", "clip_frac", "approx_kl"]):
        ref = st[key].item()
        assert abs(s[i].item() - ref) <= 1e-5 * max(1.0, abs(ref)), (key, s[i].item(), ref)
    _rel_close(dl.cpu(), gl, 1e-5, "dlogits")
    _rel_close(dv.cpu(), gv, 1e-5, "dvalues")


def _rollout_tensors(cfg, net, T, E, seed):
    mb = I.minibatch(net.ncfg, T=T, E=E, seed=seed)
    dev, ref = _dev_inputs(cfg, mb)
    od = obs_dtype(cfg)
    ro_t = {
        "obs": torch.zeros((T + 1, E, 1, net.ncfg.in_h, net.ncfg.in_w), dtype=od, device="cuda"),
        "goal": torch.zeros(T + 1, E, 3, device="cuda"),
        "prev_a": torch.zeros(T + 1, E, dtype=torch.int32, device="cuda"),
        "masks": torch.zeros(T + 1, E, dtype=torch.uint8, device="cuda"),
    }
    ro_t["obs"][:T] = dev["obs"]
    ro_t["goal"][:T] = dev["goal"]
    ro_t["prev_a"][:T] = dev["prev_a"]
    ro_t["masks"][:T] = dev["masks"]
    ro_t["actions"] = mb["actions"].int().cuda()
    ro_t["logp"] = mb["logp_old"].float().cuda()
    ro_t["adv"] = mb["adv"].float().cuda()
    ro_t["ret"] = mb["ret"].float().cuda()
    ro_t["h0"] = dev["h0"]
    ro_t["c0"] = dev["c0"]
    ref["actions"] = mb["actions"]
    ref["logp_old"] = ro_t["logp"].cpu().double()
    ref["adv"] = ro_t["adv"].cpu().double()
    ref["ret"] = ro_t["ret"].cpu().double()
    return ro_t, ref


def _view(ro_t):
    ro = B.Rollout()
    for k, v in ro_t.items():
        setattr(ro, k, v.data_ptr())
    return ro


@pytest.mark.parametrize("name,T,E,mb", [("nature_small", 6, 4, 2), ("resnet_small", 4, 4, 2)])
@pytest.mark.parametrize("norm_adv", [0, 1])
def test_ppo_update_parity(name, T, E, mb, norm_adv):
    cfg = _cfg(name, E, T, 0, mb=mb)
    net = Net(cfg, seed=7)
    try:
        ro_t, ref = _rollout_tensors(cfg, net, T, E, seed=8)
        hpb = B.default_hparams(minibatches=mb, norm_adv=norm_adv, update_index=3)
        stats = torch.zeros(2 * mb, 8, device="cuda")
        B.ddppo_ppo_update(net.h, _view(ro_t), hpb, stats)
        out = torch.zeros(net.P, device="cuda")
        B.ddppo_get_params(net.h, out)
        m = torch.zeros(net.P, device="cuda")
        step = B.ddppo_get_adam(net.h, m, torch.zeros(net.P, device="cuda"))
        torch.cuda.synchronize()
        hp = OR.PPOHParams(minibatches=mb, norm_adv=bool(norm_adv))
        ro = {k: ref[k] for k in ("obs", "goal", "prev_a", "masks", "actions", "logp_old", "adv",
                                   "ret", "h0", "c0")}
        f0 = net.flat64()
        f2, m2, v2, st2, sts = OR.ppo_update(f0, torch.zeros_like(f0), torch.zeros_like(f0), 0, ro,
                                             net.ncfg, hp, seed=cfg.seed, update=3)
        assert step == st2 == 2 * mb
        d_gpu = out.cpu().double() - f0
        d_ref = f2 - f0
        # Adam steps are ~lr per coordinate; compare the parameter change
        err = (d_gpu - d_ref).abs().max().item()
        assert err <= 0.02 * hp.lr * st2, err
        s = stats.cpu().double()
        for k, stt in enumerate(sts):
            assert abs(s[k, 0].item() - stt["loss"].item()) <= 1e-4 * max(1.0, abs(stt["loss"].item()))
            assert abs(s[k, 6].item() - stt["grad_norm"].item()) <= 1e-3 * stt["grad_norm"].item()
    finally:
        net.close()


@pytest.mark.parametrize("use_graph", [True, False])
def test_collect_matches_env_semantics(use_graph):
    """The collected rollout is a valid trajectory: re-stepping the oracle world with the
    collected actions reproduces rewards and dones bit-exactly; the policy outputs match
    an evaluate over the same segment; the bootstrap value matches an act on slot T."""
    from oracle import sim as OS
    from tests.gpu_util import sim_config_from
    E, T = 8, 12
    cfg = make_config("nature_fp32", num_envs=E, rollout_T=T, minibatches=1, hidden=32, max_steps=9)
    net = Net(cfg, seed=9)
    try:
        od = obs_dtype(cfg)
        L, Hd = cfg.lstm_layers, cfg.hidden
        ro_t = {
            "obs": torch.zeros(T + 1, E, 1, 64, 64, dtype=od, device="cuda"),
            "goal": torch.zeros(T + 1, E, 3, device="cuda"),
            "prev_a": torch.zeros(T + 1, E, dtype=torch.int32, device="cuda"),
            "masks": torch.zeros(T + 1, E, dtype=torch.uint8, device="cuda"),
            "actions": torch.zeros(T, E, dtype=torch.int32, device="cuda"),
            "logp": torch.zeros(T, E, device="cuda"),
            "values": torch.zeros(T + 1, E, device="cuda"),
            "rewards": torch.zeros(T, E, device="cuda"),
            "dones": torch.zeros(T, E, dtype=torch.uint8, device="cuda"),
            "info": torch.zeros(T, E, 4, device="cuda"),
            "adv": torch.zeros(T, E, device="cuda"),
            "ret": torch.zeros(T, E, device="cuda"),
            "h0": torch.zeros(L, E, Hd, device="cuda"),
            "c0": torch.zeros(L, E, Hd, device="cuda"),
            "h": torch.zeros(L, E, Hd, device="cuda"),
            "c": torch.zeros(L, E, Hd, device="cuda"),
            "uniforms": torch.from_numpy(I.uniforms(T, E, seed=10)).cuda(),
        }
        view = _view(ro_t)
        sim = OS.BatchSim(sim_config_from(cfg))
        sim.reset()
        for it in range(2):
            B.ddppo_collect(net.h, view, use_graph)
            torch.cuda.synchronize()
            acts = ro_t["actions"].cpu().numpy()
            for t in range(T):
                r, d, _, _ = sim.step(acts[t])
                assert (ro_t["rewards"][t].cpu().numpy() == r).all()
                assert (ro_t["dones"][t].cpu().numpy() == d).all()
            # prev_a / masks bookkeeping
            dn = ro_t["dones"].cpu().numpy()
            pa = ro_t["prev_a"].cpu().numpy()
            mk = ro_t["masks"].cpu().numpy()
            for t in range(T):
                assert (mk[t + 1] == 1 - dn[t]).all()
                assert (pa[t + 1] == np.where(dn[t] == 1, 4, acts[t])).all()
            # the policy's outputs are those of an evaluate over the whole segment
            lg = torch.zeros(T, E, 4, device="cuda")
            vv = torch.zeros(T, E, device="cuda")
            B.ddppo_policy_evaluate(net.h, T, E, ro_t["obs"][:T].contiguous(), ro_t["goal"][:T].contiguous(),
                                    ro_t["prev_a"][:T].contiguous(), ro_t["masks"][:T].contiguous(),
                                    ro_t["h0"], ro_t["c0"], lg, vv)
            lp = torch.log_softmax(lg, -1).gather(2, ro_t["actions"].long().unsqueeze(2))[..., 0]
            torch.cuda.synchronize()
            assert torch.allclose(vv, ro_t["values"][:T], atol=1e-5, rtol=1e-5)
            assert torch.allclose(lp, ro_t["logp"], atol=1e-5, rtol=1e-5)
        assert B.ddppo_device_status(net.h) == 0
    finally:
        net.close()
