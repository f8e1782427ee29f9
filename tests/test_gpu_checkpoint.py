"""Checkpoint and resume (ddppo_save / ddppo_load) through the C ABI.

A worker runs two iterations, saves, and runs two more. A second worker of the same
configuration, in the same process but with its own context, loads the checkpoint and
runs the same two iterations. Everything must agree bit for bit: the FP32 parameters and
both Adam moments, the agent states (integers), the collected rewards and actions of the
last rollout, and the LSTM state. Covered: the FP32 3-layer conv agent, the BF16
ResNet agent (autotuned GEMMs: the tuning table travels in the checkpoint) and FP8
inference (its delayed activation scales travel too). Also: a checkpoint of another
configuration, a truncated file and a missing rollout view are rejected.
"""
import os

import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker

pytestmark = pytest.mark.gpu

CASES = {
    "nature_fp32": dict(num_envs=6, rollout_T=8, minibatches=2, max_steps=12),
    "resnet": dict(num_envs=4, rollout_T=8, minibatches=2, max_steps=10),
    "wide_256_fp8": dict(num_envs=4, rollout_T=6, minibatches=2, encoder_chunk=0, max_steps=9),
}


def _snapshot(w):
    P = B.ddppo_num_params(w.h)
    p = torch.zeros(P, device="cuda")
    m = torch.zeros(P, device="cuda")
    v = torch.zeros(P, device="cuda")
    B.ddppo_get_params(w.h, p)
    step = B.ddppo_get_adam(w.h, m, v)
    st = torch.zeros(w.E, B.NSTATE, dtype=torch.int32, device="cuda")
    B.ddppo_env_state(w.h, st)
    torch.cuda.synchronize()
    out = {"params": p.cpu(), "m": m.cpu(), "v": v.cpu(), "state": st.cpu(), "step": step}
    for k in ("rewards", "actions", "dones", "logp", "values", "h", "c", "adv"):
        out[k] = w.t[k].cpu().clone()
    return out


@pytest.mark.parametrize("preset", list(CASES))
def test_resumed_run_is_bit_identical(preset, tmp_path):
    path = str(tmp_path / "ckpt.bin")
    a = Worker(preset, seed=3, **CASES[preset])
    try:
        for _ in range(2):
            a.iterate()
        a.save(path)
        for _ in range(2):
            a.iterate()
        want = _snapshot(a)
        assert B.ddppo_device_status(a.h) == 0
    finally:
        a.close()
    b = Worker(preset, seed=3, **CASES[preset])
    try:
        b.load(path)
        for _ in range(2):
            b.iterate()
        got = _snapshot(b)
        assert B.ddppo_device_status(b.h) == 0
    finally:
        b.close()
    assert got["step"] == want["step"]
    for k in want:
        if k == "step":
            continue
        assert torch.equal(got[k].view(torch.uint8), want[k].view(torch.uint8)), k


def test_load_rejects_other_configuration_and_truncated_files(tmp_path):
    path = str(tmp_path / "ckpt.bin")
    a = Worker("nature_fp32", seed=1, num_envs=4, rollout_T=4, minibatches=2)
    try:
        a.iterate()
        a.save(path)
    finally:
        a.close()
    other = Worker("nature_fp32", seed=2, num_envs=4, rollout_T=4, minibatches=2)
    try:
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_load(other.h, path, other.view)
        assert ei.value.code == -2 and "configuration" in str(ei.value)
    finally:
        other.close()
    same = Worker("nature_fp32", seed=1, num_envs=4, rollout_T=4, minibatches=2)
    try:
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_load(same.h, path)  # written with rollout state: the view is required
        assert ei.value.code == -1
        cut = str(tmp_path / "cut.bin")
        with open(path, "rb") as f:
            data = f.read()
        with open(cut, "wb") as f:
            f.write(data[: len(data) // 2])
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_load(same.h, cut, same.view)
        assert ei.value.code == -2
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_load(same.h, str(tmp_path / "missing.bin"), same.view)
        assert ei.value.code == -1
        # the complete file still loads
        B.ddppo_load(same.h, path, same.view)
        same.iterate()
        assert B.ddppo_device_status(same.h) == 0
    finally:
        same.close()
    assert os.path.getsize(path) > 0
