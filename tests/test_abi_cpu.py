"""CPU checks of the C ABI library: it loads without a GPU, exports every function
``include/ddppo.h`` declares, and rejects bad configurations before touching CUDA."""
import ctypes
import os
import re

import pytest

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.presets import PRESETS, make_config

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "ddppo.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|const char\*)\s+(ddppo_\w+)\s*\(", src)))


def test_header_declares_the_abi():
    names = _declared()
    for n in ("ddppo_create", "ddppo_env_reset", "ddppo_env_step", "ddppo_policy_act", "ddppo_gae",
              "ddppo_ppo_update"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = B.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_declared()) <= set(B.exported_symbols())


def test_bad_configs_are_rejected_before_cuda():
    bad = [dict(num_envs=0), dict(grid_min=48, grid_max=48), dict(grid_min=64, grid_max=32),
           dict(depth_h=64, depth_w=96), dict(precision=2), dict(num_envs=10, minibatches=3),
           dict(net_kind=5), dict(cam_h_m=3.0), dict(hidden=12)]
    for kw in bad:
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_create(make_config("nature_fp32", **kw))
        assert ei.value.code == -2, kw
    # FP8 inference needs the ResNet encoder at a base width that is a multiple of 64
    for name, kw in [("resnet", dict(precision=2)), ("resnet", dict(precision=3)),
                     ("blind", dict(precision=2)), ("resnet", dict(net_kind=5)),
                     ("resnet", dict(net_kind=3, base_ch=64)), ("resnet", dict(net_kind=4, base_ch=8)),
                     ("wide_256_fp8", dict(net_kind=3)), ("resnet", dict(task=3)),
                     ("resnet", dict(task=2, explore_m=0.05))]:
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_create(make_config(name, **kw))
        assert ei.value.code == -2, (name, kw)


def test_null_arguments_are_rejected():
    L = B.lib()
    assert L.ddppo_create(None, None) == -1
    assert L.ddppo_gae(None, None, None, 4, 4, ctypes.c_float(0.99), ctypes.c_float(0.95), None,
                       None, None) == -1
    assert L.ddppo_gae(None, None, None, 0, 4, ctypes.c_float(0.99), ctypes.c_float(0.95), None,
                       None, None) == 0
    assert L.ddppo_destroy(None) == 0
    assert isinstance(L.ddppo_last_error(), bytes)


def test_every_preset_passes_the_configuration_checks():
    for name in PRESETS:
        B.ddppo_config_check(make_config(name))
    for kind in (3, 4):  # the SE-ResNeXt encoders at the paper's halved widths
        B.ddppo_config_check(make_config("resnet", net_kind=kind, base_ch=32))
    for task in (1, 2):
        B.ddppo_config_check(make_config("resnet", task=task))
    with pytest.raises(B.DDPPOError) as ei:
        B.ddppo_config_check(make_config("wide_256_fp8", base_ch=32))
    assert ei.value.code == -2 and "fp8" in str(ei.value)


def test_presets_pass_validation_shapes():
    for name in PRESETS:
        cfg = make_config(name)
        assert cfg.num_envs % cfg.minibatches == 0
        assert cfg.grid_min % 32 == 0 and cfg.depth_w % 32 == 0
