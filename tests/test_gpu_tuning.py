"""The GEMM tuning cache: a table exported after the shapes of a rollout-and-update
iteration were tuned, imported into a second context of the same configuration, covers
every contraction that context launches (nothing is tuned again), survives a second
export byte for byte, and malformed images are rejected."""
import pytest
import torch

from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.worker import Worker

pytestmark = pytest.mark.gpu

SMALL = dict(num_envs=4, rollout_T=4, minibatches=1)


def test_tuning_cache_round_trip():
    w1 = Worker("resnet", seed=3, **SMALL)
    w2 = Worker("resnet", seed=3, **SMALL)
    try:
        w1.iterate()
        torch.cuda.synchronize()
        n1 = B.ddppo_autotune(w1.h, True)
        assert n1 > 0
        image = B.ddppo_autotune_export(w1.h)
        assert len(image) == 4 * (3 + 11 * n1)
        B.ddppo_autotune_import(w2.h, image)
        assert B.ddppo_autotune(w2.h, True) == n1
        w2.iterate()
        torch.cuda.synchronize()
        assert B.ddppo_autotune(w2.h, True) == n1   # every shape was already in the table
        assert B.ddppo_autotune_export(w2.h) == image
        assert B.ddppo_device_status(w2.h) == 0
        for bad in (b"", image[:-4], b"\0" * 12, image[:8] + b"\xff\xff\xff\xff" + image[12:]):
            with pytest.raises(RuntimeError):
                B.ddppo_autotune_import(w2.h, bad)
    finally:
        w1.close()
        w2.close()
