"""The device-side failure path, made to run out without faulting or hanging the GPU.

The BFS of a reset has a capped level loop (Sec. 4 "Training": the geodesic distance
field). ddppo_set_bfs_level_cap lowers the cap to two levels, far fewer than any scene
needs, so every BFS of the reset runs out: the kernel sets the sticky E_TIMEOUT word,
leaves the unreached cells at -1 and returns; the reset then finds no start 2 m away and
parks the agents. Nothing asynchronous is in flight during that loop. The test checks
the status that the host reads, that the launch completed (the stream synchronises),
and that the context stays usable: a fresh worker in the same process steps bit-exactly
against the oracle. A cap larger than any BFS needs changes nothing.
"""
import numpy as np
import pytest
import torch

from oracle import sim as OS
from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.presets import make_config
from tests.gpu_util import Env, sim_config_from

pytestmark = pytest.mark.gpu

E_TIMEOUT = -5


def _steps_match_oracle(cfg, n_steps=12, seed=3):
    env = Env(cfg)
    try:
        env.reset()
        ref = OS.BatchSim(sim_config_from(cfg))
        ref.reset()
        rng = np.random.default_rng(seed)
        for _ in range(n_steps):
            a = rng.integers(0, 4, size=cfg.num_envs).astype(np.int32)
            env.step(a)
            r, d, _, _ = ref.step(a)
            torch.cuda.synchronize()
            assert (env.reward.cpu().numpy() == r).all() and (env.done.cpu().numpy() == d).all()
        np.testing.assert_array_equal(env.get_state(), ref.states)
        return B.ddppo_device_status(env.h)
    finally:
        env.close()


def test_bfs_level_cap_runs_out_and_reports_timeout():
    cfg = make_config("nature_fp32", num_envs=4)
    env = Env(cfg)
    try:
        B.ddppo_set_bfs_level_cap(env.h, 2)
        env.reset()
        torch.cuda.synchronize()  # the launch completed: nothing hangs
        assert B.ddppo_device_status(env.h) == E_TIMEOUT
        # the fields hold only the cells within two steps of the goal
        grids, dists = env.get_grids()
        st = env.get_state()
        for e in range(cfg.num_envs):
            g = int(st[e, OS.S_GRID])
            d = dists[e, :g * g]
            assert d.max() <= 2
    finally:
        env.close()
    # the context is still usable: a new worker steps bit-exactly with a clean status
    assert _steps_match_oracle(make_config("nature_fp32", num_envs=4)) == 0


def test_bfs_level_cap_above_need_changes_nothing():
    cfg = make_config("nature_fp32", num_envs=6)
    env = Env(cfg)
    try:
        B.ddppo_set_bfs_level_cap(env.h, cfg.grid_max * cfg.grid_max)  # G levels: always enough
        env.reset()
        ref = OS.BatchSim(sim_config_from(cfg))
        ref.reset()
        np.testing.assert_array_equal(env.get_state(), ref.states)
        _, dists = env.get_grids()
        for e in range(cfg.num_envs):
            np.testing.assert_array_equal(
                dists[e, :ref.dist(e).size].reshape(ref.dist(e).shape), ref.dist(e))
        assert B.ddppo_device_status(env.h) == 0
    finally:
        env.close()


def test_bfs_level_cap_rejects_negative():
    cfg = make_config("nature_fp32", num_envs=2)
    h = B.ddppo_create(cfg)
    try:
        with pytest.raises(B.DDPPOError) as ei:
            B.ddppo_set_bfs_level_cap(h, -1)
        assert ei.value.code == -1
    finally:
        B.ddppo_destroy(h)
