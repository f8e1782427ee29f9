"""GPU parity of the transfer tasks (Sec. 5 "Transfer Learning": Flee and Exploration).

The CUDA env kernels compute the task rewards as the agent steps (task 1: the BFS field
from the episode's start and its maximum, computed when the episode is generated; task 2:
a bitmap of visited squares per env). The oracle computes them afterwards from the
trajectory: the oracle world is stepped with the same actions (motion is bit-exact, so
the trajectories coincide), each episode's positions are collected, and
oracle.sim.flee_rewards / explore_rewards give its rewards. Every reward must agree to
the last bit, over several episodes per env (auto-reset inside the step, the next
episode prepared on a side stream or generated in place), on Bernoulli and rooms worlds,
with fixed and mixed grid sizes.
"""
import numpy as np
import pytest
import torch

from oracle import sim as OS
from paper_1911_00357_gb300 import binding as B
from paper_1911_00357_gb300.presets import make_config
from tests import inputs as I
from tests.gpu_util import Env, sim_config_from

pytestmark = pytest.mark.gpu

WORLDS = {
    "bernoulli32": dict(preset="nature_fp32", num_envs=8),
    "rooms128": dict(preset="resnet", num_envs=6, precision=0),
    "rooms_mixed": dict(preset="mixed_1024", num_envs=6, precision=0),
}


@pytest.mark.parametrize("world", list(WORLDS))
@pytest.mark.parametrize("task", [1, 2])
@pytest.mark.parametrize("prefetch", [False, True])
def test_task_rewards_match_the_oracle(world, task, prefetch):
    d = dict(WORLDS[world])
    cfg = make_config(d.pop("preset"), task=task, **d)
    E = cfg.num_envs
    env = Env(cfg)
    try:
        env.reset()
        ref = OS.BatchSim(sim_config_from(cfg))
        ref.reset()
        cs = ref.cfg.cell_u
        stream = None
        if prefetch:
            stream = torch.cuda.Stream()
        # per env: the current episode's grid and positions (start first)
        grids = [ref.grid(e).copy() for e in range(E)]
        traj = [[tuple(ref.states[e, :2])] for e in range(E)]
        gpu_r = [[] for _ in range(E)]
        episodes = 0
        acts = I.random_actions(150, E, seed=7, p_stop=0.04)
        for t in range(acts.shape[0]):
            if prefetch:
                torch.cuda.current_stream().synchronize()
                B.ddppo_env_prefetch(env.h, stream)
                stream.synchronize()
            env.step(acts[t])
            torch.cuda.synchronize()
            r_gpu = env.reward.cpu().numpy()
            pre = ref.states.copy()
            _, done, _, _ = ref.step(acts[t])
            assert (env.done.cpu().numpy() == done).all()
            for e in range(E):
                gpu_r[e].append(r_gpu[e])
                if done[e]:
                    # stop (or the step cap after a move): the last position of the episode
                    if acts[t, e] == 0:
                        traj[e].append(tuple(pre[e, :2]))
                    else:  # ended by max_steps after this action: recompute its move
                        traj[e].append(tuple(_moved(grids[e], cs, pre[e], acts[t, e])))
                    _check_episode(task, grids[e], cs, traj[e], gpu_r[e], cfg.explore_m)
                    episodes += 1
                    grids[e] = ref.grid(e).copy()
                    traj[e] = [tuple(ref.states[e, :2])]
                    gpu_r[e] = []
                else:
                    traj[e].append(tuple(ref.states[e, :2]))
        for e in range(E):  # the unfinished episodes
            if gpu_r[e]:
                _check_episode(task, grids[e], cs, traj[e], gpu_r[e], cfg.explore_m)
        st = env.get_state()
        if task == 1:  # Flee keeps the geodesic from the start in the previous-geodesic slot
            st, want = np.delete(st, OS.S_GEO_PREV, 1), np.delete(ref.states, OS.S_GEO_PREV, 1)
        else:
            want = ref.states
        np.testing.assert_array_equal(st, want)
        assert episodes >= E // 2
        assert B.ddppo_device_status(env.h) == 0
    finally:
        env.close()


def _moved(grid, cs, st, a):
    """Position after action a from state st (the oracle's motion: forward blocked by the
    exact segment test, turns and stop stay)."""
    x, y = int(st[0]), int(st[1])
    if a != 1:
        return x, y
    f = OS.fwd_table()[int(st[OS.S_HEAD])]
    nx, ny = x + int(f[0]), y + int(f[1])
    return (x, y) if OS.segment_blocked(grid, cs, (x, y), (nx, ny)) else (nx, ny)


def _check_episode(task, grid, cs, traj, gpu_r, explore_m):
    xy = np.array(traj, np.int32)
    if task == 1:
        want = OS.flee_rewards(grid, cs, xy)
    else:
        want = OS.explore_rewards(xy, square_u=int(round(explore_m * 10000)))
    got = np.array(gpu_r, np.float32)
    assert got.shape == want.shape
    np.testing.assert_array_equal(got.view(np.uint32), want.view(np.uint32))
