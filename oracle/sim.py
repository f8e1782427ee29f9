"""ctypes wrapper of the C simulator oracle (``sim_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU baseline). Each function
states the passage of arXiv:1911.00357 it follows; the readings taken where
the paper is silent are listed in the header comment of ``sim_oracle.c``.

Pins (tests/test_oracle_sim.py unless noted):
  counter_hash / splitmix64  SplitMix64's published outputs for state 0
  fwd_table           closed forms at 0/30/60/90/180/270 deg, symmetries, length 2500 +- 1
  gen_scene           border walls, Bernoulli density within 4 sigma, density 0 and 1,
                      rooms connected with one-cell walls
  bfs                 scipy Dijkstra, Floyd-Warshall on small grids, Manhattan on an empty grid
  segment_blocked     exact rational Liang-Barsky clipping (Python fractions)
  BatchSim.step       the hand-worked episode tests/golden/walk_9x9.txt (both terminal modes),
                      SPL special cases, timeouts, motion invariants
  render_depth / column_twall  empty-room closed forms (walls, floor, ceiling), a single
                      wall cell, the clip at max_depth
  goal_vector         3-4-5 triangle at two headings
  flee_rewards / explore_rewards  empty-room closed forms, a networkx BFS around a wall
                      gap, a straight walk's new squares
  env_permutation     is a permutation; uniform over the 3! orders (chi-square,
                      tests/test_oracle_pins_loss.py)
  pool_obs            constant image, checkerboard, non-square ramp, odd values
                      (tests/test_oracle_pins_loss.py)
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np

from . import build as _build

S_X, S_Y, S_HEAD, S_STEPS, S_PATH, S_GEO_PREV, S_GEO_START, S_GOAL_X, S_GOAL_Y, \
    S_EPISODE, S_GRID, S_COLLIDED = range(12)
NSTATE = 12


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("gen_kind", ctypes.c_int32), ("grid_min", ctypes.c_int32),
        ("grid_max", ctypes.c_int32), ("cell_u", ctypes.c_int32),
        ("wall_density", ctypes.c_double), ("door_cells", ctypes.c_int32),
        ("min_room", ctypes.c_int32), ("max_steps", ctypes.c_int32),
        ("terminal_mode", ctypes.c_int32), ("depth_h", ctypes.c_int32),
        ("depth_w", ctypes.c_int32), ("cam_h_m", ctypes.c_double),
        ("ceil_h_m", ctypes.c_double), ("max_depth_m", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


@dataclasses.dataclass
class SimConfig:
    """World parameters (Sec. 4). ``cell_m`` is converted to whole 1e-4 m units."""
    num_envs: int = 16
    gen_kind: int = 0            # 0 Bernoulli walls, 1 rooms and doors
    grid_min: int = 32
    grid_max: int = 32
    cell_m: float = 0.25
    wall_density: float = 0.15
    door_m: float = 0.8
    min_room: int = 8
    max_steps: int = 500
    terminal_mode: int = 0       # 0: +2.5 on success, 1: +2.5*SPL (Sec. 4 "Training")
    depth_h: int = 64
    depth_w: int = 64
    cam_h_m: float = 0.88
    ceil_h_m: float = 2.5
    max_depth_m: float = 10.0
    seed: int = 0

    @property
    def cell_u(self) -> int:
        return int(round(self.cell_m * 10000))

    @property
    def door_cells(self) -> int:
        return max(1, int(round(self.door_m / self.cell_m)))

    def c_struct(self) -> _Cfg:
        return _Cfg(self.gen_kind, self.grid_min, self.grid_max, self.cell_u,
                    float(self.wall_density), self.door_cells, self.min_room,
                    self.max_steps, self.terminal_mode, self.depth_h, self.depth_w,
                    float(self.cam_h_m), float(self.ceil_h_m), float(self.max_depth_m),
                    ctypes.c_uint64(self.seed & (2**64 - 1)))


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        L = _lib
        P = ctypes.c_void_p
        L.orc_hash.restype = ctypes.c_uint64
        L.orc_hash.argtypes = [ctypes.c_uint64] * 3 + [ctypes.c_uint32, ctypes.c_uint64]
        L.orc_sm64.restype = ctypes.c_uint64
        L.orc_sm64.argtypes = [ctypes.c_uint64]
        L.orc_fwd_table.argtypes = [P]
        L.orc_grid_side.restype = ctypes.c_int32
        L.orc_grid_side.argtypes = [P, ctypes.c_int64, ctypes.c_int64]
        L.orc_gen_scene.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P]
        L.orc_bfs.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
        L.orc_reset_env.argtypes = [P, ctypes.c_int64, ctypes.c_int64, P, P, P]
        L.orc_segment_blocked.argtypes = [P, ctypes.c_int, ctypes.c_int] + [ctypes.c_int32] * 4
        L.orc_step_env.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int32, P, P, P, P]
        L.orc_goal_vector.argtypes = [P, P]
        L.orc_column_twall.restype = ctypes.c_double
        L.orc_column_twall.argtypes = [P, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 4
        L.orc_render_depth.argtypes = [P, P, P, P]
        L.orc_env_permutation.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int, P]
        L.orc_batch_reset.argtypes = [P, ctypes.c_int, P, P, P]
        L.orc_batch_step.argtypes = [P, ctypes.c_int, P, P, P, P, P, P, P, P]
        L.orc_batch_render.argtypes = [P, ctypes.c_int, P, P, P, P]
        L.orc_flee_rewards.argtypes = [P, ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P]
        L.orc_explore_rewards.argtypes = [P, ctypes.c_int, ctypes.c_int, P]
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def counter_hash(seed: int, env: int, episode: int, stream: int, index: int) -> int:
    """SplitMix64-based counter hash that every random draw of the world uses."""
    return int(lib().orc_hash(seed, env, episode, stream, index))


def splitmix64(z: int) -> int:
    """The SplitMix64 output function applied to state z (one step from z)."""
    return int(lib().orc_sm64(z & (2**64 - 1)))


def fwd_table() -> np.ndarray:
    """Forward displacement per heading, int [36, 2] in 1e-4 m (Sec. 4 "Agent": 0.25 m)."""
    out = np.zeros((36, 2), np.int32)
    lib().orc_fwd_table(_p(out))
    return out


def grid_side(cfg: SimConfig, env: int, episode: int) -> int:
    c = cfg.c_struct()
    return int(lib().orc_grid_side(ctypes.byref(c), env, episode))


def gen_scene(cfg: SimConfig, env: int, episode: int, g: int | None = None) -> np.ndarray:
    """Occupancy grid [g, g] uint8 (1 = wall) standing in for a Habitat scene (Sec. 4)."""
    c = cfg.c_struct()
    if g is None:
        g = grid_side(cfg, env, episode)
    grid = np.zeros((g, g), np.uint8)
    rc = lib().orc_gen_scene(ctypes.byref(c), env, episode, g, _p(grid))
    if rc != 0:
        raise RuntimeError("scene generation failed")
    return grid


def bfs(grid: np.ndarray, gx: int, gy: int) -> np.ndarray:
    """Geodesic distance field in cells from (gx, gy); -1 = unreachable (Sec. 4 "Training")."""
    grid = np.ascontiguousarray(grid, np.uint8)
    g = grid.shape[0]
    assert grid.shape == (g, g)
    dist = np.zeros((g, g), np.int32)
    if lib().orc_bfs(_p(grid), g, gx, gy, _p(dist)) != 0:
        raise MemoryError
    return dist


def segment_blocked(grid: np.ndarray, cell_u: int, p0, p1) -> bool:
    grid = np.ascontiguousarray(grid, np.uint8)
    return bool(lib().orc_segment_blocked(_p(grid), grid.shape[0], cell_u,
                                          int(p0[0]), int(p0[1]), int(p1[0]), int(p1[1])))


def column_twall(grid: np.ndarray, cell_u: int, px: float, py: float, dx: float, dy: float) -> float:
    grid = np.ascontiguousarray(grid, np.uint8)
    return float(lib().orc_column_twall(_p(grid), grid.shape[0], cell_u, px, py, dx, dy))


def render_depth(cfg: SimConfig, grid: np.ndarray, state: np.ndarray) -> np.ndarray:
    """Depth image [H, W] float64 in metres for one agent state."""
    c = cfg.c_struct()
    grid = np.ascontiguousarray(grid, np.uint8)
    st = np.ascontiguousarray(state, np.int32)
    assert grid.shape == (st[S_GRID], st[S_GRID])
    out = np.zeros((cfg.depth_h, cfg.depth_w), np.float64)
    lib().orc_render_depth(ctypes.byref(c), _p(grid), _p(st), _p(out))
    return out


def flee_rewards(grid: np.ndarray, cell_u: int, xy: np.ndarray) -> np.ndarray:
    """Flee (Sec. 5 "Transfer Learning"): r_t = 5 (D_t - D_t-1), D_t = Geo(s_t, s_0) / Max(s_0).
    xy int [T+1, 2] positions in u (xy[0] = the start); returns float32 [T]."""
    grid = np.ascontiguousarray(grid, np.uint8)
    xy = np.ascontiguousarray(xy, np.int32)
    T = xy.shape[0] - 1
    dist = np.zeros(grid.shape, np.int32)
    out = np.zeros(max(T, 0), np.float32)
    if lib().orc_flee_rewards(_p(grid), grid.shape[0], cell_u, _p(xy), T, _p(dist), _p(out)) != 0:
        raise ValueError("start cell is a wall")
    return out


def explore_rewards(xy: np.ndarray, square_u: int = 10000) -> np.ndarray:
    """Exploration (Sec. 5 "Transfer Learning"): r_t = 0.25 (|Visited_t| - |Visited_t-1|) over
    squares of side square_u (1 m by default). xy int [T+1, 2] positions in u; returns
    float32 [T]."""
    xy = np.ascontiguousarray(xy, np.int32)
    T = xy.shape[0] - 1
    out = np.zeros(max(T, 0), np.float32)
    lib().orc_explore_rewards(_p(xy), T, int(square_u), _p(out))
    return out


def goal_vector(state: np.ndarray) -> np.ndarray:
    """[r, cos(theta), sin(theta)] of the goal in the agent frame (App. "Goal encoder")."""
    st = np.ascontiguousarray(state, np.int32)
    out = np.zeros(3, np.float64)
    lib().orc_goal_vector(_p(st), _p(out))
    return out


def env_permutation(seed: int, update: int, epoch: int, E: int) -> np.ndarray:
    """Env order of one PPO epoch; minibatch m takes a contiguous slice of it."""
    perm = np.zeros(E, np.int32)
    lib().orc_env_permutation(seed & (2**64 - 1), update, epoch, E, _p(perm))
    return perm


def pool_obs(depth: np.ndarray, pool: bool, max_depth: float) -> np.ndarray:
    """Policy input: optional 2x2 average pool (App. "Visual Encoder"), then / max_depth."""
    d = np.asarray(depth, np.float64)
    if pool:
        *lead, H, W = d.shape
        d = d.reshape(*lead, H // 2, 2, W // 2, 2).mean(axis=(-1, -3))
    return d / max_depth


class BatchSim:
    """All E environments of one worker, stepped in lock-step (Sec. 4 "Training")."""

    def __init__(self, cfg: SimConfig):
        self.cfg = cfg
        self._c = cfg.c_struct()
        G = cfg.grid_max * cfg.grid_max
        E = cfg.num_envs
        self.grids = np.zeros((E, G), np.uint8)
        self.dists = np.zeros((E, G), np.int32)
        self.states = np.zeros((E, NSTATE), np.int32)

    def reset(self):
        rc = lib().orc_batch_reset(ctypes.byref(self._c), self.cfg.num_envs, _p(self.grids),
                                   _p(self.dists), _p(self.states))
        if rc != 0:
            raise RuntimeError("reset failed")

    def grid(self, e: int) -> np.ndarray:
        g = int(self.states[e, S_GRID])
        return self.grids[e, :g * g].reshape(g, g)

    def dist(self, e: int) -> np.ndarray:
        g = int(self.states[e, S_GRID])
        return self.dists[e, :g * g].reshape(g, g)

    def step(self, actions: np.ndarray):
        E = self.cfg.num_envs
        a = np.ascontiguousarray(actions, np.int32)
        reward = np.zeros(E, np.float32)
        done = np.zeros(E, np.uint8)
        spl = np.zeros(E, np.float32)
        info = np.zeros((E, 4), np.int32)
        rc = lib().orc_batch_step(ctypes.byref(self._c), E, _p(self.grids), _p(self.dists),
                                  _p(self.states), _p(a), _p(reward), _p(done), _p(spl), _p(info))
        if rc != 0:
            raise RuntimeError("step failed")
        return reward, done, spl, info

    def render(self):
        E = self.cfg.num_envs
        depth = np.zeros((E, self.cfg.depth_h, self.cfg.depth_w), np.float64)
        goal = np.zeros((E, 3), np.float64)
        lib().orc_batch_render(ctypes.byref(self._c), E, _p(self.grids), _p(self.states),
                               _p(depth), _p(goal))
        return depth, goal


def deg(k: int) -> float:
    return math.radians(10.0 * k)
