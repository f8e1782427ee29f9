"""Pins of the simulator oracle against closed forms, brute force and invariants.

These tests check ``oracle.sim`` against things that do not come from the
oracle itself: published test vectors, the geometry of an empty room, an
independent exact (rational) segment clip, scipy's Dijkstra, hand-worked
integer cases in ``tests/golden/``.
"""
from fractions import Fraction
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from oracle import sim as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- counter hash
def test_splitmix64_published_vectors():
    # SplitMix64 with state 0: the first three outputs of the reference generator.
    assert S.splitmix64(0) == 0xE220A8397B1DCDAF
    assert S.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    assert S.splitmix64((2 * 0x9E3779B97F4A7C15) % 2**64) == 0x06C45D188009454F


def test_counter_hash_streams_differ():
    hs = {S.counter_hash(1, e, ep, st, i) for e in range(3) for ep in range(3)
          for st in range(1, 8) for i in range(4)}
    assert len(hs) == 3 * 3 * 7 * 4


# ---------------------------------------------------------------- motion table
def test_forward_table_closed_forms():
    """0.25 m forward step at 10 degree headings (Sec. 4 "Agent")."""
    F = S.fwd_table()
    assert tuple(F[0]) == (2500, 0)
    assert tuple(F[9]) == (0, 2500)
    assert tuple(F[18]) == (-2500, 0)
    assert tuple(F[27]) == (0, -2500)
    assert tuple(F[3]) == (2165, 1250)      # 2500 cos 30 = 2165.06, 2500 sin 30 = 1250
    assert tuple(F[6]) == (1250, 2165)
    for k in range(36):
        assert abs(math.hypot(*F[k]) - 2500) < 1.0
        assert tuple(F[(36 - k) % 36]) == (F[k][0], -F[k][1])   # mirror about x
        assert tuple(F[(k + 18) % 36]) == (-F[k][0], -F[k][1])  # half turn


# ---------------------------------------------------------------- scenes
def test_bernoulli_scene_border_and_density():
    cfg = S.SimConfig(grid_min=128, grid_max=128, wall_density=0.15)
    tot, n = 0, 0
    for env in range(4):
        g = S.gen_scene(cfg, env, 0)
        assert g[0].all() and g[-1].all() and g[:, 0].all() and g[:, -1].all()
        inner = g[1:-1, 1:-1]
        tot += inner.sum()
        n += inner.size
    p = tot / n
    assert abs(p - 0.15) < 4 * math.sqrt(0.15 * 0.85 / n)


def test_bernoulli_density_extremes():
    g0 = S.gen_scene(S.SimConfig(wall_density=0.0), 0, 0)
    assert g0[1:-1, 1:-1].sum() == 0
    g1 = S.gen_scene(S.SimConfig(wall_density=1.0), 0, 0)
    assert g1.all()


@pytest.mark.parametrize("g,cell", [(128, 0.1), (64, 0.1), (32, 0.25), (256, 0.1)])
def test_rooms_scene_connected_and_straight_walls(g, cell):
    cfg = S.SimConfig(gen_kind=1, grid_min=g, grid_max=g, cell_m=cell)
    for env in range(3):
        grid = S.gen_scene(cfg, env, 0)
        assert grid[0].all() and grid[-1].all() and grid[:, 0].all() and grid[:, -1].all()
        free = np.argwhere(grid == 0)
        assert len(free) > 0
        y, x = free[0]
        d = S.bfs(grid, x, y)
        # doors are >= 2 cells wide here, so every room is reachable
        assert ((d >= 0) == (grid == 0)).all()
        # no interior 2x2 block of walls: walls are one cell thick
        inner = grid[1:-1, 1:-1].astype(int)
        blk = inner[:-1, :-1] + inner[1:, :-1] + inner[:-1, 1:] + inner[1:, 1:]
        assert (blk < 4).all()


def test_mixed_grid_sizes_cover_all_sides():
    cfg = S.SimConfig(grid_min=64, grid_max=512)
    sides = {S.grid_side(cfg, e, 0) for e in range(200)}
    assert sides == {64, 128, 256, 512}


# ---------------------------------------------------------------- BFS
def _dijkstra(grid, gx, gy):
    g = grid.shape[0]
    idx = lambda x, y: y * g + x
    rows, cols = [], []
    for y in range(g):
        for x in range(g):
            if grid[y, x]:
                continue
            for dx, dy in ((1, 0), (0, 1)):
                nx, ny = x + dx, y + dy
                if nx < g and ny < g and not grid[ny, nx]:
                    rows += [idx(x, y), idx(nx, ny)]
                    cols += [idx(nx, ny), idx(x, y)]
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(g * g, g * g))
    d = csg.dijkstra(A, indices=idx(gx, gy))
    out = np.where(np.isinf(d), -1, d).astype(np.int64).reshape(g, g)
    out[grid.astype(bool)] = -1
    return out


def _floyd(grid):
    g = grid.shape[0]
    n = g * g
    D = np.full((n, n), np.inf)
    for y in range(g):
        for x in range(g):
            if grid[y, x]:
                continue
            D[y * g + x, y * g + x] = 0
            for dx, dy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                nx, ny = x + dx, y + dy
                if 0 <= nx < g and 0 <= ny < g and not grid[ny, nx]:
                    D[y * g + x, ny * g + nx] = 1
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    return D


def test_bfs_equals_dijkstra_random_grids():
    rng = np.random.default_rng(0)
    for trial in range(30):
        g = int(rng.integers(3, 17))
        grid = (rng.random((g, g)) < 0.3).astype(np.uint8)
        free = np.argwhere(grid == 0)
        if len(free) == 0:
            continue
        y, x = free[rng.integers(len(free))]
        assert (S.bfs(grid, x, y) == _dijkstra(grid, x, y)).all()


def test_bfs_equals_floyd_warshall_tiny():
    rng = np.random.default_rng(1)
    for trial in range(10):
        g = int(rng.integers(2, 9))
        grid = (rng.random((g, g)) < 0.25).astype(np.uint8)
        D = _floyd(grid)
        for y, x in np.argwhere(grid == 0)[:5]:
            ref = D[y * g + x].reshape(g, g)
            ref = np.where(np.isinf(ref), -1, ref)
            assert (S.bfs(grid, x, y) == ref).all()


def test_bfs_empty_grid_is_manhattan():
    g = 11
    grid = np.zeros((g, g), np.uint8)
    yy, xx = np.mgrid[0:g, 0:g]
    assert (S.bfs(grid, 3, 7) == np.abs(xx - 3) + np.abs(yy - 7)).all()


def test_bfs_from_wall_all_unreachable():
    grid = np.zeros((5, 5), np.uint8)
    grid[2, 2] = 1
    assert (S.bfs(grid, 2, 2) == -1).all()


# ---------------------------------------------------------------- collision
def _clip_exact(p0, p1, box):
    """Liang-Barsky clip of the closed segment against a closed box, in Fractions."""
    x0, y0 = map(Fraction, p0)
    x1, y1 = map(Fraction, p1)
    bx0, by0, bx1, by1 = map(Fraction, box)
    t0, t1 = Fraction(0), Fraction(1)
    for p, q in ((-(x1 - x0), x0 - bx0), (x1 - x0, bx1 - x0),
                 (-(y1 - y0), y0 - by0), (y1 - y0, by1 - y0)):
        if p == 0:
            if q < 0:
                return False
        else:
            r = q / p
            if p < 0:
                t0 = max(t0, r)
            else:
                t1 = min(t1, r)
    return t0 <= t1


def _blocked_exact(grid, cs, p0, p1):
    g = grid.shape[0]
    for cy in range(-1, g + 1):
        for cx in range(-1, g + 1):
            wall = True if (cx < 0 or cy < 0 or cx >= g or cy >= g) else bool(grid[cy, cx])
            if wall and _clip_exact(p0, p1, (cx * cs, cy * cs, (cx + 1) * cs, (cy + 1) * cs)):
                return True
    return False


def test_segment_test_matches_exact_rational_clip():
    rng = np.random.default_rng(2)
    F = S.fwd_table()
    cs = 1000
    for trial in range(400):
        g = 6
        grid = (rng.random((g, g)) < 0.3).astype(np.uint8)
        grid[0, :] = grid[-1, :] = grid[:, 0] = grid[:, -1] = 1
        # start on lattice-heavy points often, to exercise corner touching
        if trial % 2:
            x0 = int(rng.integers(1, g - 1)) * cs + int(rng.choice([0, 500, 1000 - 1]))
            y0 = int(rng.integers(1, g - 1)) * cs + int(rng.choice([0, 500, 1000 - 1]))
        else:
            x0 = int(rng.integers(cs, (g - 1) * cs))
            y0 = int(rng.integers(cs, (g - 1) * cs))
        k = int(rng.integers(36))
        p1 = (x0 + int(F[k][0]), y0 + int(F[k][1]))
        assert S.segment_blocked(grid, cs, (x0, y0), p1) == _blocked_exact(grid, cs, (x0, y0), p1)


def test_segment_corner_touch_is_blocked():
    grid = np.zeros((5, 5), np.uint8)
    grid[0, :] = grid[-1, :] = grid[:, 0] = grid[:, -1] = 1
    grid[3, 3] = 1
    cs = 1000
    # ends exactly on the corner (3000, 3000) of wall cell (3, 3): touching blocks
    assert S.segment_blocked(grid, cs, (2000, 2000), (3000, 3000))
    # passes diagonally just below the corner: free
    assert not S.segment_blocked(grid, cs, (2000, 1990), (2990, 2980))


# ---------------------------------------------------------------- stepping
def _room(g, cs):
    grid = np.zeros((g, g), np.uint8)
    grid[0, :] = grid[-1, :] = grid[:, 0] = grid[:, -1] = 1
    return grid


def _state(x, y, k, goal, cs, dist, g):
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y], st[S.S_HEAD] = x, y, k
    st[S.S_GOAL_X], st[S.S_GOAL_Y] = goal
    st[S.S_GRID] = g
    geo = dist[y // cs, x // cs] * cs
    st[S.S_GEO_PREV] = st[S.S_GEO_START] = geo
    return st


def _step(cfg, grid, dist, st, a):
    import ctypes
    c = cfg.c_struct()
    r = np.zeros(1, np.float32)
    d = np.zeros(1, np.uint8)
    spl = np.zeros(1, np.float32)
    info = np.zeros(4, np.int32)
    rc = S.lib().orc_step_env(ctypes.byref(c), 0, S._p(grid), S._p(dist), S._p(st), a,
                              S._p(r), S._p(d), S._p(spl), S._p(info))
    assert rc == 0
    return float(r[0]), int(d[0]), float(spl[0]), info.copy()


def _load_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(v) for v in line.split()])
    return rows


@pytest.mark.parametrize("mode", [0, 1])
def test_golden_straight_walk_to_goal(mode):
    """Hand-worked case (tests/golden/walk_9x9.txt): reward, done, success, SPL."""
    g, cs = 9, 2500
    grid = _room(g, cs)
    gx, gy = 6, 4
    dist = np.ascontiguousarray(S.bfs(grid, gx, gy))
    st = _state(1 * cs + 1250, 4 * cs + 1250, 0, (gx * cs + 1250, gy * cs + 1250), cs, dist, g)
    cfg = S.SimConfig(grid_min=g, grid_max=g, cell_m=0.25, terminal_mode=mode, max_steps=500)
    grid = np.ascontiguousarray(grid)
    for a, x, y, k, r_int, done, succ in _load_golden("walk_9x9.txt"):
        ep0 = st[S.S_EPISODE]
        r, d, spl, info = _step(cfg, grid, dist, st, a)
        assert round(r * 10000) == r_int and r == np.float32(r_int / 10000.0)
        assert d == done and info[0] == succ
        if succ:
            assert spl == 1.0          # p = l: SPL = 1
        if not done:
            assert (st[S.S_X], st[S.S_Y], st[S.S_HEAD]) == (x, y, k)
        else:
            assert st[S.S_EPISODE] >= ep0 + 1   # auto-reset drew the next episode


def test_spl_special_cases():
    """SPL = S l / max(l, p): S=0 -> 0; p=2l -> 0.5 (Sec. 4 "PointGoal Navigation")."""
    g, cs = 9, 2500
    grid = np.ascontiguousarray(_room(g, cs))
    gx, gy = 5, 4
    dist = np.ascontiguousarray(S.bfs(grid, gx, gy))
    cfg = S.SimConfig(grid_min=g, grid_max=g, cell_m=0.25, terminal_mode=1)
    # l = 2 cells = 5000. Walk 1 back, 1 forth (turn around twice), then 2 to goal: p = 4 cells.
    st = _state(3 * cs + 1250, 4 * cs + 1250, 18, (gx * cs + 1250, gy * cs + 1250), cs, dist, g)
    seq = [1] + [2] * 18 + [1, 1, 1]
    for a in seq:
        _step(cfg, grid, dist, st, a)
    assert st[S.S_PATH] == 10000 and st[S.S_GEO_START] == 5000
    r, d, spl, info = _step(cfg, grid, dist, st, 0)
    assert info[0] == 1 and d == 1 and spl == 0.5
    assert round(r * 10000) == 0 - 100 + 12500       # +2.5 * SPL
    # stop far from the goal: S = 0, SPL = 0, reward -0.01
    st = _state(1 * cs + 1250, 1 * cs + 1250, 0, (gx * cs + 1250, gy * cs + 1250), cs, dist, g)
    r, d, spl, info = _step(cfg, grid, dist, st, 0)
    assert info[0] == 0 and spl == 0.0 and d == 1 and round(r * 10000) == -100


def test_motion_invariants():
    g, cs = 12, 1000
    grid = np.ascontiguousarray(_room(g, cs))
    dist = np.ascontiguousarray(S.bfs(grid, 6, 6))
    cfg = S.SimConfig(grid_min=g, grid_max=g, cell_m=0.1, max_steps=10**6)
    st = _state(5500, 5500, 7, (6500, 6500), cs, dist, g)
    x0 = st.copy()
    for _ in range(36):
        _step(cfg, grid, dist, st, 2)
    assert st[S.S_HEAD] == x0[S.S_HEAD] and st[S.S_X] == x0[S.S_X] and st[S.S_Y] == x0[S.S_Y]
    _step(cfg, grid, dist, st, 2)
    _step(cfg, grid, dist, st, 3)
    assert st[S.S_HEAD] == x0[S.S_HEAD]
    # forward until the wall blocks: position freezes, collided set, path stops growing
    st[S.S_HEAD] = 0
    F = S.fwd_table()
    for _ in range(10):
        px, path = st[S.S_X], st[S.S_PATH]
        r, d, spl, info = _step(cfg, grid, dist, st, 1)
        if info[1]:
            assert st[S.S_X] == px and st[S.S_PATH] == path
            break
        assert st[S.S_X] == px + F[0][0]
    else:
        raise AssertionError("never collided")
    # the blocked position: the next move would touch the wall at x = 11000
    assert st[S.S_X] + 2500 >= (g - 1) * cs


def test_timeout_ends_episode_without_success():
    g, cs = 9, 2500
    grid = np.ascontiguousarray(_room(g, cs))
    dist = np.ascontiguousarray(S.bfs(grid, 6, 4))
    cfg = S.SimConfig(grid_min=g, grid_max=g, cell_m=0.25, max_steps=3)
    st = _state(1 * cs + 1250, 4 * cs + 1250, 9, (6 * cs + 1250, 4 * cs + 1250), cs, dist, g)
    outs = [_step(cfg, grid, dist, st, 2)[1] for _ in range(3)]
    assert outs == [0, 0, 1]


# ---------------------------------------------------------------- reset
@pytest.mark.parametrize("kind,g,cell", [(0, 32, 0.25), (1, 128, 0.1)])
def test_reset_invariants(kind, g, cell):
    cfg = S.SimConfig(num_envs=8, gen_kind=kind, grid_min=g, grid_max=g, cell_m=cell)
    b = S.BatchSim(cfg)
    b.reset()
    cs = cfg.cell_u
    for e in range(cfg.num_envs):
        st = b.states[e]
        grid, dist = b.grid(e), b.dist(e)
        sx, sy = st[S.S_X] // cs, st[S.S_Y] // cs
        gx, gy = st[S.S_GOAL_X] // cs, st[S.S_GOAL_Y] // cs
        assert grid[sy, sx] == 0 and grid[gy, gx] == 0
        assert dist[gy, gx] == 0
        assert st[S.S_GEO_START] == dist[sy, sx] * cs >= 20000     # >= 2 m apart
        assert st[S.S_X] % cs == cs // 2 and st[S.S_GOAL_Y] % cs == cs // 2
        assert 0 <= st[S.S_HEAD] < 36
        assert (S.bfs(grid, gx, gy) == dist).all()


# ---------------------------------------------------------------- depth
def _empty_room_cfg(W=64, H=64):
    return S.SimConfig(grid_min=20, grid_max=20, cell_m=0.25, depth_h=H, depth_w=W)


@pytest.mark.parametrize("W", [64, 256])
def test_depth_empty_room_closed_form(W):
    """Empty rectangular room, heading 0: z-depth to the far wall is X - x0 for every
    column that hits it; side walls at (y0 - Y)/x_i; floor h/(-y_j), ceiling (2.5-h)/y_j."""
    cfg = _empty_room_cfg(W, W)
    g, cs = 20, 2500
    grid = _room(g, cs)
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y], st[S.S_HEAD], st[S.S_GRID] = 6 * cs + 700, 9 * cs + 300, 0, g
    depth = S.render_depth(cfg, grid, st)
    x0, y0 = st[S.S_X] / 1e4, st[S.S_Y] / 1e4
    Xf, Ylo, Yhi = (g - 1) * 0.25, 1 * 0.25, (g - 1) * 0.25
    for i in range(W):
        xi = (2 * i + 1) / W - 1
        tw = Xf - x0
        if xi > 0:
            tw = min(tw, (y0 - Ylo) / xi)
        elif xi < 0:
            tw = min(tw, (Yhi - y0) / (-xi))
        for j in range(W):
            yj = 1 - (2 * j + 1) / W
            tp = 0.88 / (-yj) if yj < 0 else (2.5 - 0.88) / yj
            ref = min(tw, tp, 10.0)
            assert abs(depth[j, i] - ref) < 1e-12, (i, j, depth[j, i], ref)


def test_depth_heading_90_closed_form():
    cfg = _empty_room_cfg(32, 32)
    g, cs = 20, 2500
    grid = _room(g, cs)
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y], st[S.S_HEAD], st[S.S_GRID] = 7 * cs, 5 * cs + 1, 9, g
    depth = S.render_depth(cfg, grid, st)
    # facing +y: the far wall face is y = (g-1)*cs; the horizon rows are wall-limited
    far = ((g - 1) * cs - st[S.S_Y]) / 1e4
    xs = [(2 * i + 1) / 32 - 1 for i in range(32)]
    # columns whose ray hits the far wall before the side walls (x in [cs, (g-1) cs])
    for i, xi in enumerate(xs):
        x_hit = st[S.S_X] / 1e4 + far * xi * 1.0  # right vector at 90 deg is (1, 0)
        if 0.25 < x_hit < (g - 1) * 0.25:
            j = 15  # y_j = 1/32, ceiling plane at 1.62*32 m: wall-limited
            assert abs(depth[j, i] - min(far, 10.0)) < 1e-12


def test_depth_single_wall_cell():
    cfg = _empty_room_cfg(64, 64)
    g, cs = 20, 2500
    grid = _room(g, cs)
    grid[9, 9] = 1
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y], st[S.S_HEAD], st[S.S_GRID] = 6 * cs + 1250, 9 * cs + 1250, 0, g
    depth = S.render_depth(cfg, grid, st)
    # two central columns (x_i = +-1/64) hit the face x = 9*cs of cell (9, 9)
    for i in (31, 32):
        assert abs(depth[32, i] - (9 * cs - st[S.S_X]) / 1e4) < 1e-12
        assert abs(depth[32, i] - 0.625) < 1e-12
    assert (depth >= 0).all() and (depth <= 10.0).all()


def test_depth_clip_at_max_depth():
    cfg = S.SimConfig(grid_min=64, grid_max=64, cell_m=0.25, depth_h=16, depth_w=16)
    g, cs = 64, 2500
    grid = _room(g, cs)
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y], st[S.S_HEAD], st[S.S_GRID] = 1 * cs + 100, 32 * cs, 0, g
    depth = S.render_depth(cfg, grid, st)
    # far wall 15.3 m away; horizon-adjacent rows are capped at 10 m
    assert depth[7, 8] == 10.0 and depth[8, 8] == 10.0


def test_goal_vector_closed_form():
    st = np.zeros(S.NSTATE, np.int32)
    st[S.S_X], st[S.S_Y] = 10000, 10000
    st[S.S_GOAL_X], st[S.S_GOAL_Y] = 40000, 50000      # 3 m east, 4 m north
    st[S.S_HEAD] = 0
    g = S.goal_vector(st)
    assert np.allclose(g, [5.0, 0.6, 0.8], atol=1e-12)
    st[S.S_HEAD] = 9                                    # facing north: goal 4 ahead, 3 right
    g = S.goal_vector(st)
    assert np.allclose(g, [5.0, 0.8, -0.6], atol=1e-12)


def test_env_permutation_is_permutation():
    for E in (1, 2, 16, 64):
        p = S.env_permutation(0, 3, 1, E)
        assert sorted(p.tolist()) == list(range(E))
    assert not (S.env_permutation(0, 0, 0, 64) == np.arange(64)).all()


# ---------------------------------------------------------------- transfer tasks (Sec. 5)
def _border_room(g):
    grid = np.zeros((g, g), np.uint8)
    grid[0, :] = grid[-1, :] = grid[:, 0] = grid[:, -1] = 1
    return grid


def _walk(x0, y0, steps):
    """Positions of a walk with axis-aligned unit moves of 2500 u: steps is a list of
    (dx, dy) in {-1, 0, 1}^2 (0, 0 = a turn: the agent stays)."""
    xy = [(x0, y0)]
    for dx, dy in steps:
        x, y = xy[-1]
        xy.append((x + 2500 * dx, y + 2500 * dy))
    return np.array(xy, np.int32)


def test_flee_empty_room_closed_form():
    # 16x16 room (free cells 1..14), 0.25 m cells, start at the centre of cell (3, 5):
    # Geo = Manhattan distance in cells, Max = (14 - 3) + (14 - 5) = 20, so each cell
    # walked away from the start earns 5 / 20 = 0.25, each one walked back -0.25, a turn 0.
    g, cs = 16, 2500
    grid = _border_room(g)
    x0, y0 = 3 * cs + cs // 2, 5 * cs + cs // 2
    steps = [(1, 0)] * 6 + [(0, 0)] * 3 + [(-1, 0)] * 8 + [(0, 1)] * 4
    r = S.flee_rewards(grid, cs, _walk(x0, y0, steps))
    want = [0.25] * 6 + [0.0] * 3 + [-0.25] * 6 + [0.25] * 2 + [0.25] * 4
    assert r.tolist() == want
    # the rewards telescope: sum = 5 D_T with D_T = (|x_T - 3| + |y_T - 5|) / 20
    assert abs(float(r.astype(np.float64).sum()) - 5 * (2 + 4) / 20) < 1e-12


def test_flee_geodesic_detour_against_networkx():
    # a wall across the room with one gap: geodesic distances from the start and their
    # maximum come from networkx's BFS on the free-cell graph
    nx = pytest.importorskip("networkx")
    g, cs = 12, 2500
    grid = _border_room(g)
    grid[6, 1:10] = 1                      # wall along row 6, gap at column 10
    start = (2, 3)
    G = nx.grid_2d_graph(g, g)
    G.remove_nodes_from([(y, x) for y in range(g) for x in range(g) if grid[y, x]])
    d = nx.single_source_shortest_path_length(G, (start[1], start[0]))
    mx = max(d.values())
    rng = np.random.default_rng(5)
    cells = [start]
    for _ in range(60):                    # a random walk over free cells
        x, y = cells[-1]
        opts = [(x + a, y + b) for a, b in ((1, 0), (-1, 0), (0, 1), (0, -1)) if not grid[y + b, x + a]]
        cells.append(opts[rng.integers(len(opts))])
    xy = np.array([(x * cs + 1250, y * cs + 1250) for x, y in cells], np.int32)
    r = S.flee_rewards(grid, cs, xy)
    for t in range(1, len(cells)):
        dd = d[(cells[t][1], cells[t][0])] - d[(cells[t - 1][1], cells[t - 1][0])]
        assert r[t - 1] == np.float32(5 * dd / mx)
    assert mx > 2 * (g - 2)                # the detour is longer than any Manhattan path


def test_flee_rejects_a_wall_start():
    grid = _border_room(8)
    with pytest.raises(ValueError):
        S.flee_rewards(grid, 2500, np.array([[1250, 1250], [1250, 1250]], np.int32))


def test_exploration_new_square_every_metre():
    # start at (0.5 m, 0.5 m), heading +x in 0.25 m steps: x = 0.5 + 0.25 k enters the
    # square of x = 1 m at k = 2, of 2 m at k = 6, of 3 m at k = 10; walking back over
    # visited squares earns nothing; a step into y = 1 m is a new square again
    steps = [(1, 0)] * 10 + [(-1, 0)] * 10 + [(0, 1)] * 2
    r = S.explore_rewards(_walk(5000, 5000, steps))
    want = np.zeros(22, np.float32)
    want[[1, 5, 9, 21]] = 0.25
    assert r.tolist() == want.tolist()
    assert float(r.sum()) == 0.25 * (4 + 1 - 1)


def test_exploration_total_counts_distinct_squares():
    # over any trajectory the rewards add up to 0.25 (number of distinct squares - 1),
    # and a trajectory confined to one square earns nothing
    rng = np.random.default_rng(11)
    xy = np.cumsum(rng.integers(-2500, 2501, size=(200, 2)), axis=0) + 50000
    r = S.explore_rewards(xy.astype(np.int32))
    squares = {(int(x) // 10000, int(y) // 10000) for x, y in xy}
    assert float(r.astype(np.float64).sum()) == 0.25 * (len(squares) - 1)
    still = np.tile(np.array([[12345, 61234]], np.int32), (9, 1)) + rng.integers(0, 5000, (9, 2)).astype(np.int32)
    assert not S.explore_rewards(still).any()


def test_exploration_square_side_is_a_parameter():
    # 0.5 m squares: from x = 0.125 m in 0.25 m steps the walk enters a new square every
    # second step (x = 0.625, 1.125, ... m); the total still counts distinct squares
    steps = [(1, 0)] * 8
    r = S.explore_rewards(_walk(1250, 1250, steps), square_u=5000)
    want = np.zeros(8, np.float32)
    want[[1, 3, 5, 7]] = 0.25
    assert r.tolist() == want.tolist()
    assert S.explore_rewards(_walk(1250, 1250, steps)).tolist() == [0, 0, 0, 0.25, 0, 0, 0, 0.25]
