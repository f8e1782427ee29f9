/*
 * FP64 / integer CPU oracle for the PointGoal-navigation simulator of DD-PPO
 * (arXiv:1911.00357, Sec. 4 "PointGoal Navigation", "Agent", "Training").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct
 * restatement of what the simulator computes. Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark may load it. It shares no code,
 * header, table or constant generator with the CUDA library; every quantity
 * (the forward-step table, the counter-hash draws, the segment test, the ray
 * march) is computed here from its definition.
 *
 * Readings of the paper taken here (the paper describes Habitat-Sim, whose
 * scenes and renderer are not available, so an occupancy-grid world stands in):
 *   - positions are int32 in units u = 1e-4 m; a cell is cell_u u wide;
 *     cell(p) = floor(p / cell_u) (positions are always >= 0);
 *   - heading k in [0,36), angle 10k degrees counter-clockwise from +x; x is
 *     the column axis, y the row axis;  turn_left k+1, turn_right k-1 (Sec. 4
 *     "Agent": 10 degree turns);
 *   - move_forward 0.25 m (Sec. 4 "Agent") adds FWD[k] = round(2500 cos, 2500 sin)
 *     of the heading, computed here with libm in double and rounded half away
 *     from zero; the move is blocked (no slide) when the closed segment touches
 *     the closed square of any wall cell; the path length grows by the nominal
 *     2500 u per successful forward move;
 *   - geodesic distance (Sec. 4 "Training") = 4-connected unit-cost BFS over
 *     free cells from the goal cell, times cell_u;
 *   - reward r = -(geo_new - geo_prev) - 0.01 m per step (Sec. 4 "Training"),
 *     plus a terminal bonus on success: 2.5 (mode 0) or 2.5 * SPL (mode 1);
 *   - success = the agent called stop within 0.2 m (Euclidean) of the goal;
 *     SPL = S * l / max(l, p) (Sec. 4 "PointGoal Navigation");
 *   - an episode ends on stop or when steps reach max_steps;
 *   - depth is z-depth along the optical axis, 90 degree square field of view,
 *     walls span floor to ceiling, analytic floor/ceiling planes, clipped to
 *     [0, max_depth] (Sec. 4 "Agent": 256x256 depth images).
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_STREAM_GRID 1u
#define ORC_STREAM_ROOMS 2u
#define ORC_STREAM_GOAL 3u
#define ORC_STREAM_START 4u
#define ORC_STREAM_HEADING 5u
#define ORC_STREAM_SIZE 6u
#define ORC_STREAM_PERM 7u

/* per-env agent state slots (int32) */
enum {
  S_X = 0, S_Y, S_HEAD, S_STEPS, S_PATH, S_GEO_PREV, S_GEO_START, S_GOAL_X,
  S_GOAL_Y, S_EPISODE, S_GRID, S_COLLIDED, S_NSTATE
};

typedef struct {
  int32_t gen_kind;      /* 0: Bernoulli walls, 1: rooms and doors          */
  int32_t grid_min;      /* smallest square grid side (cells)               */
  int32_t grid_max;      /* largest; sides are grid_min * 2^j up to this    */
  int32_t cell_u;        /* cell side in u                                  */
  double wall_density;   /* Bernoulli wall probability                      */
  int32_t door_cells;    /* door width in cells (rooms)                     */
  int32_t min_room;      /* minimum room side in cells (rooms)              */
  int32_t max_steps;     /* episode step cap                                */
  int32_t terminal_mode; /* 0: +2.5 on success, 1: +2.5*SPL                 */
  int32_t depth_h, depth_w;
  double cam_h_m, ceil_h_m, max_depth_m;
  uint64_t seed;
} orc_cfg;

/* ---- SplitMix64 (Steele, Lea, Flood 2014), used as a counter hash ---- */
uint64_t orc_sm64(uint64_t z);
static uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t orc_sm64(uint64_t z) { return sm64(z); }

uint64_t orc_hash(uint64_t seed, uint64_t env, uint64_t episode, uint32_t stream,
                  uint64_t index) {
  uint64_t k = sm64(seed);
  k = sm64(k + env);
  k = sm64(k + episode);
  return sm64(k + (((uint64_t)stream << 40) | (index & 0xFFFFFFFFFFull)));
}

/* integer uniform in [0, n) by multiply-shift of the high 32 bits */
static uint32_t uni(uint64_t h, uint32_t n) {
  return (uint32_t)(((h >> 32) * (uint64_t)n) >> 32);
}

/* FWD[k], k in [0,36): round half away from zero of 2500*(cos, sin)(10k deg) */
void orc_fwd_table(int32_t* out72) {
  for (int k = 0; k < 36; ++k) {
    double a = (double)k * 10.0 * M_PI / 180.0;
    out72[2 * k + 0] = (int32_t)llround(2500.0 * cos(a));
    out72[2 * k + 1] = (int32_t)llround(2500.0 * sin(a));
  }
}

int32_t orc_grid_side(const orc_cfg* c, int64_t env, int64_t episode) {
  if (c->grid_max <= c->grid_min) return c->grid_min;
  int n = 0;
  for (int s = c->grid_min; s <= c->grid_max; s *= 2) ++n;
  uint32_t j = uni(orc_hash(c->seed, env, episode, ORC_STREAM_SIZE, 0), (uint32_t)n);
  return c->grid_min << j;
}

/* ---- scene generation: grid[y*g + x] = 1 for wall, 0 for free ---- */
static void gen_bernoulli(const orc_cfg* c, int64_t env, int64_t ep, int g, uint8_t* grid) {
  uint32_t thr = (uint32_t)floor(c->wall_density * 16777216.0);
  for (int y = 0; y < g; ++y)
    for (int x = 0; x < g; ++x) {
      int border = (x == 0 || y == 0 || x == g - 1 || y == g - 1);
      uint32_t u24 = (uint32_t)(orc_hash(c->seed, env, ep, ORC_STREAM_GRID,
                                         (uint64_t)y * g + x) >> 40);
      grid[y * g + x] = (uint8_t)(border || u24 < thr);
    }
}

/* Recursive binary space partition: the longer side of a room is cut by a
 * one-cell wall with one door; rooms below 2*min_room+1 along that side stay.
 * Depth-first, the second child popped first; node n draws index 2n (wall
 * position) and 2n+1 (door position). Returns -1 on stack overflow. */
static int gen_rooms(const orc_cfg* c, int64_t env, int64_t ep, int g, uint8_t* grid) {
  for (int y = 0; y < g; ++y)
    for (int x = 0; x < g; ++x)
      grid[y * g + x] = (uint8_t)(x == 0 || y == 0 || x == g - 1 || y == g - 1);
  int stack[256][4];
  int sp = 0;
  stack[sp][0] = 1; stack[sp][1] = 1; stack[sp][2] = g - 1; stack[sp][3] = g - 1; ++sp;
  uint64_t node = 0;
  const int M = c->min_room;
  while (sp > 0) {
    --sp;
    int x0 = stack[sp][0], y0 = stack[sp][1], x1 = stack[sp][2], y1 = stack[sp][3];
    uint64_t n = node++;
    int w = x1 - x0, h = y1 - y0;
    uint64_t hp = orc_hash(c->seed, env, ep, ORC_STREAM_ROOMS, 2 * n);
    uint64_t hd = orc_hash(c->seed, env, ep, ORC_STREAM_ROOMS, 2 * n + 1);
    if (w >= h) {
      if (w < 2 * M + 1) continue;
      int p = x0 + M + (int)uni(hp, (uint32_t)(w - 2 * M));
      for (int y = y0; y < y1; ++y) grid[y * g + p] = 1;
      int D = c->door_cells < h ? c->door_cells : h;
      int d = y0 + (int)uni(hd, (uint32_t)(h - D + 1));
      for (int y = d; y < d + D; ++y) grid[y * g + p] = 0;
      if (sp + 2 > 256) return -1;
      stack[sp][0] = x0; stack[sp][1] = y0; stack[sp][2] = p; stack[sp][3] = y1; ++sp;
      stack[sp][0] = p + 1; stack[sp][1] = y0; stack[sp][2] = x1; stack[sp][3] = y1; ++sp;
    } else {
      if (h < 2 * M + 1) continue;
      int p = y0 + M + (int)uni(hp, (uint32_t)(h - 2 * M));
      for (int x = x0; x < x1; ++x) grid[p * g + x] = 1;
      int D = c->door_cells < w ? c->door_cells : w;
      int d = x0 + (int)uni(hd, (uint32_t)(w - D + 1));
      for (int x = d; x < d + D; ++x) grid[p * g + x] = 0;
      if (sp + 2 > 256) return -1;
      stack[sp][0] = x0; stack[sp][1] = y0; stack[sp][2] = x1; stack[sp][3] = p; ++sp;
      stack[sp][0] = x0; stack[sp][1] = p + 1; stack[sp][2] = x1; stack[sp][3] = y1; ++sp;
    }
  }
  return 0;
}

int orc_gen_scene(const orc_cfg* c, int64_t env, int64_t ep, int g, uint8_t* grid) {
  if (c->gen_kind == 0) { gen_bernoulli(c, env, ep, g, grid); return 0; }
  return gen_rooms(c, env, ep, g, grid);
}

/* ---- BFS distance field from (gx, gy): 4-connected, unit cost, -1 unreachable ---- */
int orc_bfs(const uint8_t* grid, int g, int gx, int gy, int32_t* dist) {
  int G = g * g;
  for (int i = 0; i < G; ++i) dist[i] = -1;
  if (grid[gy * g + gx]) return 0;
  int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)G);
  if (!q) return -1;
  int head = 0, tail = 0;
  dist[gy * g + gx] = 0;
  q[tail++] = gy * g + gx;
  while (head < tail) {
    int c = q[head++];
    int x = c % g, y = c / g;
    const int nx[4] = {x + 1, x - 1, x, x};
    const int ny[4] = {y, y, y + 1, y - 1};
    for (int k = 0; k < 4; ++k) {
      if (nx[k] < 0 || ny[k] < 0 || nx[k] >= g || ny[k] >= g) continue;
      int n = ny[k] * g + nx[k];
      if (grid[n] || dist[n] >= 0) continue;
      dist[n] = dist[c] + 1;
      q[tail++] = n;
    }
  }
  free(q);
  return 0;
}

/* ---- episode reset: scene, BFS from a uniformly drawn free goal cell, start
 * uniformly among cells at geodesic >= 2 m, heading uniform over 36.
 * Up to 64 attempts per episode counter, then the next counter (8 at most).
 * grid/dist must hold grid_max^2 entries. Returns 0 or -1. ---- */
int orc_reset_env(const orc_cfg* c, int64_t env, int64_t episode, uint8_t* grid,
                  int32_t* dist, int32_t* st) {
  for (int e = 0; e < 8; ++e, ++episode) {
    int g = orc_grid_side(c, env, episode);
    if (orc_gen_scene(c, env, episode, g, grid) != 0) return -1;
    int G = g * g;
    for (int a = 0; a < 64; ++a) {
      int gi = (int)uni(orc_hash(c->seed, env, episode, ORC_STREAM_GOAL, (uint64_t)a), (uint32_t)G);
      if (grid[gi]) continue;
      if (orc_bfs(grid, g, gi % g, gi / g, dist) != 0) return -1;
      int64_t cnt = 0;
      for (int i = 0; i < G; ++i)
        if (dist[i] >= 0 && (int64_t)dist[i] * c->cell_u >= 20000) ++cnt;
      if (cnt == 0) continue;
      int64_t k = uni(orc_hash(c->seed, env, episode, ORC_STREAM_START, (uint64_t)a), (uint32_t)cnt);
      int si = -1;
      for (int i = 0; i < G; ++i)
        if (dist[i] >= 0 && (int64_t)dist[i] * c->cell_u >= 20000) {
          if (k == 0) { si = i; break; }
          --k;
        }
      int head = (int)uni(orc_hash(c->seed, env, episode, ORC_STREAM_HEADING, (uint64_t)a), 36u);
      int half = c->cell_u / 2;
      st[S_X] = (si % g) * c->cell_u + half;
      st[S_Y] = (si / g) * c->cell_u + half;
      st[S_HEAD] = head;
      st[S_STEPS] = 0;
      st[S_PATH] = 0;
      st[S_GEO_START] = dist[si] * c->cell_u;
      st[S_GEO_PREV] = st[S_GEO_START];
      st[S_GOAL_X] = (gi % g) * c->cell_u + half;
      st[S_GOAL_Y] = (gi / g) * c->cell_u + half;
      st[S_EPISODE] = (int32_t)episode;
      st[S_GRID] = g;
      st[S_COLLIDED] = 0;
      return 0;
    }
  }
  return -1;
}

/* ---- collision: does the closed segment P0-P1 meet the closed square of cell
 * (cx, cy)? Separating-axis test in exact int64 arithmetic. ---- */
static int seg_meets_cell(int64_t x0, int64_t y0, int64_t x1, int64_t y1, int64_t cx,
                          int64_t cy, int64_t cs) {
  int64_t bx0 = cx * cs, bx1 = (cx + 1) * cs, by0 = cy * cs, by1 = (cy + 1) * cs;
  int64_t sx0 = x0 < x1 ? x0 : x1, sx1 = x0 < x1 ? x1 : x0;
  int64_t sy0 = y0 < y1 ? y0 : y1, sy1 = y0 < y1 ? y1 : y0;
  if (sx1 < bx0 || sx0 > bx1 || sy1 < by0 || sy0 > by1) return 0;
  int64_t dx = x1 - x0, dy = y1 - y0;
  int pos = 0, neg = 0;
  const int64_t qx[4] = {bx0, bx1, bx0, bx1};
  const int64_t qy[4] = {by0, by0, by1, by1};
  for (int i = 0; i < 4; ++i) {
    int64_t cr = dx * (qy[i] - y0) - dy * (qx[i] - x0);
    if (cr > 0) ++pos;
    else if (cr < 0) ++neg;
  }
  return !(pos == 4 || neg == 4);
}

/* Blocked iff some wall cell, or some cell outside the grid, meets the segment.
 * Brute force over every cell of the grid plus a one-cell ring outside it. */
int orc_segment_blocked(const uint8_t* grid, int g, int cs, int32_t x0, int32_t y0,
                        int32_t x1, int32_t y1) {
  for (int cy = -1; cy <= g; ++cy)
    for (int cx = -1; cx <= g; ++cx) {
      int wall = (cx < 0 || cy < 0 || cx >= g || cy >= g) ? 1 : grid[cy * g + cx];
      if (wall && seg_meets_cell(x0, y0, x1, y1, cx, cy, cs)) return 1;
    }
  return 0;
}

/* ---- one environment step with auto-reset (Sec. 4 "Training", "PointGoal
 * Navigation"). info[0]=success, info[1]=collided, info[2]=steps of the finished
 * step, info[3]=episode of the finished step. ---- */
int orc_step_env(const orc_cfg* c, int64_t env, uint8_t* grid, int32_t* dist, int32_t* st,
                 int32_t action, float* reward, uint8_t* done, float* spl, int32_t* info) {
  int32_t fwd[72];
  orc_fwd_table(fwd);
  int g = st[S_GRID];
  int cs = c->cell_u;
  int success = 0, finished = 0, collided = 0;
  st[S_STEPS] += 1;
  if (action == 0) {
    int64_t dx = (int64_t)st[S_GOAL_X] - st[S_X], dy = (int64_t)st[S_GOAL_Y] - st[S_Y];
    success = (dx * dx + dy * dy <= (int64_t)2000 * 2000);
    finished = 1;
  } else if (action == 1) {
    int32_t nx = st[S_X] + fwd[2 * st[S_HEAD]], ny = st[S_Y] + fwd[2 * st[S_HEAD] + 1];
    if (orc_segment_blocked(grid, g, cs, st[S_X], st[S_Y], nx, ny)) {
      collided = 1;
    } else {
      st[S_X] = nx; st[S_Y] = ny; st[S_PATH] += 2500;
    }
  } else if (action == 2) {
    st[S_HEAD] = (st[S_HEAD] + 1) % 36;
  } else if (action == 3) {
    st[S_HEAD] = (st[S_HEAD] + 35) % 36;
  } else {
    return -1;
  }
  int cx = st[S_X] / cs, cy = st[S_Y] / cs;
  int32_t geo_new = dist[cy * g + cx] * cs;
  int64_t r = (int64_t)st[S_GEO_PREV] - geo_new - 100;
  int64_t l = st[S_GEO_START], p = st[S_PATH];
  int64_t m = l > p ? l : p;
  if (success) {
    if (c->terminal_mode == 0) r += 25000;
    else r += (2 * 25000 * l + m) / (2 * m);
  }
  st[S_GEO_PREV] = geo_new;
  st[S_COLLIDED] = collided;
  if (!finished && st[S_STEPS] >= c->max_steps) finished = 1;
  *reward = (float)((double)r / 10000.0);
  *done = (uint8_t)finished;
  *spl = success ? (float)((double)l / (double)m) : 0.0f;
  info[0] = success;
  info[1] = collided;
  info[2] = st[S_STEPS];
  info[3] = st[S_EPISODE];
  if (finished) return orc_reset_env(c, env, (int64_t)st[S_EPISODE] + 1, grid, dist, st);
  return 0;
}

/* ---- transfer tasks (Sec. 5 "Transfer Learning"), as rewards of a trajectory ----
 * xy: int32 [T+1, 2] agent positions in u, xy[0] the episode's start; rewards: [T].
 *
 * Flee: D_t = Geo(s_t, s_0) / Max(s_0), Geo the 4-connected unit-cost BFS distance from
 * the start cell (the same geodesic as the PointGoal reward, from another source) and
 * Max(s_0) the largest distance over the cells reachable from it; r_t = 5 (D_t - D_t-1).
 * In cells the cell size cancels: r_t = 5 (d_t - d_t-1) / Max, two exact integers and
 * one correctly rounded division (double, then float: innocuous for integers < 2^24).
 * dist: scratch [g * g]. Returns -1 when the start cell is a wall (or out of memory). */
int orc_flee_rewards(const uint8_t* grid, int g, int cs, const int32_t* xy, int T,
                     int32_t* dist, float* rewards) {
  int sx = xy[0] / cs, sy = xy[1] / cs;
  if (grid[sy * g + sx]) return -1;
  if (orc_bfs(grid, g, sx, sy, dist) != 0) return -1;
  int32_t mx = 0;
  for (int i = 0; i < g * g; ++i)
    if (dist[i] > mx) mx = dist[i];
  for (int t = 1; t <= T; ++t) {
    int32_t d1 = dist[(xy[2 * t + 1] / cs) * g + xy[2 * t] / cs];
    int32_t d0 = dist[(xy[2 * t - 1] / cs) * g + xy[2 * t - 2] / cs];
    rewards[t - 1] = mx > 0 ? (float)((double)(5 * (d1 - d0)) / (double)mx) : 0.0f;
  }
  return 0;
}

/* Exploration: Visited_t = the distinct squares of side sq u (the paper's 1 m cubes:
 * sq = 10000; floor(p / sq) on each axis) of positions 0..t, the start included;
 * r_t = 0.25 (|Visited_t| - |Visited_t-1|), exact in FP32. Brute force over the earlier
 * positions. */
void orc_explore_rewards(const int32_t* xy, int T, int sq, float* rewards) {
  for (int t = 1; t <= T; ++t) {
    int qx = xy[2 * t] / sq, qy = xy[2 * t + 1] / sq, seen = 0;
    for (int k = 0; k < t && !seen; ++k)
      seen = xy[2 * k] / sq == qx && xy[2 * k + 1] / sq == qy;
    rewards[t - 1] = seen ? 0.0f : 0.25f;
  }
}

/* ---- goal vector [r (m), cos(theta), sin(theta)]: the goal in the agent's
 * egocentric polar frame (App. "Goal encoder"); (r, 1, 0) when r = 0. ---- */
void orc_goal_vector(const int32_t* st, double* out3) {
  double dx = ((double)st[S_GOAL_X] - st[S_X]) / 10000.0;
  double dy = ((double)st[S_GOAL_Y] - st[S_Y]) / 10000.0;
  double a = (double)st[S_HEAD] * 10.0 * M_PI / 180.0;
  double f = dx * cos(a) + dy * sin(a);
  double l = -dx * sin(a) + dy * cos(a);
  double r = sqrt(dx * dx + dy * dy);
  out3[0] = r;
  out3[1] = r > 0 ? f / r : 1.0;
  out3[2] = r > 0 ? l / r : 0.0;
}

/* ---- depth: for each image column, march the grid cell by cell in double
 * with the crossing parameter recomputed from the boundary plane at every
 * step (an exact-corner tie crosses x first); the z-depth of the first wall
 * cell entered is t_wall. Each pixel is min(t_wall, t_plane) clipped to
 * [0, max_depth], t_plane from the floor (below the horizon) or ceiling
 * (above). Camera at the agent's position and heading; f = (cos, sin),
 * right = (sin, -cos); column i looks along f + x_i * right with
 * x_i = (2i+1)/W - 1; row j has slope y_j = 1 - (2j+1)/H. ---- */
double orc_column_twall(const uint8_t* grid, int g, int cs, double px, double py,
                        double dx, double dy) {
  int cx = (int)floor(px / cs), cy = (int)floor(py / cs);
  int sx = dx > 0 ? 1 : (dx < 0 ? -1 : 0);
  int sy = dy > 0 ? 1 : (dy < 0 ? -1 : 0);
  for (int it = 0; it < 8 * g + 8; ++it) {
    double tx = sx ? (((double)(cx + (sx > 0)) * cs) - px) / dx : INFINITY;
    double ty = sy ? (((double)(cy + (sy > 0)) * cs) - py) / dy : INFINITY;
    double t;
    if (tx <= ty) { cx += sx; t = tx; } else { cy += sy; t = ty; }
    if (cx < 0 || cy < 0 || cx >= g || cy >= g) return INFINITY;
    if (grid[cy * g + cx]) return t;
  }
  return INFINITY;
}

void orc_render_depth(const orc_cfg* c, const uint8_t* grid, const int32_t* st, double* depth) {
  int g = st[S_GRID], cs = c->cell_u, H = c->depth_h, W = c->depth_w;
  double a = (double)st[S_HEAD] * 10.0 * M_PI / 180.0;
  double fx = cos(a), fy = sin(a), rx = sin(a), ry = -cos(a);
  double px = st[S_X], py = st[S_Y];
  for (int i = 0; i < W; ++i) {
    double xi = (2.0 * i + 1.0) / W - 1.0;
    double tw = orc_column_twall(grid, g, cs, px, py, fx + xi * rx, fy + xi * ry) / 10000.0;
    for (int j = 0; j < H; ++j) {
      double yj = 1.0 - (2.0 * j + 1.0) / H;
      double tp = yj < 0 ? c->cam_h_m / (-yj) : (c->ceil_h_m - c->cam_h_m) / yj;
      double d = tw < tp ? tw : tp;
      if (d > c->max_depth_m) d = c->max_depth_m;
      if (d < 0) d = 0;
      depth[(size_t)j * W + i] = d;
    }
  }
}

/* ---- minibatch permutation of envs for one epoch (Fisher-Yates) ---- */
void orc_env_permutation(uint64_t seed, int64_t update, int64_t epoch, int E, int32_t* perm) {
  for (int i = 0; i < E; ++i) perm[i] = i;
  for (int i = E - 1; i >= 1; --i) {
    uint64_t h = orc_hash(seed, 0, (uint64_t)update, ORC_STREAM_PERM, (uint64_t)epoch * E + i);
    int j = (int)uni(h, (uint32_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
}

/* ---- batched helpers over envs (threads over envs; each env independent) ---- */
int orc_batch_reset(const orc_cfg* c, int E, uint8_t* grids, int32_t* dists, int32_t* states) {
  int bad = 0;
  size_t G = (size_t)c->grid_max * c->grid_max;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
  for (int e = 0; e < E; ++e)
    bad |= orc_reset_env(c, e, 0, grids + G * e, dists + G * e, states + S_NSTATE * e) != 0;
  return bad ? -1 : 0;
}

int orc_batch_step(const orc_cfg* c, int E, uint8_t* grids, int32_t* dists, int32_t* states,
                   const int32_t* actions, float* reward, uint8_t* done, float* spl,
                   int32_t* info) {
  int bad = 0;
  size_t G = (size_t)c->grid_max * c->grid_max;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
  for (int e = 0; e < E; ++e)
    bad |= orc_step_env(c, e, grids + G * e, dists + G * e, states + S_NSTATE * e, actions[e],
                        reward + e, done + e, spl + e, info + 4 * e) != 0;
  return bad ? -1 : 0;
}

void orc_batch_render(const orc_cfg* c, int E, const uint8_t* grids, const int32_t* states,
                      double* depth, double* goal) {
  size_t G = (size_t)c->grid_max * c->grid_max;
  size_t P = (size_t)c->depth_h * c->depth_w;
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < E; ++e) {
    orc_render_depth(c, grids + G * e, states + S_NSTATE * e, depth + P * e);
    orc_goal_vector(states + S_NSTATE * e, goal + 3 * e);
  }
}
