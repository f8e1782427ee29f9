// Batched PointGoal simulator on occupancy grids (arXiv:1911.00357, Sec. 4).
//
//   reset_kernel  : one CTA per env. Scene generation (counter-hash Bernoulli walls or
//                   recursive rooms and doors), a bit-parallel BFS geodesic field from
//                   the goal held in shared memory, and the start/goal/heading draw.
//   step_kernel   : one thread per env. Integer fixed-point motion (0.25 m forward,
//                   10 degree turns, Sec. 4 "Agent"), exact segment-vs-cell collision,
//                   geodesic reward (Sec. 4 "Training"), success/SPL (Sec. 4 "PointGoal
//                   Navigation"), episode end, reset request.
//   render_kernel : one CTA per env, one thread per image column. The env's bit-packed
//                   grid is staged into shared memory by a bulk TMA copy; each thread
//                   marches its column ray cell by cell (DDA with the crossing parameter
//                   recomputed from the boundary plane), then writes the column's z-depth
//                   against the analytic floor and ceiling, fused with the optional 2x2
//                   average pool, the 1/max_depth normalisation and the cast to the
//                   encoder's dtype; thread 0 writes the egocentric goal vector.
//
// Every integer quantity (grid, BFS distances, positions, rewards, done, SPL) is exact;
// depth and the goal vector are FP32.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace ddppo {

__constant__ int2 c_fwd[36];
__constant__ float c_cos[36];
__constant__ float c_sin[36];

int sim_upload_tables() {
  int2 fwd[36];
  float cs[36], sn[36];
  for (int k = 0; k < 36; ++k) {
    double a = (double)k * 10.0 * M_PI / 180.0;
    fwd[k].x = (int)llround(2500.0 * cos(a));
    fwd[k].y = (int)llround(2500.0 * sin(a));
    cs[k] = (float)cos(a);
    sn[k] = (float)sin(a);
  }
  DDPPO_CHECK_CUDA(cudaMemcpyToSymbol(c_fwd, fwd, sizeof(fwd)));
  DDPPO_CHECK_CUDA(cudaMemcpyToSymbol(c_cos, cs, sizeof(cs)));
  DDPPO_CHECK_CUDA(cudaMemcpyToSymbol(c_sin, sn, sizeof(sn)));
  return DDPPO_OK;
}

// ---- counter hash: SplitMix64 (Steele, Lea, Flood 2014) output function, chained ----
__device__ __forceinline__ uint64_t sm64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t chash(uint64_t seed, uint64_t env, uint64_t ep, uint32_t stream,
                                          uint64_t idx) {
  uint64_t k = sm64(seed);
  k = sm64(k + env);
  k = sm64(k + ep);
  return sm64(k + (((uint64_t)stream << 40) | (idx & 0xFFFFFFFFFFull)));
}
__device__ __forceinline__ uint32_t uni(uint64_t h, uint32_t n) {
  return (uint32_t)(((h >> 32) * (uint64_t)n) >> 32);
}
enum : uint32_t { SM_GRID = 1, SM_ROOMS = 2, SM_GOAL = 3, SM_START = 4, SM_HEAD = 5, SM_SIZE = 6 };

__device__ __forceinline__ int grid_side(const SimParams& p, int env, int64_t ep) {
  if (p.nsizes <= 1) return p.grid_min;
  return p.grid_min << uni(chash(p.seed, env, ep, SM_SIZE, 0), (uint32_t)p.nsizes);
}

// scene buffers of env e in slot sl (0 / 1)
__device__ __forceinline__ size_t slot_index(const SimParams& p, int e, int sl) {
  return (size_t)sl * p.E + e;
}
__device__ __forceinline__ size_t cur_index(const SimParams& p, const SimBuffers& b, int e) {
  return slot_index(p, e, b.slot[e]);
}

__device__ __forceinline__ void set_err(int32_t* err, int32_t f) {
  if (err) atomicOr(err, f);
}

// ---- block-wide exclusive scan of one int per thread (blockDim multiple of 32) ----
__device__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;  // inclusive per warp
  }
  __syncthreads();
  int base = wid > 0 ? sh[wid - 1] : 0;
  *total = sh[nw - 1];
  __syncthreads();
  return base + x - v;
}

// ---- bit-parallel 4-connected BFS from cell `goal` over free bits Fw ----
// One level per iteration: next = dilate(frontier) & free & ~visited, 32 cells per word.
// The level loop is capped: at G + 1 levels (more than any BFS of a G-cell grid needs),
// or at `level_cap` when that is positive (a test setting that makes the cap run out).
// A run-out sets the sticky timeout flag and leaves the cells not reached at -1.
__device__ void bfs_block(const uint32_t* __restrict__ Fw, uint32_t* Vw, uint32_t* A, uint32_t* B,
                          int32_t* dist, int g, int goal, int32_t* err, int level_cap) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int G = g * g, R = g >> 5, NW = G >> 5;
  for (int i = tid; i < G; i += nt) dist[i] = -1;
  for (int w = tid; w < NW; w += nt) { Vw[w] = 0u; A[w] = 0u; }
  __syncthreads();
  if (tid == 0) {
    Vw[goal >> 5] = 1u << (goal & 31);
    A[goal >> 5] = 1u << (goal & 31);
    dist[goal] = 0;
  }
  __syncthreads();
  int level = 0;
  bool finished = false;
  const int max_levels = level_cap > 0 && level_cap <= G ? level_cap : G + 1;
  for (int it = 0; it < max_levels; ++it) {
    ++level;
    int any = 0;
    for (int w = tid; w < NW; w += nt) {
      const int y = w / R, wx = w - y * R;
      const uint32_t a = A[w];
      const uint32_t l = wx > 0 ? A[w - 1] : 0u;
      const uint32_t r = wx < R - 1 ? A[w + 1] : 0u;
      const uint32_t u = y > 0 ? A[w - R] : 0u;
      const uint32_t d = y < g - 1 ? A[w + R] : 0u;
      uint32_t n = ((a << 1) | (l >> 31) | (a >> 1) | (r << 31) | u | d) & Fw[w] & ~Vw[w];
      B[w] = n;
      if (n) {
        any = 1;
        Vw[w] |= n;
        const int base = w << 5;
        while (n) {
          const int b = __ffs(n) - 1;
          n &= n - 1;
          dist[base + b] = level;
        }
      }
    }
    any = __syncthreads_or(any);
    uint32_t* t = A; A = B; B = t;
    if (!any) { finished = true; break; }
  }
  if (!finished && tid == 0) set_err(err, ERRF_TIMEOUT);
  __syncthreads();
}

// ---- rooms and doors: recursive binary split, depth first, second child popped first ----
__device__ int rooms_segments(const SimParams& p, int env, int64_t ep, int g, int4* segs, int* stk) {
  int sp = 0, nseg = 0;
  stk[0] = 1; stk[1] = 1; stk[2] = g - 1; stk[3] = g - 1;
  sp = 1;
  uint64_t node = 0;
  const int M = p.min_room;
  while (sp > 0) {
    --sp;
    const int x0 = stk[4 * sp], y0 = stk[4 * sp + 1], x1 = stk[4 * sp + 2], y1 = stk[4 * sp + 3];
    const uint64_t n = node++;
    const int w = x1 - x0, h = y1 - y0;
    const bool vert = w >= h;
    const int span = vert ? w : h, other = vert ? h : w;
    if (span < 2 * M + 1) continue;
    const uint64_t hp = chash(p.seed, env, ep, SM_ROOMS, 2 * n);
    const uint64_t hd = chash(p.seed, env, ep, SM_ROOMS, 2 * n + 1);
    const int lo0 = vert ? x0 : y0;
    const int pos = lo0 + M + (int)uni(hp, (uint32_t)(span - 2 * M));
    const int olo = vert ? y0 : x0, ohi = vert ? y1 : x1;
    const int D = p.door_cells < other ? p.door_cells : other;
    const int dlo = olo + (int)uni(hd, (uint32_t)(other - D + 1));
    if (nseg >= p.max_segs || sp + 2 > 256) return -1;
    segs[nseg++] = make_int4(vert ? 0 : 1, pos, olo | (ohi << 16), dlo | ((dlo + D) << 16));
    if (vert) {
      stk[4 * sp] = x0; stk[4 * sp + 1] = y0; stk[4 * sp + 2] = pos; stk[4 * sp + 3] = y1; ++sp;
      stk[4 * sp] = pos + 1; stk[4 * sp + 1] = y0; stk[4 * sp + 2] = x1; stk[4 * sp + 3] = y1; ++sp;
    } else {
      stk[4 * sp] = x0; stk[4 * sp + 1] = y0; stk[4 * sp + 2] = x1; stk[4 * sp + 3] = pos; ++sp;
      stk[4 * sp] = x0; stk[4 * sp + 1] = pos + 1; stk[4 * sp + 2] = x1; stk[4 * sp + 3] = y1; ++sp;
    }
  }
  return nseg;
}

constexpr int RESET_THREADS = 512;

size_t reset_smem_bytes(const SimParams& p) {
  size_t words = (size_t)p.grid_max * p.grid_max / 32;
  return 4 * words * sizeof(uint32_t) + 256 * 4 * sizeof(int) + 32 * sizeof(int);
}

// Block-wide generation of an episode of env e into scene slot sl: the scene of episode
// `episode` (or of the next ones, up to 8 draws, when a scene has no valid start), its
// BFS geodesic field, and the start state written to st_out. smem holds
// reset_smem_bytes(p) bytes. Callers read whatever they need of the env's state before
// the call; st_out may be the env's own state.
__device__ void gen_episode(const SimParams& p, const SimBuffers& b, int e, int64_t episode, int sl,
                            int32_t* st, uint32_t* smem) {
  const int WMAX = p.grid_max * p.grid_max / 32;
  uint32_t* Fw = smem;
  uint32_t* Vw = Fw + WMAX;
  uint32_t* A = Vw + WMAX;
  uint32_t* B = A + WMAX;
  int* stk = (int*)(B + WMAX);
  int* scan_sh = stk + 256 * 4;
  __shared__ int s_nseg, s_sel;

  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t GM = (size_t)p.grid_max * p.grid_max;
  const size_t si_ = slot_index(p, e, sl);
  uint8_t* grid = b.grids + GM * si_;
  uint32_t* bits = b.bits + (size_t)WMAX * si_;
  int32_t* dist = b.dists + GM * si_;
  __syncthreads();  // every thread has read the caller's state before thread 0 may rewrite it

  for (int tries = 0; tries < 8; ++tries, ++episode) {
    const int g = grid_side(p, e, episode);
    const int G = g * g, NW = G >> 5;
    // 1. scene
    if (p.gen_kind == 0) {
      for (int i = tid; i < G; i += nt) {
        const int x = i % g, y = i / g;
        const bool border = x == 0 || y == 0 || x == g - 1 || y == g - 1;
        const uint32_t u24 = (uint32_t)(chash(p.seed, e, episode, SM_GRID, (uint64_t)i) >> 40);
        grid[i] = (uint8_t)(border || u24 < p.wall_thr24);
      }
    } else {
      for (int i = tid; i < G; i += nt) {
        const int x = i % g, y = i / g;
        grid[i] = (uint8_t)(x == 0 || y == 0 || x == g - 1 || y == g - 1);
      }
      if (tid == 0) s_nseg = rooms_segments(p, e, episode, g, b.segs + (size_t)p.max_segs * e, stk);
      __syncthreads();
      int nseg = s_nseg;
      if (nseg < 0) {
        if (tid == 0) set_err(b.err, ERRF_BOUNDS);
        nseg = 0;
      }
      const int4* segs = b.segs + (size_t)p.max_segs * e;
      for (int s = tid; s < nseg; s += nt) {
        const int4 sg = segs[s];
        const int lo = sg.z & 0xFFFF, hi = sg.z >> 16, dlo = sg.w & 0xFFFF, dhi = sg.w >> 16;
        for (int q = lo; q < hi; ++q) {
          const uint8_t wall = (uint8_t)!(q >= dlo && q < dhi);
          if (sg.x == 0) grid[q * g + sg.y] = wall;
          else grid[sg.y * g + q] = wall;
        }
      }
    }
    __syncthreads();
    // 2. wall bits (global copy for the renderer) and free bits (shared, for BFS)
    for (int w = tid; w < NW; w += nt) {
      uint32_t m = 0u;
      const uint8_t* cell = grid + (w << 5);
      for (int k = 0; k < 32; ++k) m |= (uint32_t)(cell[k] != 0) << k;
      bits[w] = m;
      Fw[w] = ~m;
    }
    __syncthreads();
    // 3. goal, BFS, start
    for (int a = 0; a < 64; ++a) {
      const int gi = (int)uni(chash(p.seed, e, episode, SM_GOAL, (uint64_t)a), (uint32_t)G);
      if (grid[gi]) continue;
      bfs_block(Fw, Vw, A, B, dist, g, gi, b.err, p.bfs_level_cap);
      const int chunk = (G + nt - 1) / nt;
      const int lo = min(G, tid * chunk), hi = min(G, lo + chunk);
      int cnt = 0;
      for (int i = lo; i < hi; ++i) cnt += dist[i] >= p.min_start_cells;
      int total;
      const int before = block_exclusive_scan(cnt, scan_sh, &total);
      if (total == 0) continue;
      const int k = (int)uni(chash(p.seed, e, episode, SM_START, (uint64_t)a), (uint32_t)total);
      if (k >= before && k < before + cnt) {
        int r = k - before;
        for (int i = lo; i < hi; ++i)
          if (dist[i] >= p.min_start_cells) {
            if (r == 0) { s_sel = i; break; }
            --r;
          }
      }
      __syncthreads();
      if (tid == 0) {
        const int si = s_sel, cs = p.cell_u, half = cs / 2;
        st[ST_X] = (si % g) * cs + half;
        st[ST_Y] = (si / g) * cs + half;
        st[ST_HEAD] = (int)uni(chash(p.seed, e, episode, SM_HEAD, (uint64_t)a), 36u);
        st[ST_STEPS] = 0;
        st[ST_PATH] = 0;
        st[ST_GEO_START] = dist[si] * cs;
        st[ST_GEO_PREV] = dist[si] * cs;
        st[ST_GOAL_X] = (gi % g) * cs + half;
        st[ST_GOAL_Y] = (gi / g) * cs + half;
        st[ST_EPISODE] = (int32_t)episode;
        st[ST_GRID] = g;
        st[ST_COLLIDED] = 0;
      }
      if (p.task == TASK_FLEE) {
        // Flee measures geodesics from the start: the slot's field becomes the BFS from
        // the start cell (the goal field was needed only to draw the start), and Max(s_0)
        // is its largest entry
        const int si = s_sel;
        __syncthreads();  // thread 0 has read the goal field for the start state
        bfs_block(Fw, Vw, A, B, dist, g, si, b.err, p.bfs_level_cap);
        __shared__ int s_mx;
        if (tid == 0) s_mx = 0;
        __syncthreads();
        int mx = 0;
        for (int i = tid; i < G; i += nt) mx = max(mx, dist[i]);
        atomicMax(&s_mx, mx);
        __syncthreads();
        if (tid == 0) {
          b.tmax[si_] = s_mx;
          st[ST_GEO_PREV] = 0;
        }
      }
      return;
    }
  }
  // no valid episode in 8 scene draws: flag it and park the agent on the goal-free state
  if (tid == 0) {
    set_err(b.err, ERRF_RESET);
    const int g = grid_side(p, e, episode - 1), cs = p.cell_u;
    st[ST_X] = cs + cs / 2; st[ST_Y] = cs + cs / 2; st[ST_HEAD] = 0; st[ST_STEPS] = 0;
    st[ST_PATH] = 0; st[ST_GEO_START] = 0; st[ST_GEO_PREV] = 0; st[ST_GOAL_X] = st[ST_X];
    st[ST_GOAL_Y] = st[ST_Y]; st[ST_EPISODE] = (int32_t)episode; st[ST_GRID] = g; st[ST_COLLIDED] = 0;
  }
}

// Exploration: the visited squares of env e's new episode are its start square alone
__device__ void explore_begin(const SimParams& p, const SimBuffers& b, int e) {
  if (p.task != TASK_EXPLORE) return;  // uniform over the block
  uint32_t* vw = b.visited + (size_t)e * p.vis_words;
  for (int w = threadIdx.x; w < p.vis_words; w += blockDim.x) vw[w] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int32_t* st = b.states + (size_t)ST_N * e;
    const int sq = (st[ST_Y] / p.explore_u) * p.vis_side + st[ST_X] / p.explore_u;
    vw[sq >> 5] |= 1u << (sq & 31);
  }
  __syncthreads();
}

// the episode that follows env e's current one: the prepared slot when ready, else
// generated now into the other slot
__device__ void next_episode(const SimParams& p, const SimBuffers& b, int e, uint32_t* smem) {
  int32_t* st = b.states + (size_t)ST_N * e;
  const int tid = threadIdx.x;
  const int ready = b.ready[e], sl = b.slot[e];
  const int64_t ep = (int64_t)st[ST_EPISODE] + 1;
  __syncthreads();
  if (ready) {
    if (tid < ST_N) st[tid] = b.pend[(size_t)ST_N * e + tid];
  } else {
    gen_episode(p, b, e, ep, sl ^ 1, st, smem);
  }
  __syncthreads();
  if (tid == 0) {
    b.slot[e] = (uint8_t)(sl ^ 1);
    b.ready[e] = 0;
  }
  __syncthreads();
  explore_begin(p, b, e);
}

__global__ void __launch_bounds__(RESET_THREADS) reset_kernel(SimParams p, SimBuffers b, int all) {
  DDPPO_PDL_ENTRY();
  const int e = blockIdx.x;
  if (e >= p.E) return;
  if (!all && !b.need[e]) return;
  extern __shared__ __align__(16) uint32_t smem[];
  if (all) {
    gen_episode(p, b, e, 0, 0, b.states + (size_t)ST_N * e, smem);
    __syncthreads();
    if (threadIdx.x == 0) {
      b.slot[e] = 0;
      b.ready[e] = 0;
    }
    explore_begin(p, b, e);
  } else {
    next_episode(p, b, e, smem);
  }
}

int launch_reset(const SimParams& p, const SimBuffers& b, bool all, cudaStream_t s) {
  ::ddppo::launch_k(reset_kernel, p.E, RESET_THREADS, reset_smem_bytes(p), s, p, b, all ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- exact closed-segment vs closed-cell-square test (separating axes, int64) ----
__device__ __forceinline__ bool seg_meets_cell(int64_t x0, int64_t y0, int64_t x1, int64_t y1,
                                               int64_t cx, int64_t cy, int64_t cs) {
  const int64_t bx0 = cx * cs, bx1 = bx0 + cs, by0 = cy * cs, by1 = by0 + cs;
  const int64_t sx0 = min(x0, x1), sx1 = max(x0, x1), sy0 = min(y0, y1), sy1 = max(y0, y1);
  if (sx1 < bx0 || sx0 > bx1 || sy1 < by0 || sy0 > by1) return false;
  const int64_t dx = x1 - x0, dy = y1 - y0;
  int pos = 0, neg = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t qx = (i & 1) ? bx1 : bx0, qy = (i & 2) ? by1 : by0;
    const int64_t cr = dx * (qy - y0) - dy * (qx - x0);
    pos += cr > 0;
    neg += cr < 0;
  }
  return !(pos == 4 || neg == 4);
}

__device__ __forceinline__ int floordiv(int a, int b) {
  int q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Blocked iff some wall (or outside) cell among those whose square can meet the
// segment's bounding box touches the segment.
__device__ bool segment_blocked(const uint8_t* grid, int g, int cs, int x0, int y0, int x1, int y1) {
  const int cx0 = floordiv(min(x0, x1), cs) - 1, cx1 = floordiv(max(x0, x1), cs);
  const int cy0 = floordiv(min(y0, y1), cs) - 1, cy1 = floordiv(max(y0, y1), cs);
  for (int cy = cy0; cy <= cy1; ++cy)
    for (int cx = cx0; cx <= cx1; ++cx) {
      const bool wall = (cx < 0 || cy < 0 || cx >= g || cy >= g) ? true : grid[cy * g + cx] != 0;
      if (wall && seg_meets_cell(x0, y0, x1, y1, cx, cy, cs)) return true;
    }
  return false;
}

// one env step (thread-level); returns 1 when the episode ended
__device__ int step_env(const SimParams& p, const SimBuffers& b, int e,
                        const int32_t* __restrict__ actions, float* __restrict__ reward,
                        uint8_t* __restrict__ done, float* __restrict__ info) {
  int32_t* st = b.states + (size_t)ST_N * e;
  const size_t ci = cur_index(p, b, e);
  const uint8_t* grid = b.grids + (size_t)p.grid_max * p.grid_max * ci;
  const int32_t* dist = b.dists + (size_t)p.grid_max * p.grid_max * ci;
  int a = actions[e];
  if (a < 0 || a > 3) { set_err(b.err, ERRF_BOUNDS); a = 0; }
  const int g = st[ST_GRID], cs = p.cell_u;
  int x = st[ST_X], y = st[ST_Y], k = st[ST_HEAD], steps = st[ST_STEPS] + 1, path = st[ST_PATH];
  int success = 0, finished = 0, collided = 0;
  if (a == 0) {
    const int64_t dx = (int64_t)st[ST_GOAL_X] - x, dy = (int64_t)st[ST_GOAL_Y] - y;
    success = dx * dx + dy * dy <= (int64_t)2000 * 2000;
    finished = 1;
  } else if (a == 1) {
    const int2 f = c_fwd[k];
    const int nx = x + f.x, ny = y + f.y;
    if (segment_blocked(grid, g, cs, x, y, nx, ny)) {
      collided = 1;
    } else {
      x = nx; y = ny; path += 2500;
    }
  } else if (a == 2) {
    k = k == 35 ? 0 : k + 1;
  } else {
    k = k == 0 ? 35 : k - 1;
  }
  const int cx = x / cs, cy = y / cs;
  int32_t dcell = -1;
  if (cx >= 0 && cy >= 0 && cx < g && cy < g) dcell = dist[cy * g + cx];
  else set_err(b.err, ERRF_BOUNDS);
  const int32_t geo_new = dcell * cs;
  int64_t r = (int64_t)st[ST_GEO_PREV] - geo_new - 100;
  float task_r = 0.0f;
  if (p.task == TASK_FLEE) {
    // 5 (D_t - D_t-1) with D = Geo(s, s_0) / Max(s_0): in cells, one rounded division
    const int32_t d0 = st[ST_GEO_PREV] / cs, mx = b.tmax[ci];
    task_r = mx > 0 ? (float)((double)(5 * (dcell - d0)) / (double)mx) : 0.0f;
  } else if (p.task == TASK_EXPLORE) {
    uint32_t* vw = b.visited + (size_t)e * p.vis_words;
    const int sq = (y / p.explore_u) * p.vis_side + x / p.explore_u;
    const uint32_t bit = 1u << (sq & 31);
    task_r = (vw[sq >> 5] & bit) ? 0.0f : 0.25f;
    vw[sq >> 5] |= bit;
  }
  const int64_t l = st[ST_GEO_START], pl = path, m = l > pl ? l : pl;
  if (success) {
    if (p.terminal_mode == 0) r += 25000;
    else r += (2 * 25000 * l + m) / (2 * m);
  }
  if (!finished && steps >= p.max_steps) finished = 1;
  st[ST_X] = x; st[ST_Y] = y; st[ST_HEAD] = k; st[ST_STEPS] = steps; st[ST_PATH] = path;
  st[ST_GEO_PREV] = geo_new; st[ST_COLLIDED] = collided;
  reward[e] = p.task == TASK_POINTGOAL ? (float)r / 10000.0f : task_r;
  done[e] = (uint8_t)finished;
  b.need[e] = (uint8_t)finished;
  if (info) {
    info[4 * e + 0] = (float)success;
    info[4 * e + 1] = success ? (float)l / (float)m : 0.0f;
    info[4 * e + 2] = (float)collided;
    info[4 * e + 3] = (float)steps;
  }
  return finished;
}

__global__ void step_kernel(SimParams p, SimBuffers b, const int32_t* __restrict__ actions,
                            float* __restrict__ reward, uint8_t* __restrict__ done,
                            float* __restrict__ info) {
  DDPPO_PDL_ENTRY();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.E) return;
  step_env(p, b, e, actions, reward, done, info);
}

int launch_step(const SimParams& p, const SimBuffers& b, const int32_t* actions, float* reward,
                uint8_t* done, float* info, cudaStream_t s) {
  const int th = 128;
  ::ddppo::launch_k(step_kernel, (p.E + th - 1) / th, th, 0, s, p, b, actions, reward, done, info);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- ray-cast depth ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Render env e with the whole block: TMA bulk copy of the bit-packed grid into smem (the
// mbarrier `bar` completes phase `phase`), then one column ray per thread (looping when
// the image is wider than the block), depth against the analytic planes, the optional
// 2x2 pool, normalisation and cast; thread 0 writes the goal vector. Returns false (the
// same for every thread) when the wait for the copy ran out: the timeout flag is set,
// nothing is rendered, and the caller must not reuse `sbits` or `bar` -- the copy may
// still land there.
__device__ bool render_env_block(const SimParams& p, const SimBuffers& b, int e,
                                 void* __restrict__ obs, float* __restrict__ goal,
                                 float* __restrict__ depth_raw, uint32_t* sbits, uint64_t* mbar,
                                 uint32_t phase) {
  const int tid = threadIdx.x;
  const int32_t* st = b.states + (size_t)ST_N * e;
  const int g = st[ST_GRID];
  const int WMAX = p.grid_max * p.grid_max / 32;
  const uint32_t bytes = (uint32_t)(g * g / 8);
  const uint32_t bar = smem_u32(mbar);
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sbits)),
        "l"(b.bits + (size_t)WMAX * cur_index(p, b, e)), "r"(bytes), "r"(bar)
        : "memory");
  }
  uint32_t ok = 0;
  for (int it = 0; it < (1 << 24) && !ok; ++it) {
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
  }
  if (!__syncthreads_and(ok)) {
    if (tid == 0) set_err(b.err, ERRF_TIMEOUT);
    return false;
  }
  const int cs = p.cell_u;
  const int k = st[ST_HEAD];
  const float c = c_cos[k], s = c_sin[k];
  const float px = (float)st[ST_X], py = (float)st[ST_Y];
  const int R = g >> 5;
  const float up = p.ceil_h - p.cam_h, H = (float)p.H;
  if (tid == 0 && goal) {
    const float gx = (float)(st[ST_GOAL_X] - st[ST_X]) * 1e-4f;
    const float gy = (float)(st[ST_GOAL_Y] - st[ST_Y]) * 1e-4f;
    const float f = gx * c + gy * s, l = -gx * s + gy * c;
    const float r = sqrtf(gx * gx + gy * gy);
    goal[3 * e + 0] = r;
    goal[3 * e + 1] = r > 0.f ? f / r : 1.0f;
    goal[3 * e + 2] = r > 0.f ? l / r : 0.0f;
  }
  float* raw = depth_raw ? depth_raw + (size_t)e * p.H * p.W : nullptr;
  const float inv_max = 1.0f / p.max_depth;
  for (int i = tid; i < p.W; i += blockDim.x) {
    // column ray: forward + x_i * right, right = (sin, -cos)
    const float xi = (float)(2 * i + 1) / (float)p.W - 1.0f;
    const float dx = c + xi * s, dy = s - xi * c;
    int cx = st[ST_X] / cs, cy = st[ST_Y] / cs;
    const int sx = dx > 0.f ? 1 : (dx < 0.f ? -1 : 0);
    const int sy = dy > 0.f ? 1 : (dy < 0.f ? -1 : 0);
    float t = INFINITY;
    for (int it = 0; it < 8 * g + 8; ++it) {
      const float tx = sx ? ((float)((cx + (sx > 0)) * cs) - px) / dx : INFINITY;
      const float ty = sy ? ((float)((cy + (sy > 0)) * cs) - py) / dy : INFINITY;
      float tc;
      if (tx <= ty) { cx += sx; tc = tx; } else { cy += sy; tc = ty; }
      if (cx < 0 || cy < 0 || cx >= g || cy >= g) break;
      if ((sbits[cy * R + (cx >> 5)] >> (cx & 31)) & 1u) { t = tc; break; }
    }
    const float tw = t * 1e-4f;  // metres
    for (int j = 0; j < p.H; j += 2) {
      float d2[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const float yj = 1.0f - (float)(2 * (j + q) + 1) / H;
        const float tp = yj > 0.f ? up / yj : p.cam_h / (-yj);
        float d = fminf(tw, tp);
        d = fminf(d, p.max_depth);
        d = fmaxf(d, 0.0f);
        d2[q] = d;
        if (raw) raw[(size_t)(j + q) * p.W + i] = d;
      }
      if (obs) {
        if (p.pool) {
          const float sum = d2[0] + d2[1];
          const float other = __shfl_xor_sync(0xffffffffu, sum, 1);
          if ((i & 1) == 0) {
            const float v = (sum + other) * 0.25f * inv_max;
            const size_t o = ((size_t)e * p.obs_h + (j >> 1)) * p.obs_w + (i >> 1);
            if (p.bf16_obs) ((__nv_bfloat16*)obs)[o] = __float2bfloat16_rn(v);
            else ((float*)obs)[o] = v;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const size_t o = ((size_t)e * p.obs_h + j + q) * p.obs_w + i;
            const float v = d2[q] * inv_max;
            if (p.bf16_obs) ((__nv_bfloat16*)obs)[o] = __float2bfloat16_rn(v);
            else ((float*)obs)[o] = v;
          }
        }
      }
    }
  }
  return true;
}

__global__ void render_kernel(SimParams p, SimBuffers b, void* __restrict__ obs,
                              float* __restrict__ goal, float* __restrict__ depth_raw) {
  DDPPO_PDL_ENTRY();
  extern __shared__ __align__(128) uint32_t sbits[];
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  render_env_block(p, b, blockIdx.x, obs, goal, depth_raw, sbits, &mbar, 0);
}

// One persistent launch for the whole env step: CTAs take envs from an atomic work
// counter (so a CTA stuck on an expensive reset -- a BFS over a 512x512 grid -- does not
// hold up the others), and per env do: step (thread 0); if the episode ended, the
// block-wide reset of the next episode; the TMA-staged render of the new frame. The last
// CTA to finish re-arms the counter for the next launch (graph replays included).
__global__ void __launch_bounds__(RESET_THREADS)
    env_step_persistent_kernel(SimParams p, SimBuffers b, const int32_t* __restrict__ actions,
                               void* __restrict__ obs, float* __restrict__ goal,
                               float* __restrict__ reward, uint8_t* __restrict__ done,
                               float* __restrict__ info) {
  DDPPO_PDL_ENTRY();
  extern __shared__ __align__(128) uint32_t smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int s_env, s_fin;
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  for (int guard = 0; guard <= p.E; ++guard) {
    if (tid == 0) s_env = atomicAdd(&b.work[0], 1);
    __syncthreads();
    const int e = s_env;
    if (e >= p.E) break;
    if (tid == 0) s_fin = step_env(p, b, e, actions, reward, done, info);
    __syncthreads();
    if (s_fin) {
      next_episode(p, b, e, smem);
      // new wall bits may have been written through the generic proxy; the TMA copy that
      // reads them next goes through the async proxy
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    __syncthreads();
    // a copy that did not arrive may still land in smem: this CTA takes no further env
    // (the others drain the work counter; the sticky flag reports the run-out)
    if (!render_env_block(p, b, e, obs, goal, nullptr, smem, &mbar, phase)) break;
    phase ^= 1u;
    __syncthreads();  // smem is reused by the next env
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&b.work[1], 1) == (int)gridDim.x - 1) {
      b.work[0] = 0;
      b.work[1] = 0;
      __threadfence();
    }
  }
}

// Prefetch: CTAs take envs from a second self-re-arming work counter and generate the
// next episode of every env whose other slot is not ready. Runs beside the policy's
// forward pass; the next env step adopts the prepared slot instead of generating it.
__global__ void __launch_bounds__(RESET_THREADS) env_prefetch_kernel(SimParams p, SimBuffers b) {
  DDPPO_PDL_ENTRY();
  extern __shared__ __align__(128) uint32_t smem[];
  __shared__ int s_env;
  const int tid = threadIdx.x;
  for (int guard = 0; guard <= p.E; ++guard) {
    if (tid == 0) s_env = atomicAdd(&b.work[2], 1);
    __syncthreads();
    const int e = s_env;
    __syncthreads();
    if (e >= p.E) break;
    if (b.ready[e]) continue;
    const int32_t* st = b.states + (size_t)ST_N * e;
    const int64_t ep = (int64_t)st[ST_EPISODE] + 1;
    gen_episode(p, b, e, ep, b.slot[e] ^ 1, b.pend + (size_t)ST_N * e, smem);
    __syncthreads();
    if (tid == 0) b.ready[e] = 1;
  }
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&b.work[3], 1) == (int)gridDim.x - 1) {
      b.work[2] = 0;
      b.work[3] = 0;
      __threadfence();
    }
  }
}

int launch_env_prefetch(const SimParams& p, const SimBuffers& b, int grid, cudaStream_t s) {
  ::ddppo::launch_k(env_prefetch_kernel, grid, RESET_THREADS, reset_smem_bytes(p), s, p, b);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void copy_current_kernel(SimParams p, SimBuffers b, uint8_t* __restrict__ grids,
                                    int32_t* __restrict__ dists) {
  DDPPO_PDL_ENTRY();
  const int e = blockIdx.y;
  const size_t GM = (size_t)p.grid_max * p.grid_max, ci = cur_index(p, b, e);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < GM;
       i += (size_t)gridDim.x * blockDim.x) {
    if (grids) grids[GM * e + i] = b.grids[GM * ci + i];
    if (dists) dists[GM * e + i] = b.dists[GM * ci + i];
  }
}

int launch_copy_current(const SimParams& p, const SimBuffers& b, uint8_t* grids, int32_t* dists,
                        cudaStream_t s) {
  if (p.E > 65535) { set_error("env_grids: too many envs"); return DDPPO_E_CONFIG; }
  const size_t GM = (size_t)p.grid_max * p.grid_max;
  const unsigned bx = (unsigned)std::min<size_t>((GM + 255) / 256, 64);
  ::ddppo::launch_k(copy_current_kernel, dim3(bx, p.E), 256, 0, s, p, b, grids, dists);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_env_step(const SimParams& p, const SimBuffers& b, int grid, const int32_t* actions,
                    void* obs, float* goal, float* reward, uint8_t* done, float* info,
                    cudaStream_t s) {
  const size_t smem = max(reset_smem_bytes(p), (size_t)p.grid_max * p.grid_max / 8);
  ::ddppo::launch_k(env_step_persistent_kernel, grid, RESET_THREADS, smem, s, p, b, actions, obs, goal, reward,
                                                               done, info);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_render(const SimParams& p, const SimBuffers& b, void* obs, float* goal, float* depth_raw,
                  cudaStream_t s) {
  const size_t smem = (size_t)p.grid_max * p.grid_max / 8;
  ::ddppo::launch_k(render_kernel, p.E, p.W, smem, s, p, b, obs, goal, depth_raw);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo

namespace ddppo {
int sim_configure(const SimParams& p) {
  const size_t rs = reset_smem_bytes(p);
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(reset_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)rs));
  const size_t gs = (size_t)p.grid_max * p.grid_max / 8;
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(render_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)gs));
  const size_t ps = rs > gs ? rs : gs;
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(env_step_persistent_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ps));
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(env_prefetch_kernel,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rs));
  return DDPPO_OK;
}

int env_step_grid(const SimParams& p, int num_sms) {
  const size_t rs = reset_smem_bytes(p), gs = (size_t)p.grid_max * p.grid_max / 8;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, env_step_persistent_kernel,
                                                    RESET_THREADS, rs > gs ? rs : gs) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  const int g = per_sm * num_sms;
  return g < p.E ? g : p.E;
}
}  // namespace ddppo
