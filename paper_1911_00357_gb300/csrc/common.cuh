// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

#include <string>

#include "../../include/ddppo.h"

namespace ddppo {

// ---- error reporting (thread-local message, status codes of ddppo.h) ----
void set_error(const std::string& msg);
#define DDPPO_CHECK_CUDA(expr)                                                        \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess) {                                                          \
      ::ddppo::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return DDPPO_E_CUDA;                                                            \
    }                                                                                 \
  } while (0)
#define DDPPO_CHECK_LAUNCH() DDPPO_CHECK_CUDA(cudaGetLastError())
#define DDPPO_TRY(expr)              \
  do {                               \
    int _rc = (expr);                \
    if (_rc != DDPPO_OK) return _rc; \
  } while (0)

// ---- programmatic dependent launch ----
// Every kernel of the library is launched through launch_k with the programmatic
// stream-serialization attribute: its blocks may become resident while the previous kernel
// in the stream is still running, which hides the launch gap and the block prologue.
// DDPPO_PDL_ENTRY() therefore comes before a kernel's first global-memory access (read or
// write): griddepcontrol.wait returns once the previous kernel has completed and its
// writes are visible (a no-op without a programmatic predecessor). The launch_dependents
// after it lets the next kernel's blocks become resident; since a block triggers only after
// its own wait has returned, at most one kernel waits ahead of the running one, and
// kernels that allocate tensor memory do so before the trigger, so a waiting kernel never
// holds columns a running one still needs.
#define DDPPO_PDL_ENTRY() \
  asm volatile("griddepcontrol.wait;\n\tgriddepcontrol.launch_dependents;" ::: "memory")

// process-wide switch (ddppo_set_launch_overlap); graphs captured before a change keep the
// form they were captured with
bool pdl_enabled();
// process-wide switch (ddppo_set_tma_epilogue): tensor-core GEMM tiles whose rows are whole
// output rows leave through a tensor store from shared memory (on) or through the
// transpose and per-row stores (off); bit-identical results either way
bool tma_epilogue_enabled();

template <typename... P, typename... A>
inline void launch_k(void (*kern)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  (void)cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);  // checked by the caller
}

// sticky device error word: bit flags
enum : int32_t { ERRF_BOUNDS = 1, ERRF_TIMEOUT = 2, ERRF_RESET = 4 };
enum : int { TASK_POINTGOAL = 0, TASK_FLEE = 1, TASK_EXPLORE = 2 };

// agent state slots (int32), same meaning as ddppo_env_state
enum {
  ST_X = 0, ST_Y, ST_HEAD, ST_STEPS, ST_PATH, ST_GEO_PREV, ST_GEO_START, ST_GOAL_X,
  ST_GOAL_Y, ST_EPISODE, ST_GRID, ST_COLLIDED, ST_N
};
static_assert(ST_N == DDPPO_NSTATE, "state layout");

// ---- world parameters passed to the simulator kernels by value ----
struct SimParams {
  int E;
  int gen_kind;
  int grid_min, grid_max, nsizes;
  int cell_u;
  uint32_t wall_thr24;
  int door_cells, min_room;
  int max_steps, terminal_mode;
  int min_start_cells;  // ceil(2 m / cell)
  int H, W, pool, obs_h, obs_w;
  float cam_h, ceil_h, max_depth;
  uint64_t seed;
  int max_segs;
  int bf16_obs;
  int bfs_level_cap;  // 0: none (G + 1 levels); > 0: cap the BFS level loop (tests)
  int task;           // 0 PointGoal, 1 Flee, 2 Exploration (the reward of env_step)
  int explore_u;      // Exploration square side (u)
  int vis_side, vis_words;  // Exploration squares per side, bitmap words per env
};

// Every env owns two scene slots: the current episode's and the next one's, which the
// prefetch kernel generates ahead of time (off the critical path of the rollout).
struct SimBuffers {
  uint8_t* grids;     // [2, E, gmax^2]
  uint32_t* bits;     // [2, E, gmax^2/32] wall bits, row-major words
  int32_t* dists;     // [2, E, gmax^2]
  int32_t* states;    // [E, ST_N]
  int32_t* pend;      // [E, ST_N] start state of the prepared next episode
  uint8_t* slot;      // [E] slot of the current episode
  uint8_t* ready;     // [E] 1: the other slot holds the next episode (start state in pend)
  int4* segs;         // [E, max_segs] room walls (gen_kind 1)
  uint8_t* need;      // [E] reset request
  int32_t* err;       // [1] sticky
  int32_t* work;      // [4] env-step and prefetch work counters + CTAs finished (self re-arming)
  int32_t* tmax;      // [2, E] Flee: Max(s_0) (cells) of the episode in each scene slot
  uint32_t* visited;  // [E, vis_words] Exploration: squares visited in the current episode
};

// host-side launchers (sim.cu)
int sim_upload_tables();
size_t reset_smem_bytes(const SimParams& p);
int launch_reset(const SimParams& p, const SimBuffers& b, bool all, cudaStream_t s);
int launch_step(const SimParams& p, const SimBuffers& b, const int32_t* actions, float* reward,
                uint8_t* done, float* info, cudaStream_t s);
int launch_render(const SimParams& p, const SimBuffers& b, void* obs, float* goal, float* depth_raw,
                  cudaStream_t s);
// fused persistent step + auto-reset + render over all envs
int launch_env_step(const SimParams& p, const SimBuffers& b, int grid, const int32_t* actions,
                    void* obs, float* goal, float* reward, uint8_t* done, float* info,
                    cudaStream_t s);
int env_step_grid(const SimParams& p, int num_sms);
// generate the next episode of every env whose other slot is not ready yet
int launch_env_prefetch(const SimParams& p, const SimBuffers& b, int grid, cudaStream_t s);
// copy the current slot's grids / distance fields of every env to dense [E, gmax^2] buffers
int launch_copy_current(const SimParams& p, const SimBuffers& b, uint8_t* grids, int32_t* dists,
                        cudaStream_t s);

// rl.cu
int launch_gae(const float* r, const uint8_t* d, const float* v, int T, int E, float gamma,
               float lam, float* adv, float* ret, cudaStream_t s);

}  // namespace ddppo
