// C ABI of the library (include/ddppo.h): argument checking, the worker context,
// and the environment / GAE entry points. The network and update entry points are in
// net_abi.cu.
#include <math.h>
#include <stdio.h>

#include <mutex>
#include <string>

#include <atomic>
#include <cstdlib>

#include "net.cuh"

namespace ddppo {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

}  // namespace ddppo

using namespace ddppo;

#define ARG_CHECK(cond, msg)            \
  do {                                  \
    if (!(cond)) {                      \
      set_error(std::string("ddppo: ") + msg); \
      return DDPPO_E_ARG;               \
    }                                   \
  } while (0)
#define CFG_CHECK(cond, msg)            \
  do {                                  \
    if (!(cond)) {                      \
      set_error(std::string("ddppo config: ") + msg); \
      return DDPPO_E_CONFIG;            \
    }                                   \
  } while (0)

extern "C" const char* ddppo_last_error(void) { return g_last_error.c_str(); }

namespace ddppo {
// launch overlap (programmatic dependent launch): on unless DDPPO_LAUNCH_OVERLAP=0
static std::atomic<int> g_pdl{-1};
bool pdl_enabled() {
  int v = g_pdl.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("DDPPO_LAUNCH_OVERLAP");
    v = (e && e[0] == '0') ? 0 : 1;
    g_pdl.store(v, std::memory_order_relaxed);
  }
  return v != 0;
}
// tensor-store epilogue of the tcgen05 GEMM: on unless DDPPO_TMA_EPILOGUE=0
static std::atomic<int> g_tma_epi{-1};
bool tma_epilogue_enabled() {
  int v = g_tma_epi.load(std::memory_order_relaxed);
  if (v < 0) {
    const char* e = getenv("DDPPO_TMA_EPILOGUE");
    v = (e && e[0] == '0') ? 0 : 1;
    g_tma_epi.store(v, std::memory_order_relaxed);
  }
  return v != 0;
}
}  // namespace ddppo

extern "C" int ddppo_set_tma_epilogue(int32_t on) {
  ddppo::g_tma_epi.store(on ? 1 : 0, std::memory_order_relaxed);
  return DDPPO_OK;
}

extern "C" int ddppo_tma_epilogue(int32_t* on) {
  if (!on) {
    ddppo::set_error("tma_epilogue: null argument");
    return DDPPO_E_ARG;
  }
  *on = ddppo::tma_epilogue_enabled() ? 1 : 0;
  return DDPPO_OK;
}

extern "C" int ddppo_set_launch_overlap(int32_t on) {
  ddppo::g_pdl.store(on ? 1 : 0, std::memory_order_relaxed);
  return DDPPO_OK;
}

extern "C" int ddppo_launch_overlap(int32_t* on) {
  if (!on) {
    ddppo::set_error("launch_overlap: null argument");
    return DDPPO_E_ARG;
  }
  *on = ddppo::pdl_enabled() ? 1 : 0;
  return DDPPO_OK;
}

static bool pow2_multiple(int a, int b) {
  if (a <= 0 || b < a || b % a) return false;
  int q = b / a;
  return (q & (q - 1)) == 0;
}

static int validate(const ddppo_config* c) {
  CFG_CHECK(c->num_envs >= 1 && c->num_envs <= (1 << 16), "num_envs must be in [1, 65536]");
  CFG_CHECK(c->gen_kind == 0 || c->gen_kind == 1, "gen_kind must be 0 or 1");
  CFG_CHECK(c->grid_min >= 32 && c->grid_max <= 512 && c->grid_min % 32 == 0 &&
                pow2_multiple(c->grid_min, c->grid_max),
            "grid sides must be multiples of 32 in [32, 512], grid_max = grid_min * 2^j");
  CFG_CHECK(c->cell_m >= 0.01f && c->cell_m <= 1.0f, "cell_m must be in [0.01, 1]");
  CFG_CHECK(c->wall_density >= 0.f && c->wall_density <= 1.f, "wall_density must be in [0, 1]");
  CFG_CHECK(c->gen_kind == 0 || (c->min_room >= 2 && c->door_m > 0.f), "rooms need min_room >= 2");
  CFG_CHECK(c->max_steps >= 1, "max_steps must be >= 1");
  CFG_CHECK(c->terminal_mode == 0 || c->terminal_mode == 1, "terminal_mode must be 0 or 1");
  CFG_CHECK(c->depth_h == c->depth_w && c->depth_w >= 32 && c->depth_w <= 1024 &&
                c->depth_w % 32 == 0,
            "depth must be square, a multiple of 32, at most 1024");
  CFG_CHECK(c->pool2x2 == 0 || c->pool2x2 == 1, "pool2x2 must be 0 or 1");
  CFG_CHECK(c->max_depth_m > 0.f && c->ceil_h_m > c->cam_h_m && c->cam_h_m > 0.f,
            "camera must sit between floor and ceiling");
  CFG_CHECK(c->net_kind >= 0 && c->net_kind <= 4,
            "net_kind must be 0 (3-layer conv), 1 (ResNet), 2 (blind), 3 (SE-ResNeXt50) or 4 "
            "(SE-ResNeXt101)");
  CFG_CHECK(c->net_kind < 3 || c->base_ch == 16 || c->base_ch == 32,
            "SE-ResNeXt base_ch must be 16 or 32 (32 groups of at most 16 channels)");
  CFG_CHECK(c->precision >= 0 && c->precision <= 2,
            "precision must be 0 (fp32), 1 (bf16) or 2 (fp8 inference, bf16 training)");
  CFG_CHECK(c->precision != 2 || (c->net_kind == 1 && c->base_ch % 64 == 0),
            "fp8 inference needs the ResNet encoder with a base width that is a multiple of 64");
  CFG_CHECK(c->lstm_layers >= 1 && c->lstm_layers <= 4, "lstm_layers must be in [1, 4]");
  CFG_CHECK(c->hidden >= 8 && c->hidden % 8 == 0 && c->hidden <= 2048,
            "hidden must be a multiple of 8 in [8, 2048]");
  CFG_CHECK(c->net_kind != 1 || (c->base_ch >= 4 && c->base_ch % 4 == 0 && c->base_ch <= 128),
            "base_ch must be a multiple of 4 in [4, 128]");
  CFG_CHECK(c->rollout_T >= 1 && c->rollout_T <= 4096, "rollout_T must be in [1, 4096]");
  CFG_CHECK(c->minibatches >= 1 && c->num_envs % c->minibatches == 0,
            "minibatches must divide num_envs");
  CFG_CHECK(c->encoder_chunk >= 0, "encoder_chunk must be >= 0");
  CFG_CHECK(c->task >= 0 && c->task <= 2, "task must be 0 (PointGoal), 1 (Flee) or 2 (Exploration)");
  CFG_CHECK(c->task != 2 || (c->explore_m >= c->cell_m && c->explore_m <= 100.f),
            "explore_m must be in [cell_m, 100]");
  return DDPPO_OK;
}

static SimParams make_sim_params(const ddppo_config* c) {
  SimParams p{};
  p.E = c->num_envs;
  p.gen_kind = c->gen_kind;
  p.grid_min = c->grid_min;
  p.grid_max = c->grid_max;
  p.nsizes = 0;
  for (int s = c->grid_min; s <= c->grid_max; s *= 2) ++p.nsizes;
  p.cell_u = (int)llround((double)c->cell_m * 10000.0);
  p.wall_thr24 = (uint32_t)floor((double)c->wall_density * 16777216.0);
  p.door_cells = c->gen_kind == 1 ? (int)llround((double)c->door_m / (double)c->cell_m) : 1;
  if (p.door_cells < 1) p.door_cells = 1;
  p.min_room = c->min_room;
  p.max_steps = c->max_steps;
  p.terminal_mode = c->terminal_mode;
  p.min_start_cells = (20000 + p.cell_u - 1) / p.cell_u;
  p.H = c->depth_h;
  p.W = c->depth_w;
  p.pool = c->pool2x2;
  p.obs_h = c->depth_h >> c->pool2x2;
  p.obs_w = c->depth_w >> c->pool2x2;
  p.cam_h = c->cam_h_m;
  p.ceil_h = c->ceil_h_m;
  p.max_depth = c->max_depth_m;
  p.seed = c->seed;
  p.max_segs = c->gen_kind == 1
                   ? (c->grid_max - 2) * (c->grid_max - 2) / (c->min_room * c->min_room) + 1
                   : 0;
  p.bf16_obs = c->precision >= 1;
  p.task = c->task;
  if (c->task == 2) {
    p.explore_u = (int)llround((double)c->explore_m * 10000.0);
    // squares per side: positions lie in [0, grid_max * cell_u)
    p.vis_side = (c->grid_max * p.cell_u + p.explore_u - 1) / p.explore_u;
    p.vis_words = (p.vis_side * p.vis_side + 31) / 32;
  }
  return p;
}

template <class T>
static int dmalloc(T** p, size_t n) {
  if (n == 0) { *p = nullptr; return DDPPO_OK; }
  DDPPO_CHECK_CUDA(cudaMalloc((void**)p, n * sizeof(T)));
  return DDPPO_OK;
}

namespace ddppo {
void ctx_free_world(ddppo_ctx* x) {
  cudaFree(x->sb.grids); cudaFree(x->sb.bits); cudaFree(x->sb.dists); cudaFree(x->sb.states);
  cudaFree(x->sb.pend); cudaFree(x->sb.slot); cudaFree(x->sb.ready);
  cudaFree(x->sb.segs); cudaFree(x->sb.need); cudaFree(x->sb.err); cudaFree(x->sb.work);
  cudaFree(x->sb.tmax); cudaFree(x->sb.visited);
  if (x->ev_fork) cudaEventDestroy(x->ev_fork);
  if (x->ev_join) cudaEventDestroy(x->ev_join);
  if (x->side) cudaStreamDestroy(x->side);
}
}  // namespace ddppo

extern "C" int ddppo_config_check(const ddppo_config* cfg) {
  ARG_CHECK(cfg != nullptr, "ddppo_config_check: null argument");
  return validate(cfg);
}

extern "C" int ddppo_create(const ddppo_config* cfg, ddppo_ctx** out) {
  ARG_CHECK(cfg != nullptr && out != nullptr, "ddppo_create: null argument");
  DDPPO_TRY(validate(cfg));
  ddppo_ctx* x = new ddppo_ctx();
  x->cfg = *cfg;
  x->sp = make_sim_params(cfg);
  int rc = DDPPO_OK;
  do {
    if (cudaGetDevice(&x->device) != cudaSuccess) { set_error("no CUDA device"); rc = DDPPO_E_CUDA; break; }
    if ((rc = sim_upload_tables()) != DDPPO_OK) break;
    if ((rc = sim_configure(x->sp)) != DDPPO_OK) break;
    const size_t E = cfg->num_envs, GM = (size_t)cfg->grid_max * cfg->grid_max;
    if ((rc = dmalloc(&x->sb.grids, 2 * E * GM)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.bits, 2 * E * GM / 32)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.dists, 2 * E * GM)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.states, E * ST_N)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.pend, E * ST_N)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.slot, E)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.ready, E)) != DDPPO_OK) break;
    if (cudaMemset(x->sb.slot, 0, E) != cudaSuccess || cudaMemset(x->sb.ready, 0, E) != cudaSuccess) {
      set_error("cudaMemset failed"); rc = DDPPO_E_CUDA; break;
    }
    if (cudaStreamCreateWithFlags(&x->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      set_error("stream/event creation failed"); rc = DDPPO_E_CUDA; break;
    }
    if ((rc = dmalloc(&x->sb.segs, E * (size_t)x->sp.max_segs)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.tmax, cfg->task == 1 ? 2 * E : 0)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.visited, E * (size_t)x->sp.vis_words)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.need, E)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.err, 1)) != DDPPO_OK) break;
    if ((rc = dmalloc(&x->sb.work, 4)) != DDPPO_OK) break;
    if (cudaMemset(x->sb.work, 0, 4 * sizeof(int32_t)) != cudaSuccess) { set_error("cudaMemset failed"); rc = DDPPO_E_CUDA; break; }
    {
      int nsm = 152;
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, x->device);
      x->env_grid = env_step_grid(x->sp, nsm);
      // half the SMs at most: the prefetch runs beside the policy's forward pass
      x->prefetch_grid = std::max(1, std::min(cfg->num_envs, nsm / 2));
    }
    if (cudaMemset(x->sb.err, 0, sizeof(int32_t)) != cudaSuccess ||
        cudaMemset(x->sb.need, 0, E) != cudaSuccess ||
        cudaMemset(x->sb.states, 0, E * ST_N * sizeof(int32_t)) != cudaSuccess) {
      set_error("cudaMemset failed"); rc = DDPPO_E_CUDA; break;
    }
    if ((rc = net_create(x)) != DDPPO_OK) break;
    if (cudaDeviceSynchronize() != cudaSuccess) { set_error("create: device sync failed"); rc = DDPPO_E_CUDA; break; }
  } while (0);
  if (rc != DDPPO_OK) {
    net_destroy(x);
    ctx_free_world(x);
    delete x;
    return rc;
  }
  *out = x;
  return DDPPO_OK;
}

extern "C" int ddppo_destroy(ddppo_ctx* x) {
  if (!x) return DDPPO_OK;
  cudaDeviceSynchronize();
  net_destroy(x);
  ctx_free_world(x);
  delete x;
  return DDPPO_OK;
}

extern "C" int ddppo_device_status(ddppo_ctx* x, int32_t* code_out, void* stream) {
  ARG_CHECK(x && code_out, "device_status: null argument");
  int32_t w = 0;
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(&w, x->sb.err, sizeof(w), cudaMemcpyDeviceToHost, s));
  DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
  if (w & ERRF_BOUNDS) *code_out = DDPPO_E_DEVICE_BOUNDS;
  else if (w & ERRF_TIMEOUT) *code_out = DDPPO_E_TIMEOUT;
  else if (w & ERRF_RESET) *code_out = DDPPO_E_CONFIG;
  else *code_out = DDPPO_OK;
  return DDPPO_OK;
}

extern "C" int ddppo_set_bfs_level_cap(ddppo_ctx* x, int32_t cap) {
  ARG_CHECK(x, "set_bfs_level_cap: null ctx");
  ARG_CHECK(cap >= 0, "set_bfs_level_cap: negative cap");
  x->sp.bfs_level_cap = cap;
  return DDPPO_OK;
}

// ---- environment ----
extern "C" int ddppo_env_reset(ddppo_ctx* x, void* obs, float* goal, void* stream) {
  ARG_CHECK(x && obs && goal, "env_reset: null argument");
  ARG_CHECK(((uintptr_t)obs & 15) == 0 && ((uintptr_t)goal & 3) == 0, "env_reset: misaligned");
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_TRY(launch_reset(x->sp, x->sb, true, s));
  DDPPO_TRY(launch_render(x->sp, x->sb, obs, goal, nullptr, s));
  x->env_ready = true;
  return DDPPO_OK;
}

extern "C" int ddppo_env_step(ddppo_ctx* x, const int32_t* actions, void* obs, float* goal,
                              float* reward, uint8_t* done, float* info, void* stream) {
  ARG_CHECK(x && actions && obs && goal && reward && done, "env_step: null argument");
  if (!x->env_ready) { set_error("env_step before env_reset"); return DDPPO_E_STATE; }
  cudaStream_t s = (cudaStream_t)stream;
  KernelTimer* t = x->net ? &x->net->rc_timer : nullptr;
  const bool rec = t && t->on && t->n + 2 <= 2 * 4096;
  if (rec) cudaEventRecord(t->ev[t->n], s);
  DDPPO_TRY(launch_env_step(x->sp, x->sb, x->env_grid, actions, obs, goal, reward, done, info, s));
  if (rec) {
    cudaEventRecord(t->ev[t->n + 1], s);
    // algorithmic bytes: the encoder input written plus the goal vectors
    const double out = (double)x->cfg.num_envs *
                       ((double)x->sp.obs_h * x->sp.obs_w * (x->sp.bf16_obs ? 2 : 4) + 12.0);
    t->work[t->n / 2] = out;
    t->bytes[t->n / 2] = out;
    t->n += 2;
    t->launches += 1;
    t->flops += out;
  }
  return DDPPO_OK;
}

extern "C" int ddppo_env_prefetch(ddppo_ctx* x, void* stream) {
  ARG_CHECK(x, "env_prefetch: null ctx");
  if (!x->env_ready) { set_error("env_prefetch before env_reset"); return DDPPO_E_STATE; }
  return launch_env_prefetch(x->sp, x->sb, x->prefetch_grid, (cudaStream_t)stream);
}

extern "C" int ddppo_env_state(ddppo_ctx* x, int32_t* state, void* stream) {
  ARG_CHECK(x && state, "env_state: null argument");
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(state, x->sb.states,
                                   sizeof(int32_t) * ST_N * x->cfg.num_envs,
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return DDPPO_OK;
}

extern "C" int ddppo_env_set_state(ddppo_ctx* x, const int32_t* state, void* stream) {
  ARG_CHECK(x && state, "env_set_state: null argument");
  if (!x->env_ready) { set_error("env_set_state before env_reset"); return DDPPO_E_STATE; }
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(x->sb.states, state, sizeof(int32_t) * ST_N * x->cfg.num_envs,
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  // prepared next episodes were drawn for the replaced episode counters
  DDPPO_CHECK_CUDA(cudaMemsetAsync(x->sb.ready, 0, x->cfg.num_envs, (cudaStream_t)stream));
  return DDPPO_OK;
}

extern "C" int ddppo_env_grids(ddppo_ctx* x, uint8_t* grids, int32_t* dists, void* stream) {
  ARG_CHECK(x, "env_grids: null ctx");
  if (!grids && !dists) return DDPPO_OK;
  return launch_copy_current(x->sp, x->sb, grids, dists, (cudaStream_t)stream);
}

extern "C" int ddppo_env_depth(ddppo_ctx* x, float* depth, void* stream) {
  ARG_CHECK(x && depth, "env_depth: null argument");
  if (!x->env_ready) { set_error("env_depth before env_reset"); return DDPPO_E_STATE; }
  return launch_render(x->sp, x->sb, nullptr, nullptr, depth, (cudaStream_t)stream);
}

// ---- GAE ----
extern "C" int ddppo_gae(const float* reward, const uint8_t* done, const float* value, int32_t T,
                         int32_t E, float gamma, float lam, float* adv, float* ret, void* stream) {
  ARG_CHECK(T >= 0 && E >= 0, "gae: negative size");
  if (T == 0 || E == 0) return DDPPO_OK;
  ARG_CHECK(reward && done && value && adv && ret, "gae: null argument");
  return launch_gae(reward, done, value, T, E, gamma, lam, adv, ret, (cudaStream_t)stream);
}
