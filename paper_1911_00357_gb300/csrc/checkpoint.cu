// Checkpoint and resume of a worker (ddppo_save / ddppo_load).
//
// The paper trains for days on many machines and relies on its cluster's preemption and
// restart (Sec. 3 runs under SLURM; Sec. 4 "Training": 2.5 billion frames), so a worker's
// whole learning state has to survive a restart. A checkpoint holds everything that
// decides the rest of a run, so that a resumed run is bit-identical to an uninterrupted
// one:
//   - the FP32 parameters, both Adam moments and the Adam step count;
//   - the world: both scene slots of every env (grid, wall bits, BFS field), the agent
//     states, the prepared next episodes (start state, slot index, ready flag), and the
//     transfer tasks' per-episode state (Flee's Max(s_0), Exploration's visited squares);
//   - the delayed activation scales of FP8 inference;
//   - the GEMM autotuner's table (a re-tuned table could choose split-K for a shape the
//     saved run reduced in one pass, which changes the bits of the sums);
//   - optionally, the rollout state carried into the next collect: slot T of the
//     observation, goal, previous action and mask, and the LSTM state h, c.
// The file is a sequence of tagged, sized sections after a header holding the
// configuration; ddppo_load checks that the configuration and every section size match.
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "net.cuh"

namespace ddppo {
int net_prep_weights(Net& n, cudaStream_t s);
}  // namespace ddppo

using namespace ddppo;

namespace {

constexpr char kMagic[8] = {'D', 'D', 'P', 'P', 'O', 'C', 'K', 'P'};
constexpr uint32_t kVersion = 1;

enum : uint32_t {
  SEC_PARAMS = 1, SEC_ADAM_M, SEC_ADAM_V, SEC_ADAM_T, SEC_GRIDS, SEC_BITS, SEC_DISTS,
  SEC_STATES, SEC_PEND, SEC_SLOT, SEC_READY, SEC_FLAGS, SEC_F8_SCALE, SEC_F8_AMAX, SEC_TUNER,
  SEC_RO_OBS, SEC_RO_GOAL, SEC_RO_PREVA, SEC_RO_MASKS, SEC_RO_H, SEC_RO_C, SEC_TMAX, SEC_VISITED,
  SEC_END = 0xFFFFFFFFu
};

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

int fail(int code, const std::string& msg) {
  set_error("checkpoint: " + msg);
  return code;
}

// one section: tag, byte count, bytes (device memory copied through the host)
int put(FILE* f, uint32_t tag, const void* src, size_t bytes, bool device, cudaStream_t s) {
  std::vector<uint8_t> h(bytes);
  if (bytes && device) {
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(h.data(), src, bytes, cudaMemcpyDeviceToHost, s));
    DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
  } else if (bytes) {
    memcpy(h.data(), src, bytes);
  }
  const uint64_t n = bytes;
  if (fwrite(&tag, 4, 1, f) != 1 || fwrite(&n, 8, 1, f) != 1 ||
      (bytes && fwrite(h.data(), 1, bytes, f) != bytes))
    return fail(DDPPO_E_ARG, "write failed");
  return DDPPO_OK;
}

int get(FILE* f, uint32_t tag, void* dst, size_t bytes, bool device, cudaStream_t s) {
  uint32_t t = 0;
  uint64_t n = 0;
  if (fread(&t, 4, 1, f) != 1 || fread(&n, 8, 1, f) != 1)
    return fail(DDPPO_E_CONFIG, "truncated file");
  if (t != tag) return fail(DDPPO_E_CONFIG, "section " + std::to_string(t) + " where " +
                                               std::to_string(tag) + " was expected");
  if (n != bytes) return fail(DDPPO_E_CONFIG, "section " + std::to_string(tag) + " holds " +
                                                 std::to_string(n) + " bytes, expected " +
                                                 std::to_string(bytes));
  std::vector<uint8_t> h(bytes);
  if (bytes && fread(h.data(), 1, bytes, f) != bytes) return fail(DDPPO_E_CONFIG, "truncated file");
  if (bytes && device) {
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(dst, h.data(), bytes, cudaMemcpyHostToDevice, s));
    DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
  } else if (bytes) {
    memcpy(dst, h.data(), bytes);
  }
  return DDPPO_OK;
}

// sizes of the world sections
struct Sizes {
  size_t E, GM, P, L, H, ob;
};

Sizes sizes(const ddppo_ctx* x) {
  const Net& n = *x->net;
  Sizes z;
  z.E = (size_t)x->cfg.num_envs;
  z.GM = (size_t)x->cfg.grid_max * x->cfg.grid_max;
  z.P = (size_t)n.P;
  z.L = (size_t)n.L;
  z.H = (size_t)n.H;
  z.ob = n.pix * (n.bf ? 2 : 4);
  return z;
}

}  // namespace

extern "C" int ddppo_save(ddppo_ctx* x, const ddppo_rollout* ro, const char* path, void* stream) {
  if (!x || !x->net || !path) return fail(DDPPO_E_ARG, "null argument");
  if (ro && !(ro->obs && ro->goal && ro->prev_a && ro->masks && ro->h && ro->c))
    return fail(DDPPO_E_ARG, "rollout view has a null buffer");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  const Sizes z = sizes(x);
  File F;
  F.f = fopen(path, "wb");
  if (!F.f) return fail(DDPPO_E_ARG, std::string("cannot open ") + path + " for writing");
  FILE* f = F.f;
  const uint32_t ver = kVersion, cfg_bytes = sizeof(ddppo_config);
  if (fwrite(kMagic, 1, 8, f) != 8 || fwrite(&ver, 4, 1, f) != 1 || fwrite(&cfg_bytes, 4, 1, f) != 1 ||
      fwrite(&x->cfg, sizeof(ddppo_config), 1, f) != 1)
    return fail(DDPPO_E_ARG, "write failed");
  DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));  // the state of every enqueued call
  DDPPO_TRY(put(f, SEC_PARAMS, n.params, z.P * 4, true, s));
  DDPPO_TRY(put(f, SEC_ADAM_M, n.adam_m, z.P * 4, true, s));
  DDPPO_TRY(put(f, SEC_ADAM_V, n.adam_v, z.P * 4, true, s));
  DDPPO_TRY(put(f, SEC_ADAM_T, &n.adam_t, 8, false, s));
  DDPPO_TRY(put(f, SEC_GRIDS, x->sb.grids, 2 * z.E * z.GM, true, s));
  DDPPO_TRY(put(f, SEC_BITS, x->sb.bits, 2 * z.E * z.GM / 32 * 4, true, s));
  DDPPO_TRY(put(f, SEC_DISTS, x->sb.dists, 2 * z.E * z.GM * 4, true, s));
  DDPPO_TRY(put(f, SEC_STATES, x->sb.states, z.E * ST_N * 4, true, s));
  DDPPO_TRY(put(f, SEC_PEND, x->sb.pend, z.E * ST_N * 4, true, s));
  DDPPO_TRY(put(f, SEC_SLOT, x->sb.slot, z.E, true, s));
  DDPPO_TRY(put(f, SEC_READY, x->sb.ready, z.E, true, s));
  DDPPO_TRY(put(f, SEC_TMAX, x->sb.tmax, x->cfg.task == 1 ? 2 * z.E * 4 : 0, true, s));
  DDPPO_TRY(put(f, SEC_VISITED, x->sb.visited, z.E * (size_t)x->sp.vis_words * 4, true, s));
  const int32_t flags[3] = {x->env_ready ? 1 : 0, n.collect_started ? 1 : 0, n.T_last};
  DDPPO_TRY(put(f, SEC_FLAGS, flags, sizeof(flags), false, s));
  DDPPO_TRY(put(f, SEC_F8_SCALE, n.f8_scale, (size_t)n.f8_slots * 4, true, s));
  DDPPO_TRY(put(f, SEC_F8_AMAX, n.f8_amax, (size_t)n.f8_slots * 4, true, s));
  const size_t tb = tc_tuner_export(n.gws.tuner, nullptr, 0);
  std::vector<uint8_t> tbuf(tb);
  if (tb) tc_tuner_export(n.gws.tuner, tbuf.data(), tb);
  DDPPO_TRY(put(f, SEC_TUNER, tbuf.data(), tb, false, s));
  if (ro) {
    const size_t oT = (size_t)x->cfg.rollout_T * z.E;
    DDPPO_TRY(put(f, SEC_RO_OBS, (const char*)ro->obs + oT * z.ob, z.E * z.ob, true, s));
    DDPPO_TRY(put(f, SEC_RO_GOAL, ro->goal + oT * 3, z.E * 12, true, s));
    DDPPO_TRY(put(f, SEC_RO_PREVA, ro->prev_a + oT, z.E * 4, true, s));
    DDPPO_TRY(put(f, SEC_RO_MASKS, ro->masks + oT, z.E, true, s));
    DDPPO_TRY(put(f, SEC_RO_H, ro->h, z.L * z.E * z.H * 4, true, s));
    DDPPO_TRY(put(f, SEC_RO_C, ro->c, z.L * z.E * z.H * 4, true, s));
  }
  DDPPO_TRY(put(f, SEC_END, nullptr, 0, false, s));
  if (fflush(f) != 0) return fail(DDPPO_E_ARG, "write failed");
  return DDPPO_OK;
}

extern "C" int ddppo_load(ddppo_ctx* x, const ddppo_rollout* ro, const char* path, void* stream) {
  if (!x || !x->net || !path) return fail(DDPPO_E_ARG, "null argument");
  if (ro && !(ro->obs && ro->goal && ro->prev_a && ro->masks && ro->h && ro->c))
    return fail(DDPPO_E_ARG, "rollout view has a null buffer");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  const Sizes z = sizes(x);
  File F;
  F.f = fopen(path, "rb");
  if (!F.f) return fail(DDPPO_E_ARG, std::string("cannot open ") + path);
  FILE* f = F.f;
  char magic[8];
  uint32_t ver = 0, cfg_bytes = 0;
  ddppo_config cfg{};
  if (fread(magic, 1, 8, f) != 8 || memcmp(magic, kMagic, 8) != 0)
    return fail(DDPPO_E_CONFIG, "not a checkpoint of this library");
  if (fread(&ver, 4, 1, f) != 1 || ver != kVersion || fread(&cfg_bytes, 4, 1, f) != 1 ||
      cfg_bytes != sizeof(ddppo_config))
    return fail(DDPPO_E_CONFIG, "unsupported checkpoint version");
  if (fread(&cfg, sizeof(cfg), 1, f) != 1) return fail(DDPPO_E_CONFIG, "truncated file");
  if (memcmp(&cfg, &x->cfg, sizeof(cfg)) != 0)
    return fail(DDPPO_E_CONFIG, "the checkpoint was written by a worker with another configuration");
  DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
  DDPPO_TRY(get(f, SEC_PARAMS, n.params, z.P * 4, true, s));
  DDPPO_TRY(get(f, SEC_ADAM_M, n.adam_m, z.P * 4, true, s));
  DDPPO_TRY(get(f, SEC_ADAM_V, n.adam_v, z.P * 4, true, s));
  int64_t adam_t = 0;
  DDPPO_TRY(get(f, SEC_ADAM_T, &adam_t, 8, false, s));
  DDPPO_TRY(get(f, SEC_GRIDS, x->sb.grids, 2 * z.E * z.GM, true, s));
  DDPPO_TRY(get(f, SEC_BITS, x->sb.bits, 2 * z.E * z.GM / 32 * 4, true, s));
  DDPPO_TRY(get(f, SEC_DISTS, x->sb.dists, 2 * z.E * z.GM * 4, true, s));
  DDPPO_TRY(get(f, SEC_STATES, x->sb.states, z.E * ST_N * 4, true, s));
  DDPPO_TRY(get(f, SEC_PEND, x->sb.pend, z.E * ST_N * 4, true, s));
  DDPPO_TRY(get(f, SEC_SLOT, x->sb.slot, z.E, true, s));
  DDPPO_TRY(get(f, SEC_READY, x->sb.ready, z.E, true, s));
  DDPPO_TRY(get(f, SEC_TMAX, x->sb.tmax, x->cfg.task == 1 ? 2 * z.E * 4 : 0, true, s));
  DDPPO_TRY(get(f, SEC_VISITED, x->sb.visited, z.E * (size_t)x->sp.vis_words * 4, true, s));
  int32_t flags[3] = {0, 0, 0};
  DDPPO_TRY(get(f, SEC_FLAGS, flags, sizeof(flags), false, s));
  // the GEMM-layout (and E4M3) weight copies follow the loaded parameters; the FP8
  // activation scales are restored after, since the weight preparation leaves them alone
  DDPPO_TRY(net_prep_weights(n, s));
  DDPPO_TRY(get(f, SEC_F8_SCALE, n.f8_scale, (size_t)n.f8_slots * 4, true, s));
  DDPPO_TRY(get(f, SEC_F8_AMAX, n.f8_amax, (size_t)n.f8_slots * 4, true, s));
  {
    uint32_t t = 0;
    uint64_t tb = 0;
    if (fread(&t, 4, 1, f) != 1 || t != SEC_TUNER || fread(&tb, 8, 1, f) != 1)
      return fail(DDPPO_E_CONFIG, "missing tuning table");
    std::vector<uint8_t> tbuf(tb);
    if (tb && fread(tbuf.data(), 1, tb, f) != tb) return fail(DDPPO_E_CONFIG, "truncated file");
    if (tb && n.gws.tuner) DDPPO_TRY(tc_tuner_import(n.gws.tuner, tbuf.data(), tb));
  }
  uint32_t next = 0;
  long pos = ftell(f);
  if (fread(&next, 4, 1, f) != 1) return fail(DDPPO_E_CONFIG, "truncated file");
  fseek(f, pos, SEEK_SET);
  const bool has_ro = next == SEC_RO_OBS;
  if (ro && !has_ro) return fail(DDPPO_E_CONFIG, "the checkpoint holds no rollout state");
  if (has_ro) {
    if (!ro) return fail(DDPPO_E_ARG, "the checkpoint holds rollout state: pass the rollout view");
    const size_t oT = (size_t)x->cfg.rollout_T * z.E;
    DDPPO_TRY(get(f, SEC_RO_OBS, (char*)ro->obs + oT * z.ob, z.E * z.ob, true, s));
    DDPPO_TRY(get(f, SEC_RO_GOAL, ro->goal + oT * 3, z.E * 12, true, s));
    DDPPO_TRY(get(f, SEC_RO_PREVA, ro->prev_a + oT, z.E * 4, true, s));
    DDPPO_TRY(get(f, SEC_RO_MASKS, ro->masks + oT, z.E, true, s));
    DDPPO_TRY(get(f, SEC_RO_H, ro->h, z.L * z.E * z.H * 4, true, s));
    DDPPO_TRY(get(f, SEC_RO_C, ro->c, z.L * z.E * z.H * 4, true, s));
  }
  DDPPO_TRY(get(f, SEC_END, nullptr, 0, false, s));
  n.adam_t = adam_t;
  x->env_ready = flags[0] != 0;
  n.collect_started = flags[1] != 0 && has_ro;
  n.T_last = flags[2];
  n.ev_valid = false;
  return DDPPO_OK;
}
