// The worker context behind the opaque ddppo_ctx handle.
#pragma once

#include "common.cuh"

namespace ddppo {
struct Net;
int sim_configure(const SimParams& p);
int net_create(ddppo_ctx* x);
void net_destroy(ddppo_ctx* x);
void ctx_free_world(ddppo_ctx* x);
}  // namespace ddppo

struct ddppo_ctx {
  ddppo_config cfg{};
  ddppo::SimParams sp{};
  ddppo::SimBuffers sb{};
  int device = 0;
  bool env_ready = false;
  int env_grid = 1;  // CTAs of the persistent env-step kernel
  int prefetch_grid = 1;  // CTAs of the next-episode prefetch kernel
  cudaStream_t side = nullptr;  // prefetch stream (forked from and joined to the rollout stream)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ddppo::Net* net = nullptr;
};
