// Network entry points (placeholder until the network kernels land).
#include "ctx.cuh"

namespace ddppo {
int net_create(ddppo_ctx*) { return DDPPO_OK; }
void net_destroy(ddppo_ctx*) {}
}  // namespace ddppo

static int not_built() {
  ddppo::set_error("network path not built");
  return DDPPO_E_CONFIG;
}
extern "C" {
int ddppo_num_params(const ddppo_ctx*, int64_t*) { return not_built(); }
int ddppo_get_params(ddppo_ctx*, float*, int64_t, void*) { return not_built(); }
int ddppo_set_params(ddppo_ctx*, const float*, int64_t, void*) { return not_built(); }
int ddppo_get_adam(ddppo_ctx*, float*, float*, int64_t, int64_t*, void*) { return not_built(); }
int ddppo_policy_act(ddppo_ctx*, const void*, const float*, const int32_t*, const uint8_t*, float*,
                     float*, const float*, int32_t*, float*, float*, void*) { return not_built(); }
int ddppo_policy_evaluate(ddppo_ctx*, int32_t, int32_t, const void*, const float*, const int32_t*,
                          const uint8_t*, const float*, const float*, float*, float*, void*) {
  return not_built();
}
int ddppo_policy_backward(ddppo_ctx*, const float*, const float*, float*, void*) { return not_built(); }
int ddppo_ppo_loss(int32_t, const float*, const float*, const int32_t*, const float*, const float*,
                   const float*, float, float, float, float*, float*, float*, void*) {
  return not_built();
}
int ddppo_ppo_update(ddppo_ctx*, const ddppo_rollout*, const ddppo_ppo_hparams*, float*, void*) {
  return not_built();
}
int ddppo_collect(ddppo_ctx*, const ddppo_rollout*, int32_t, void*) { return not_built(); }
int ddppo_timing_enable(ddppo_ctx*, int32_t) { return not_built(); }
int ddppo_timing_read(ddppo_ctx*, int32_t, double*, int64_t*, double*) { return not_built(); }
}
