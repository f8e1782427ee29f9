// C ABI entry points of the policy and the learning step (include/ddppo.h): parameters,
// act / evaluate / backward, PPO loss, the PPO update (Sec. 4 "Training") and rollout
// collection captured as a CUDA graph (Sec. 3: the collection stage of the loop).
#include <string.h>

#include <algorithm>
#include <vector>

#include "net.cuh"
#include "nn_kernels.cuh"
#include "rl.cuh"

namespace ddppo {
// infer: an act-time pass (policy_act, the collect loop, the bootstrap value); under FP8
// inference its encoder runs on E4M3 operands
int net_forward(Net& n, int T, int E, const void* obs, const float* goal, const int32_t* prev_a,
                const uint8_t* masks, const float* h0, const float* c0, const float* u,
                int32_t* action, float* logp, cudaStream_t s, bool infer = false);
int net_backward(Net& n, const float* dlogits, const float* dvalues, cudaStream_t s);
int net_prep_weights(Net& n, cudaStream_t s);
int net_encoder_forward(Net& n, int N, const void* obs, float* feat, cudaStream_t s);
int net_encoder_backward(Net& n, const float* dfeat, cudaStream_t s);
int net_lstm_forward(Net& n, int T, int E, const float* x, const uint8_t* masks, const float* h0,
                     const float* c0, float* y, cudaStream_t s);
int net_lstm_backward(Net& n, const float* dy, float* dx, cudaStream_t s);
}  // namespace ddppo

using namespace ddppo;

#define ARG(cond, msg)                                   \
  do {                                                   \
    if (!(cond)) {                                       \
      set_error(std::string("ddppo: ") + (msg));         \
      return DDPPO_E_ARG;                                \
    }                                                    \
  } while (0)

static inline size_t op_bytes(const Net& n) { return n.bf ? 2 : 4; }

extern "C" int ddppo_num_params(const ddppo_ctx* x, int64_t* n_out) {
  ARG(x && x->net && n_out, "num_params: null argument");
  *n_out = x->net->P;
  return DDPPO_OK;
}

extern "C" int ddppo_get_params(ddppo_ctx* x, float* flat, int64_t n, void* stream) {
  ARG(x && x->net && flat, "get_params: null argument");
  ARG(n == x->net->P, "get_params: size mismatch");
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(flat, x->net->params, n * 4, cudaMemcpyDeviceToDevice,
                                   (cudaStream_t)stream));
  return DDPPO_OK;
}

extern "C" int ddppo_set_params(ddppo_ctx* x, const float* flat, int64_t n, void* stream) {
  ARG(x && x->net && flat, "set_params: null argument");
  Net& N = *x->net;
  ARG(n == N.P, "set_params: size mismatch");
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(N.params, flat, n * 4, cudaMemcpyDeviceToDevice, s));
  DDPPO_CHECK_CUDA(cudaMemsetAsync(N.adam_m, 0, n * 4, s));
  DDPPO_CHECK_CUDA(cudaMemsetAsync(N.adam_v, 0, n * 4, s));
  N.adam_t = 0;
  return net_prep_weights(N, s);
}

extern "C" int ddppo_get_adam(ddppo_ctx* x, float* m, float* v, int64_t n, int64_t* step,
                              void* stream) {
  ARG(x && x->net, "get_adam: null ctx");
  Net& N = *x->net;
  ARG(n == N.P, "get_adam: size mismatch");
  cudaStream_t s = (cudaStream_t)stream;
  if (m) DDPPO_CHECK_CUDA(cudaMemcpyAsync(m, N.adam_m, n * 4, cudaMemcpyDeviceToDevice, s));
  if (v) DDPPO_CHECK_CUDA(cudaMemcpyAsync(v, N.adam_v, n * 4, cudaMemcpyDeviceToDevice, s));
  if (step) *step = N.adam_t;
  return DDPPO_OK;
}

// copy the step-0 LSTM state of the last forward into h/c [L, E, H]
static int copy_state_out(Net& n, int E, float* h, float* c, cudaStream_t s) {
  const size_t bytes = (size_t)E * n.H * sizeof(float);
  for (int l = 0; l < n.L; ++l) {
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(h + (size_t)l * E * n.H, n.lstm[l].h, bytes,
                                     cudaMemcpyDeviceToDevice, s));
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(c + (size_t)l * E * n.H, n.lstm[l].c, bytes,
                                     cudaMemcpyDeviceToDevice, s));
  }
  return DDPPO_OK;
}

static int act_impl(ddppo_ctx* x, const void* obs, const float* goal, const int32_t* prev_a,
                    const uint8_t* masks, float* h, float* c, const float* u, int32_t* action,
                    float* logp, float* value, cudaStream_t s) {
  Net& n = *x->net;
  const int E = x->cfg.num_envs;
  DDPPO_TRY(net_forward(n, 1, E, obs, goal, prev_a, masks, h, c, u, action, logp, s, true));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(value, n.values, (size_t)E * 4, cudaMemcpyDeviceToDevice, s));
  n.ev_valid = false;  // the act workspace is not kept for a backward pass
  return copy_state_out(n, E, h, c, s);
}

extern "C" int ddppo_policy_act(ddppo_ctx* x, const void* obs, const float* goal,
                                const int32_t* prev_a, const uint8_t* masks, float* h, float* c,
                                const float* uniforms, int32_t* action, float* logp, float* value,
                                void* stream) {
  ARG(x && x->net && obs && goal && prev_a && masks && h && c && uniforms && action && logp && value,
      "policy_act: null argument");
  return act_impl(x, obs, goal, prev_a, masks, h, c, uniforms, action, logp, value,
                  (cudaStream_t)stream);
}

extern "C" int ddppo_policy_evaluate(ddppo_ctx* x, int32_t T, int32_t E, const void* obs,
                                     const float* goal, const int32_t* prev_a, const uint8_t* masks,
                                     const float* h0, const float* c0, float* logits, float* values,
                                     void* stream) {
  ARG(x && x->net && obs && goal && prev_a && masks && h0 && c0 && logits && values,
      "policy_evaluate: null argument");
  ARG(T >= 1 && E >= 1, "policy_evaluate: empty segment");
  Net& n = *x->net;
  if ((int64_t)T * E > n.NS || E > n.E) {
    set_error("policy_evaluate: T*E exceeds rollout_T*num_envs/minibatches (or E > num_envs)");
    return DDPPO_E_CONFIG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_TRY(net_forward(n, T, E, obs, goal, prev_a, masks, h0, c0, nullptr, nullptr, nullptr, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(logits, n.logits, (size_t)T * E * 16, cudaMemcpyDeviceToDevice, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(values, n.values, (size_t)T * E * 4, cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

extern "C" int ddppo_policy_backward(ddppo_ctx* x, const float* dlogits, const float* dvalues,
                                     float* grad, void* stream) {
  ARG(x && x->net && dlogits && dvalues && grad, "policy_backward: null argument");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_TRY(net_backward(n, dlogits, dvalues, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(grad, n.grad, n.P * 4, cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

extern "C" int ddppo_encoder_forward(ddppo_ctx* x, int32_t N, const void* obs, float* feat,
                                     void* stream) {
  ARG(x && x->net && obs && feat, "encoder_forward: null argument");
  return net_encoder_forward(*x->net, N, obs, feat, (cudaStream_t)stream);
}

extern "C" int ddppo_encoder_backward(ddppo_ctx* x, const float* dfeat, float* grad, void* stream) {
  ARG(x && x->net && dfeat && grad, "encoder_backward: null argument");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_TRY(net_encoder_backward(n, dfeat, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(grad, n.grad, (size_t)n.P * 4, cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

extern "C" int ddppo_lstm_forward(ddppo_ctx* x, int32_t T, int32_t E, const float* in,
                                  const uint8_t* masks, const float* h0, const float* c0, float* y,
                                  void* stream) {
  ARG(x && x->net && in && masks && h0 && c0 && y, "lstm_forward: null argument");
  return net_lstm_forward(*x->net, T, E, in, masks, h0, c0, y, (cudaStream_t)stream);
}

extern "C" int ddppo_lstm_backward(ddppo_ctx* x, const float* dy, float* dx, float* grad,
                                   void* stream) {
  ARG(x && x->net && dy && grad, "lstm_backward: null argument");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_TRY(net_lstm_backward(n, dy, dx, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(grad, n.grad, (size_t)n.P * 4, cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

extern "C" int ddppo_ppo_loss(int32_t n, const float* logits, const float* values,
                              const int32_t* actions, const float* logp_old, const float* adv,
                              const float* ret, float clip, float value_coef, float entropy_coef,
                              float* stats, float* dlogits, float* dvalues, void* stream) {
  ARG(n >= 0, "ppo_loss: negative size");
  if (n == 0) return DDPPO_OK;
  ARG(logits && values && actions && logp_old && adv && ret && stats && dlogits && dvalues,
      "ppo_loss: null argument");
  return launch_ppo_loss(n, logits, values, actions, logp_old, adv, ret, clip, value_coef,
                         entropy_coef, stats, dlogits, dvalues, nullptr, 0, (cudaStream_t)stream);
}

__global__ void set_steps_kernel(int64_t* d, int64_t update_index, int64_t adam_t) {
  DDPPO_PDL_ENTRY();
  d[0] = update_index;
  d[1] = adam_t;
}

// one PPO update (epochs x minibatches) on stream s; the update index and the Adam step
// count are read from n.d_steps, so the same launches replay for every update
static int update_body(ddppo_ctx* x, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                       float* stats, cudaStream_t s) {
  Net& n = *x->net;
  const ddppo_config& c = x->cfg;
  const int T = c.rollout_T, E = c.num_envs, Emb = n.Emb, L = n.L, Hd = n.H;
  const int Nmb = T * Emb;
  const float* adv = ro->adv;
  if (hp->norm_adv) {
    DDPPO_TRY(launch_normalize_adv(ro->adv, n.adv_norm, (size_t)T * E, n.scal, n.scratch,
                                   n.scratch_elems, s));
    adv = n.adv_norm;
  }
  int k = 0;
  for (int ep = 0; ep < hp->epochs; ++ep) {
    DDPPO_TRY(launch_permutation(c.seed, n.d_steps, ep, E, n.perm, s));
    for (int mb = 0; mb < hp->minibatches; ++mb, ++k) {
      const int32_t* idx = n.perm + (size_t)mb * Emb;
      DDPPO_TRY(launch_gather_rows(ro->obs, n.obs_mb, idx, T, E, Emb, n.pix * op_bytes(n), s));
      DDPPO_TRY(launch_gather_rows(ro->goal, n.goal_mb, idx, T, E, Emb, 12, s));
      DDPPO_TRY(launch_gather_rows(ro->prev_a, n.preva_mb, idx, T, E, Emb, 4, s));
      DDPPO_TRY(launch_gather_rows(ro->masks, n.masks_mb, idx, T, E, Emb, 1, s));
      DDPPO_TRY(launch_gather_rows(ro->actions, n.act_mb, idx, T, E, Emb, 4, s));
      DDPPO_TRY(launch_gather_rows(ro->logp, n.logp_mb, idx, T, E, Emb, 4, s));
      DDPPO_TRY(launch_gather_rows(adv, n.adv_mb, idx, T, E, Emb, 4, s));
      DDPPO_TRY(launch_gather_rows(ro->ret, n.ret_mb, idx, T, E, Emb, 4, s));
      DDPPO_TRY(launch_gather_rows(ro->h0, n.h0_mb, idx, L, E, Emb, (size_t)Hd * 4, s));
      DDPPO_TRY(launch_gather_rows(ro->c0, n.c0_mb, idx, L, E, Emb, (size_t)Hd * 4, s));
      DDPPO_TRY(net_forward(n, T, Emb, n.obs_mb, n.goal_mb, n.preva_mb, n.masks_mb, n.h0_mb,
                            n.c0_mb, nullptr, nullptr, nullptr, s));
      float* st = stats ? stats + (size_t)k * DDPPO_NSTATS : n.stats_tmp + (size_t)(k % 64) * 8;
      DDPPO_TRY(launch_ppo_loss(Nmb, n.logits, n.values, n.act_mb, n.logp_mb, n.adv_mb, n.ret_mb,
                                hp->clip, hp->value_coef, hp->entropy_coef, st, n.dlogits,
                                n.dvalues, n.scratch, n.scratch_elems, s));
      DDPPO_TRY(net_backward(n, n.dlogits, n.dvalues, s));
      DDPPO_TRY(launch_grad_norm(n.grad, n.P, n.norm, n.scratch, n.scratch_elems, s));
      DDPPO_TRY(launch_copy_scalar(st + 6, n.norm, s));
      DDPPO_TRY(launch_adam(n.params, n.grad, n.adam_m, n.adam_v, n.P,
                            hp->max_grad_norm > 0.f ? n.norm : nullptr, hp->max_grad_norm, hp->lr,
                            hp->beta1, hp->beta2, hp->adam_eps, n.d_steps + 1, k + 1, s));
      DDPPO_TRY(net_prep_weights(n, s));
    }
  }
  return DDPPO_OK;
}

// ---- the update one minibatch at a time (gradients exchanged between workers, Eq. 4) ----
__global__ void scale_copy_kernel(const float* __restrict__ g, float scale, float* __restrict__ out,
                                  size_t n) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = scale * g[i];
}

extern "C" int ddppo_ppo_grad(ddppo_ctx* x, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                              int32_t T_valid, int32_t epoch, int32_t k, float* grad, float* stats,
                              void* stream) {
  ARG(x && x->net && ro && hp && grad, "ppo_grad: null argument");
  ARG(ro->obs && ro->goal && ro->prev_a && ro->masks && ro->actions && ro->logp && ro->adv &&
          ro->ret && ro->h0 && ro->c0,
      "ppo_grad: rollout view has a null buffer");
  Net& n = *x->net;
  const ddppo_config& c = x->cfg;
  if (hp->minibatches != c.minibatches || epoch < 0 || epoch >= hp->epochs || k < 0 ||
      k >= hp->minibatches || T_valid < 1 || T_valid > c.rollout_T) {
    set_error("ppo_grad: minibatches must equal the config's, 0 <= epoch < epochs, "
              "0 <= k < minibatches, 1 <= T_valid <= rollout_T");
    return DDPPO_E_CONFIG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int E = c.num_envs, Emb = n.Emb, L = n.L, Hd = n.H, T = T_valid;
  ::ddppo::launch_k(set_steps_kernel, 1, 1, 0, s, n.d_steps, hp->update_index, n.adam_t);
  DDPPO_CHECK_LAUNCH();
  const float* adv = ro->adv;
  if (hp->norm_adv) {
    DDPPO_TRY(launch_normalize_adv(ro->adv, n.adv_norm, (size_t)T * E, n.scal, n.scratch,
                                   n.scratch_elems, s));
    adv = n.adv_norm;
  }
  DDPPO_TRY(launch_permutation(c.seed, n.d_steps, epoch, E, n.perm, s));
  const int32_t* idx = n.perm + (size_t)k * Emb;
  DDPPO_TRY(launch_gather_rows(ro->obs, n.obs_mb, idx, T, E, Emb, n.pix * op_bytes(n), s));
  DDPPO_TRY(launch_gather_rows(ro->goal, n.goal_mb, idx, T, E, Emb, 12, s));
  DDPPO_TRY(launch_gather_rows(ro->prev_a, n.preva_mb, idx, T, E, Emb, 4, s));
  DDPPO_TRY(launch_gather_rows(ro->masks, n.masks_mb, idx, T, E, Emb, 1, s));
  DDPPO_TRY(launch_gather_rows(ro->actions, n.act_mb, idx, T, E, Emb, 4, s));
  DDPPO_TRY(launch_gather_rows(ro->logp, n.logp_mb, idx, T, E, Emb, 4, s));
  DDPPO_TRY(launch_gather_rows(adv, n.adv_mb, idx, T, E, Emb, 4, s));
  DDPPO_TRY(launch_gather_rows(ro->ret, n.ret_mb, idx, T, E, Emb, 4, s));
  DDPPO_TRY(launch_gather_rows(ro->h0, n.h0_mb, idx, L, E, Emb, (size_t)Hd * 4, s));
  DDPPO_TRY(launch_gather_rows(ro->c0, n.c0_mb, idx, L, E, Emb, (size_t)Hd * 4, s));
  DDPPO_TRY(net_forward(n, T, Emb, n.obs_mb, n.goal_mb, n.preva_mb, n.masks_mb, n.h0_mb, n.c0_mb,
                        nullptr, nullptr, nullptr, s));
  float* st = stats ? stats : n.stats_tmp;
  DDPPO_TRY(launch_ppo_loss(T * Emb, n.logits, n.values, n.act_mb, n.logp_mb, n.adv_mb, n.ret_mb,
                            hp->clip, hp->value_coef, hp->entropy_coef, st, n.dlogits, n.dvalues,
                            n.scratch, n.scratch_elems, s));
  DDPPO_TRY(net_backward(n, n.dlogits, n.dvalues, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(grad, n.grad, (size_t)n.P * 4, cudaMemcpyDeviceToDevice, s));
  n.ev_valid = false;
  return DDPPO_OK;
}

extern "C" int ddppo_apply_grad(ddppo_ctx* x, const float* grad, float scale,
                                const ddppo_ppo_hparams* hp, float* stats, void* stream) {
  ARG(x && x->net && grad && hp, "apply_grad: null argument");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t P = (size_t)n.P;
  ::ddppo::launch_k(scale_copy_kernel, (unsigned)std::min<size_t>((P + 255) / 256, 4096), 256, 0, s, grad, scale,
                                                                                     n.grad, P);
  DDPPO_CHECK_LAUNCH();
  DDPPO_TRY(launch_grad_norm(n.grad, P, n.norm, n.scratch, n.scratch_elems, s));
  if (stats) DDPPO_TRY(launch_copy_scalar(stats + 6, n.norm, s));
  ::ddppo::launch_k(set_steps_kernel, 1, 1, 0, s, n.d_steps, hp->update_index, n.adam_t);
  DDPPO_CHECK_LAUNCH();
  DDPPO_TRY(launch_adam(n.params, n.grad, n.adam_m, n.adam_v, P,
                        hp->max_grad_norm > 0.f ? n.norm : nullptr, hp->max_grad_norm, hp->lr,
                        hp->beta1, hp->beta2, hp->adam_eps, n.d_steps + 1, 1, s));
  DDPPO_TRY(net_prep_weights(n, s));
  n.adam_t += 1;
  return DDPPO_OK;
}

constexpr int kMeanMax = 64;
struct MeanArgs {
  const float* p[kMeanMax];
};
__global__ void grad_mean_kernel(MeanArgs a, int nb, size_t len, float* __restrict__ out) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len;
       i += (size_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int r = 0; r < nb; ++r) acc += a.p[r][i];  // fixed order: worker 0 first
    out[i] = acc / (float)nb;
  }
}

extern "C" int ddppo_grad_mean(int32_t n, const float* const* bufs, int64_t len, float* out,
                               void* stream) {
  ARG(n >= 1 && n <= kMeanMax && len >= 0 && bufs && out, "grad_mean: bad arguments");
  if (len == 0) return DDPPO_OK;
  MeanArgs a{};
  for (int r = 0; r < n; ++r) {
    ARG(bufs[r] != nullptr, "grad_mean: null buffer");
    a.p[r] = bufs[r];
  }
  ::ddppo::launch_k(grad_mean_kernel, (unsigned)std::min<int64_t>((len + 255) / 256, 4096), 256, 0, (cudaStream_t)stream, a, n, (size_t)len, out);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

static bool same_hparams(const ddppo_ppo_hparams& a, const ddppo_ppo_hparams& b) {
  ddppo_ppo_hparams x = a, y = b;
  x.update_index = 0;
  y.update_index = 0;
  return memcmp(&x, &y, sizeof(x)) == 0;
}

extern "C" int ddppo_ppo_update(ddppo_ctx* x, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                                float* stats, void* stream) {
  ARG(x && x->net && ro && hp, "ppo_update: null argument");
  ARG(ro->obs && ro->goal && ro->prev_a && ro->masks && ro->actions && ro->logp && ro->adv &&
          ro->ret && ro->h0 && ro->c0,
      "ppo_update: rollout view has a null buffer");
  Net& n = *x->net;
  const ddppo_config& c = x->cfg;
  if (hp->minibatches != c.minibatches || hp->epochs < 1) {
    set_error("ppo_update: minibatches must equal the config's, epochs >= 1");
    return DDPPO_E_CONFIG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // this update's index and the Adam steps taken so far, as device scalars (kernel
  // arguments: valid inside a caller's capture too)
  ::ddppo::launch_k(set_steps_kernel, 1, 1, 0, s, n.d_steps, hp->update_index, n.adam_t);
  DDPPO_CHECK_LAUNCH();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  DDPPO_CHECK_CUDA(cudaStreamIsCapturing(s, &cs));
  // the update is ~10K launches, most of them small: replaying it as one graph removes
  // the host launch cost. The kernel census and a caller's own capture run it directly;
  // so does the first update (the autotuner times its contraction shapes outside any
  // capture).
  const bool use_graph = n.upd_tuned && n.upd_graph_on && !n.upd_no_graph &&
                         cs == cudaStreamCaptureStatusNone;
  if (use_graph) {
    // with GEMM timing on, the graph carries the timer's event records (as event nodes);
    // it is valid while the timer's next record index is the one it was captured at
    const bool timed = n.timer.on;
    const bool same = n.upd_exec && memcmp(&n.upd_ro, ro, sizeof(*ro)) == 0 &&
                      same_hparams(n.upd_hp, *hp) && n.upd_stats == stats && n.upd_timed == timed &&
                      (!timed || n.upd_t_n0 == n.timer.n);
    if (!same) {
      if (n.upd_exec) { cudaGraphExecDestroy(n.upd_exec); n.upd_exec = nullptr; }
      DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
      const KernelTimer t0 = n.timer;
      const GemmTcCount c0 = n.tc_count;
      DDPPO_CHECK_CUDA(cudaStreamBeginCapture(n.cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = update_body(x, ro, hp, stats, n.cap_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(n.cap_stream, &g);
      if (rc != DDPPO_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (ce != cudaSuccess) { set_error(std::string("update capture: ") + cudaGetErrorString(ce)); return DDPPO_E_CUDA; }
      const cudaError_t ie = cudaGraphInstantiate(&n.upd_exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) { n.upd_exec = nullptr; set_error(std::string("update instantiate: ") + cudaGetErrorString(ie)); return DDPPO_E_CUDA; }
      n.upd_ro = *ro;
      n.upd_hp = *hp;
      n.upd_stats = stats;
      n.upd_timed = timed;
      // what the capture added to the host-side counters; replays add it again
      n.upd_t_n0 = t0.n;
      n.upd_t_dn = n.timer.n - t0.n;
      n.upd_t_flops = n.timer.flops - t0.flops;
      n.upd_t_flops_all = n.timer.flops_all - t0.flops_all;
      n.upd_t_launches = n.timer.launches - t0.launches;
      n.upd_tc_flops = n.tc_count.flops - c0.flops;
      n.upd_tc_launches = n.tc_count.launches - c0.launches;
      n.timer.n = t0.n; n.timer.flops = t0.flops; n.timer.flops_all = t0.flops_all;
      n.timer.launches = t0.launches;
      n.tc_count.flops = c0.flops; n.tc_count.launches = c0.launches;
    }
    DDPPO_CHECK_CUDA(cudaGraphLaunch(n.upd_exec, s));
    if (timed) {
      n.timer.n += n.upd_t_dn;
      n.timer.flops += n.upd_t_flops;
      n.timer.flops_all += n.upd_t_flops_all;
      n.timer.launches += n.upd_t_launches;
      if (n.tc_count.on) {
        n.tc_count.flops += n.upd_tc_flops;
        n.tc_count.launches += n.upd_tc_launches;
      }
    }
  } else {
    DDPPO_TRY(update_body(x, ro, hp, stats, s));
    if (cs == cudaStreamCaptureStatusNone) n.upd_tuned = true;
  }
  n.adam_t += (int64_t)hp->epochs * hp->minibatches;
  n.ev_valid = false;
  return DDPPO_OK;
}

// ---- collection ----
__global__ void post_step_kernel(int E, const int32_t* __restrict__ a, const uint8_t* __restrict__ d,
                                 int32_t* __restrict__ prev_a, uint8_t* __restrict__ masks) {
  DDPPO_PDL_ENTRY();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  prev_a[e] = d[e] ? 4 : a[e];
  masks[e] = d[e] ? 0 : 1;
}
__global__ void start_slot_kernel(int E, int32_t* prev_a, uint8_t* masks) {
  DDPPO_PDL_ENTRY();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  prev_a[e] = 4;
  masks[e] = 0;
}

extern "C" int ddppo_env_step(ddppo_ctx*, const int32_t*, void*, float*, float*, uint8_t*, float*,
                              void*);
extern "C" int ddppo_env_reset(ddppo_ctx*, void*, float*, void*);

static int collect_body(ddppo_ctx* x, const ddppo_rollout* ro, cudaStream_t s) {
  Net& n = *x->net;
  const int E = x->cfg.num_envs, T = x->cfg.rollout_T;
  const size_t ob = n.pix * op_bytes(n);
  // the next episodes of the envs are generated on a side stream while the policy acts:
  //   act(t) | prefetch(t-1)  ->  env_step(t)  ->  act(t+1) | prefetch(t) ...
  auto fork_prefetch = [&]() -> int {
    DDPPO_CHECK_CUDA(cudaEventRecord(x->ev_fork, s));
    DDPPO_CHECK_CUDA(cudaStreamWaitEvent(x->side, x->ev_fork, 0));
    DDPPO_TRY(launch_env_prefetch(x->sp, x->sb, x->prefetch_grid, x->side));
    DDPPO_CHECK_CUDA(cudaEventRecord(x->ev_join, x->side));
    return DDPPO_OK;
  };
  DDPPO_TRY(fork_prefetch());
  for (int t = 0; t < T; ++t) {
    const size_t o = (size_t)t * E;
    DDPPO_TRY(act_impl(x, (const char*)ro->obs + o * ob, ro->goal + o * 3, ro->prev_a + o,
                       ro->masks + o, ro->h, ro->c, ro->uniforms + o, ro->actions + o, ro->logp + o,
                       ro->values + o, s));
    DDPPO_CHECK_CUDA(cudaStreamWaitEvent(s, x->ev_join, 0));
    const size_t o1 = (size_t)(t + 1) * E;
    DDPPO_TRY(ddppo_env_step(x, ro->actions + o, (char*)ro->obs + o1 * ob, ro->goal + o1 * 3,
                             ro->rewards + o, ro->dones + o, ro->info ? ro->info + o * 4 : nullptr, s));
    ::ddppo::launch_k(post_step_kernel, (E + 127) / 128, 128, 0, s, E, ro->actions + o, ro->dones + o,
                                                     ro->prev_a + o1, ro->masks + o1);
    DDPPO_CHECK_LAUNCH();
    if (t + 1 < T) DDPPO_TRY(fork_prefetch());
  }
  return DDPPO_OK;
}

// prologue of a collection: slot 0 is the previous rollout's last slot (slot T, or the
// preempted length of a step-wise collection; first call: reset everything), h0/c0 <- h/c
static int collect_prologue(ddppo_ctx* x, const ddppo_rollout* ro, cudaStream_t s) {
  Net& n = *x->net;
  const int E = x->cfg.num_envs, L = n.L, Hd = n.H;
  const size_t ob = n.pix * op_bytes(n);
  const size_t st_bytes = (size_t)L * E * Hd * 4;
  if (!n.collect_started || !x->env_ready) {
    DDPPO_TRY(ddppo_env_reset(x, ro->obs, ro->goal, s));
    ::ddppo::launch_k(start_slot_kernel, (E + 127) / 128, 128, 0, s, E, ro->prev_a, ro->masks);
    DDPPO_CHECK_LAUNCH();
    DDPPO_CHECK_CUDA(cudaMemsetAsync(ro->h, 0, st_bytes, s));
    DDPPO_CHECK_CUDA(cudaMemsetAsync(ro->c, 0, st_bytes, s));
    n.collect_started = true;
  } else {
    const size_t oT = (size_t)n.T_last * E;
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->obs, (const char*)ro->obs + oT * ob, (size_t)E * ob,
                                     cudaMemcpyDeviceToDevice, s));
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->goal, ro->goal + oT * 3, (size_t)E * 12,
                                     cudaMemcpyDeviceToDevice, s));
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->prev_a, ro->prev_a + oT, (size_t)E * 4,
                                     cudaMemcpyDeviceToDevice, s));
    DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->masks, ro->masks + oT, (size_t)E,
                                     cudaMemcpyDeviceToDevice, s));
  }
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->h0, ro->h, st_bytes, cudaMemcpyDeviceToDevice, s));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->c0, ro->c, st_bytes, cudaMemcpyDeviceToDevice, s));
  return DDPPO_OK;
}

// bootstrap value V(o_Tv) with the state after step Tv - 1; the state itself is not advanced
static int collect_bootstrap(ddppo_ctx* x, const ddppo_rollout* ro, int Tv, cudaStream_t s) {
  Net& n = *x->net;
  const int E = x->cfg.num_envs;
  const size_t ob = n.pix * op_bytes(n);
  const size_t oT = (size_t)Tv * E;
  DDPPO_TRY(net_forward(n, 1, E, (const char*)ro->obs + oT * ob, ro->goal + oT * 3,
                        ro->prev_a + oT, ro->masks + oT, ro->h, ro->c, nullptr, nullptr, nullptr, s,
                        true));
  DDPPO_CHECK_CUDA(cudaMemcpyAsync(ro->values + oT, n.values, (size_t)E * 4,
                                   cudaMemcpyDeviceToDevice, s));
  n.ev_valid = false;
  n.T_last = Tv;
  return DDPPO_OK;
}

static bool collect_view_ok(const ddppo_rollout* ro) {
  return ro->obs && ro->goal && ro->prev_a && ro->masks && ro->actions && ro->logp && ro->values &&
         ro->rewards && ro->dones && ro->h0 && ro->c0 && ro->h && ro->c && ro->uniforms;
}

extern "C" int ddppo_collect_begin(ddppo_ctx* x, const ddppo_rollout* ro, void* stream) {
  ARG(x && x->net && ro && collect_view_ok(ro), "collect_begin: null argument or buffer");
  DDPPO_TRY(collect_prologue(x, ro, (cudaStream_t)stream));
  x->net->step_next = 0;
  return DDPPO_OK;
}

extern "C" int ddppo_collect_step(ddppo_ctx* x, const ddppo_rollout* ro, int32_t t, void* stream) {
  ARG(x && x->net && ro && collect_view_ok(ro), "collect_step: null argument or buffer");
  Net& n = *x->net;
  const int E = x->cfg.num_envs;
  if (t != n.step_next || t < 0 || t >= x->cfg.rollout_T) {
    set_error("collect_step: steps must follow collect_begin in order, t < rollout_T");
    return DDPPO_E_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ob = n.pix * op_bytes(n);
  // the next episodes are prepared on the side stream while the policy acts, and joined
  // before the env step: the same overlap as a whole collection
  DDPPO_CHECK_CUDA(cudaEventRecord(x->ev_fork, s));
  DDPPO_CHECK_CUDA(cudaStreamWaitEvent(x->side, x->ev_fork, 0));
  DDPPO_TRY(launch_env_prefetch(x->sp, x->sb, x->prefetch_grid, x->side));
  DDPPO_CHECK_CUDA(cudaEventRecord(x->ev_join, x->side));
  const size_t o = (size_t)t * E, o1 = (size_t)(t + 1) * E;
  DDPPO_TRY(act_impl(x, (const char*)ro->obs + o * ob, ro->goal + o * 3, ro->prev_a + o,
                     ro->masks + o, ro->h, ro->c, ro->uniforms + o, ro->actions + o, ro->logp + o,
                     ro->values + o, s));
  DDPPO_CHECK_CUDA(cudaStreamWaitEvent(s, x->ev_join, 0));
  DDPPO_TRY(ddppo_env_step(x, ro->actions + o, (char*)ro->obs + o1 * ob, ro->goal + o1 * 3,
                           ro->rewards + o, ro->dones + o, ro->info ? ro->info + o * 4 : nullptr, s));
  ::ddppo::launch_k(post_step_kernel, (E + 127) / 128, 128, 0, s, E, ro->actions + o, ro->dones + o,
                                                   ro->prev_a + o1, ro->masks + o1);
  DDPPO_CHECK_LAUNCH();
  n.step_next = t + 1;
  return DDPPO_OK;
}

extern "C" int ddppo_collect_end(ddppo_ctx* x, const ddppo_rollout* ro, int32_t T_valid,
                                 void* stream) {
  ARG(x && x->net && ro && collect_view_ok(ro), "collect_end: null argument or buffer");
  Net& n = *x->net;
  if (T_valid < 1 || T_valid != n.step_next) {
    set_error("collect_end: T_valid must equal the number of steps taken (>= 1)");
    return DDPPO_E_STATE;
  }
  n.step_next = -1;
  return collect_bootstrap(x, ro, T_valid, (cudaStream_t)stream);
}

extern "C" int ddppo_collect(ddppo_ctx* x, const ddppo_rollout* ro, int32_t use_graph,
                             void* stream) {
  ARG(x && x->net && ro, "collect: null argument");
  ARG(ro->obs && ro->goal && ro->prev_a && ro->masks && ro->actions && ro->logp && ro->values &&
          ro->rewards && ro->dones && ro->h0 && ro->c0 && ro->h && ro->c && ro->uniforms,
      "collect: rollout view has a null buffer");
  Net& n = *x->net;
  cudaStream_t s = (cudaStream_t)stream;
  const int E = x->cfg.num_envs, T = x->cfg.rollout_T;
  const size_t ob = n.pix * op_bytes(n);
  DDPPO_TRY(collect_prologue(x, ro, s));
  if (use_graph) {
    if (!n.graph_exec || memcmp(&n.graph_ro, ro, sizeof(*ro)) != 0) {
      // one act step outside the capture (state into scratch buffers) so that the GEMM
      // autotuner sees the act shapes before they are frozen into the graph
      if (n.gws.tuner) {
        // the pass leaves no trace: FP8 inference's delayed activation scales are put back
        // (a resumed run, whose first collect captures again, then matches an unbroken one)
        const size_t fa = (size_t)n.f8_act_slots * 4;
        if (n.f8) {
          DDPPO_CHECK_CUDA(cudaMemcpyAsync(n.f8_keep, n.f8_scale, fa, cudaMemcpyDeviceToDevice, s));
          DDPPO_CHECK_CUDA(cudaMemcpyAsync(n.f8_keep + n.f8_act_slots, n.f8_amax, fa,
                                           cudaMemcpyDeviceToDevice, s));
        }
        DDPPO_TRY(net_forward(n, 1, E, ro->obs, ro->goal, ro->prev_a, ro->masks, ro->h, ro->c,
                              ro->uniforms, (int32_t*)n.perm, n.dvalues, s, true));
        n.ev_valid = false;
        if (n.f8) {
          DDPPO_CHECK_CUDA(cudaMemcpyAsync(n.f8_scale, n.f8_keep, fa, cudaMemcpyDeviceToDevice, s));
          DDPPO_CHECK_CUDA(cudaMemcpyAsync(n.f8_amax, n.f8_keep + n.f8_act_slots, fa,
                                           cudaMemcpyDeviceToDevice, s));
        }
      }
      if (n.graph_exec) { cudaGraphExecDestroy(n.graph_exec); n.graph_exec = nullptr; }
      DDPPO_CHECK_CUDA(cudaStreamSynchronize(s));
      const bool t0 = n.timer.on, t1 = n.rc_timer.on;
      n.timer.on = false; n.rc_timer.on = false;
      DDPPO_CHECK_CUDA(cudaStreamBeginCapture(n.cap_stream, cudaStreamCaptureModeThreadLocal));
      const int rc = collect_body(x, ro, n.cap_stream);
      cudaGraph_t g = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(n.cap_stream, &g);
      n.timer.on = t0; n.rc_timer.on = t1;
      if (rc != DDPPO_OK) { if (g) cudaGraphDestroy(g); return rc; }
      if (ce != cudaSuccess) { set_error(std::string("collect capture: ") + cudaGetErrorString(ce)); return DDPPO_E_CUDA; }
      const cudaError_t ie = cudaGraphInstantiate(&n.graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) { set_error(std::string("collect instantiate: ") + cudaGetErrorString(ie)); return DDPPO_E_CUDA; }
      n.graph_ro = *ro;
    }
    DDPPO_CHECK_CUDA(cudaGraphLaunch(n.graph_exec, s));
  } else {
    DDPPO_TRY(collect_body(x, ro, s));
  }
  return collect_bootstrap(x, ro, T, s);
}

// ---- timing ----
extern "C" int ddppo_timing_enable(ddppo_ctx* x, int32_t on) {
  ARG(x && x->net, "timing_enable: null ctx");
  Net& n = *x->net;
  n.tc_count.on = on != 0;
  n.tc_count.launches = 0;
  n.tc_count.flops = 0.0;
  for (KernelTimer* t : {&n.timer, &n.rc_timer}) {
    t->on = on != 0;
    t->n = 0;
    t->flops = 0.0;
    t->flops_all = 0.0;
    t->launches = 0;
  }
  return DDPPO_OK;
}

extern "C" int ddppo_timing_read(ddppo_ctx* x, int32_t family, double* ms, int64_t* launches,
                                 double* work) {
  ARG(x && x->net && ms && launches && work, "timing_read: null argument");
  ARG(family >= 0 && family <= 2, "timing_read: family must be 0, 1 or 2");
  if (family == 2) {
    // tcgen05 launches; ms carries the FLOPs of every GEMM launch (tensor core or not)
    *ms = x->net->timer.flops_all;
    *launches = x->net->tc_count.launches;
    *work = x->net->tc_count.flops;
    return DDPPO_OK;
  }
  KernelTimer& t = family == 0 ? x->net->timer : x->net->rc_timer;
  double acc = 0.0;
  for (int i = 0; i + 1 < t.n; i += 2) {
    DDPPO_CHECK_CUDA(cudaEventSynchronize(t.ev[i + 1]));
    float v = 0.f;
    DDPPO_CHECK_CUDA(cudaEventElapsedTime(&v, t.ev[i], t.ev[i + 1]));
    acc += v;
  }
  *ms = acc;
  *launches = t.launches;
  *work = t.flops;
  return DDPPO_OK;
}

// ---- kernel census of one steady-state iteration ----
static int count_kernel_nodes(cudaGraph_t g, int64_t* count) {
  size_t num = 0;
  DDPPO_CHECK_CUDA(cudaGraphGetNodes(g, nullptr, &num));
  std::vector<cudaGraphNode_t> nodes(num);
  DDPPO_CHECK_CUDA(cudaGraphGetNodes(g, nodes.data(), &num));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    DDPPO_CHECK_CUDA(cudaGraphNodeGetType(nd, &ty));
    if (ty == cudaGraphNodeTypeKernel) {
      ++*count;
    } else if (ty == cudaGraphNodeTypeGraph) {
      cudaGraph_t child;
      DDPPO_CHECK_CUDA(cudaGraphChildGraphNodeGetGraph(nd, &child));
      DDPPO_TRY(count_kernel_nodes(child, count));
    }
  }
  return DDPPO_OK;
}

extern "C" int ddppo_count_kernels(ddppo_ctx* x, const ddppo_rollout* ro,
                                   const ddppo_ppo_hparams* hp, float gamma, float lam,
                                   int64_t* count) {
  ARG(x && x->net && ro && hp && count, "count_kernels: null argument");
  Net& n = *x->net;
  if (!x->env_ready) { set_error("count_kernels before the first collect"); return DDPPO_E_STATE; }
  const int E = x->cfg.num_envs, T = x->cfg.rollout_T;
  const int64_t adam_t = n.adam_t;
  n.upd_no_graph = true;
  const bool t0 = n.timer.on, t1 = n.rc_timer.on, t2 = n.tc_count.on;
  n.timer.on = n.rc_timer.on = n.tc_count.on = false;
  DDPPO_CHECK_CUDA(cudaDeviceSynchronize());
  DDPPO_CHECK_CUDA(cudaStreamBeginCapture(n.cap_stream, cudaStreamCaptureModeThreadLocal));
  int rc = collect_body(x, ro, n.cap_stream);
  const size_t ob = n.pix * op_bytes(n);
  const size_t oT = (size_t)T * E;
  if (rc == DDPPO_OK)
    rc = net_forward(n, 1, E, (const char*)ro->obs + oT * ob, ro->goal + oT * 3, ro->prev_a + oT,
                     ro->masks + oT, ro->h, ro->c, nullptr, nullptr, nullptr, n.cap_stream, true);
  if (rc == DDPPO_OK)
    rc = launch_gae(ro->rewards, ro->dones, ro->values, T, E, gamma, lam, ro->adv, ro->ret,
                    n.cap_stream);
  if (rc == DDPPO_OK) rc = ddppo_ppo_update(x, ro, hp, nullptr, n.cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(n.cap_stream, &g);
  n.adam_t = adam_t;
  n.upd_no_graph = false;
  n.timer.on = t0; n.rc_timer.on = t1; n.tc_count.on = t2;
  n.ev_valid = false;
  if (rc != DDPPO_OK) { if (g) cudaGraphDestroy(g); return rc; }
  if (ce != cudaSuccess) { set_error(std::string("count capture: ") + cudaGetErrorString(ce)); return DDPPO_E_CUDA; }
  *count = 0;
  rc = count_kernel_nodes(g, count);
  cudaGraphDestroy(g);
  return rc;
}

// ---- stand-alone GEMM (the contraction every network layer uses) ----
extern "C" int ddppo_gemm(int32_t M, int32_t N, int32_t K, int32_t op_bf16, const void* A,
                          int32_t lda, int32_t a_t, const void* B, int32_t ldb, int32_t b_t,
                          void* C, int32_t ldc, int32_t c_bf16, float beta, const float* bias,
                          int32_t relu, int32_t* status, void* stream) {
  ARG(M >= 0 && N >= 0 && K >= 1, "gemm: bad sizes");
  if (M == 0 || N == 0) return DDPPO_OK;
  ARG(A && B && C, "gemm: null argument");
  ARG(lda >= (a_t ? M : K) && ldb >= (b_t ? N : K) && ldc >= N,
      "gemm: leading dimension smaller than the row");
  static float* partial[64] = {};
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  ARG(dev < 64, "gemm: device ordinal out of range");
  const size_t elems = (size_t)16 << 20;
  if (!partial[dev]) DDPPO_CHECK_CUDA(cudaMalloc(&partial[dev], elems * sizeof(float)));
  GemmWorkspace ws;
  ws.partial = partial[dev];
  ws.partial_elems = elems;
  cudaDeviceGetAttribute(&ws.num_sms, cudaDevAttrMultiProcessorCount, dev);
  ws.err = status;
  GemmDesc d;
  d.M = M; d.N = N; d.K = K; d.A = A; d.lda = lda; d.B = B; d.ldb = ldb; d.C = C; d.ldc = ldc;
  d.c_bf16 = c_bf16; d.beta = beta; d.bias = bias; d.relu = relu;
  d.a_t = a_t ? 1 : 0; d.b_t = b_t ? 1 : 0;
  return gemm(d, op_bf16 != 0, ws, (cudaStream_t)stream, nullptr);
}

extern "C" int ddppo_gemm_backend(int32_t M, int32_t N, int32_t K, int32_t op_bf16,
                                  const void* A, int32_t lda, const void* B, int32_t ldb,
                                  int32_t* tensor_cores) {
  ARG(tensor_cores, "gemm_backend: null argument");
  GemmDesc d;
  d.M = M; d.N = N; d.K = K; d.A = A; d.lda = lda; d.B = B; d.ldb = ldb;
  *tensor_cores = (op_bf16 && gemm_tc_supported(d)) ? 1 : 0;
  return DDPPO_OK;
}

extern "C" int ddppo_timing_launches(ddppo_ctx* x, int32_t family, double* ms, double* work,
                                     double* bytes, int64_t cap, int64_t* count) {
  ARG(x && x->net && count, "timing_launches: null argument");
  ARG(family == 0 || family == 1, "timing_launches: family must be 0 or 1");
  KernelTimer& t = family == 0 ? x->net->timer : x->net->rc_timer;
  const int64_t n = t.n / 2;
  *count = n;
  for (int64_t i = 0; i < n && i < cap; ++i) {
    float v = 0.f;
    DDPPO_CHECK_CUDA(cudaEventSynchronize(t.ev[2 * i + 1]));
    DDPPO_CHECK_CUDA(cudaEventElapsedTime(&v, t.ev[2 * i], t.ev[2 * i + 1]));
    if (ms) ms[i] = v;
    if (work) work[i] = t.work[i];
    if (bytes) bytes[i] = t.bytes[i];
  }
  return DDPPO_OK;
}

extern "C" int ddppo_update_graph(ddppo_ctx* x, int32_t on) {
  ARG(x && x->net, "update_graph: null ctx");
  x->net->upd_graph_on = on != 0;
  return DDPPO_OK;
}

extern "C" int ddppo_lstm_whole_segment(ddppo_ctx* x, int32_t mode) {
  ARG(x && x->net, "lstm_whole_segment: null ctx");
  ARG(mode >= 0 && mode <= 2, "lstm_whole_segment: mode must be 0, 1 or 2");
  x->net->lstm_mode = mode;
  return DDPPO_OK;
}

extern "C" int ddppo_autotune(ddppo_ctx* x, int32_t on, int64_t* tuned_shapes) {
  ARG(x && x->net, "autotune: null ctx");
  tc_tuner_enable(x->net->gws.tuner, on != 0);
  if (tuned_shapes) *tuned_shapes = tc_tuner_shapes(x->net->gws.tuner);
  return DDPPO_OK;
}

extern "C" int ddppo_autotune_export(ddppo_ctx* x, void* buf, size_t cap, size_t* size) {
  ARG(x && x->net && size, "autotune_export: null argument");
  *size = tc_tuner_export(x->net->gws.tuner, buf, cap);
  ARG(!buf || cap >= *size, "autotune_export: buffer too small");
  return DDPPO_OK;
}

extern "C" int ddppo_autotune_import(ddppo_ctx* x, const void* buf, size_t size) {
  ARG(x && x->net && buf, "autotune_import: null argument");
  return tc_tuner_import(x->net->gws.tuner, buf, size);
}

// ---- stand-alone GroupNorm (C/2 groups, the encoder's normalisation) ----
extern "C" int ddppo_group_norm(int32_t N, int32_t HW, int32_t C, const float* z, const float* gamma,
                                const float* beta, const float* resid, int32_t relu, float* out,
                                float* mean, float* rstd, void* stream) {
  ARG(N >= 1 && N <= 8192 && HW >= 1 && C >= 2 && C <= 1024 && C % 2 == 0,
      "group_norm: N in [1, 8192], C even in [2, 1024]");
  ARG(z && gamma && beta && out && mean && rstd, "group_norm: null argument");
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  ARG(dev < 64, "group_norm: device ordinal out of range");
  static GnScratch ws[64];
  if (!ws[dev].part) {
    GnScratch w;
    w.max_images = 8192;
    w.part_elems = gn_part_elems(w.max_images, 1024);
    DDPPO_CHECK_CUDA(cudaMalloc(&w.part, w.part_elems * sizeof(float)));
    DDPPO_CHECK_CUDA(cudaMalloc(&w.cnt, (size_t)w.max_images * sizeof(int)));
    DDPPO_CHECK_CUDA(cudaMemset(w.cnt, 0, (size_t)w.max_images * sizeof(int)));
    DDPPO_CHECK_CUDA(cudaMalloc(&w.cnt2, (size_t)w.max_images * sizeof(int)));
    DDPPO_CHECK_CUDA(cudaMemset(w.cnt2, 0, (size_t)w.max_images * sizeof(int)));
    ws[dev] = w;
  }
  cudaStream_t s = (cudaStream_t)stream;
  GNApply a{};
  a.z = z; a.mean = mean; a.rstd = rstd; a.gamma = gamma; a.beta = beta;
  a.resid = resid; a.out = out; a.relu = relu ? 1 : 0;
  bool done = false;
  DDPPO_TRY(launch_gn_fused(a, N, HW, C, 1e-5f, ws[dev], nullptr, s, &done));
  if (done) return DDPPO_OK;
  DDPPO_TRY(launch_gn_stats(z, N, HW, C, 1e-5f, mean, rstd, ws[dev], s));
  return launch_gn_apply(a, N, HW, C, s);
}

extern "C" int ddppo_group_norm_one_launch(ddppo_ctx* x, int32_t on) {
  ARG(x && x->net, "group_norm_one_launch: null ctx");
  x->net->gn_fused_on = on != 0;
  return DDPPO_OK;
}

// ---- stand-alone SE-ResNeXt pieces: grouped 3x3 convolution and squeeze-excite ----
extern "C" int ddppo_grouped_conv3x3(int32_t N, int32_t H, int32_t W, int32_t C, int32_t groups,
                                     int32_t stride, const float* x, const float* w, float* z,
                                     void* stream) {
  ARG(N >= 1 && H >= 1 && W >= 1 && groups >= 1 && C % groups == 0 && C / groups <= 16 &&
          (stride == 1 || stride == 2) && C <= 1024,
      "grouped_conv3x3: bad sizes (C / groups <= 16, C <= 1024, stride 1 or 2)");
  ARG(x && w && z, "grouped_conv3x3: null argument");
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  ARG(dev < 64, "grouped_conv3x3: device ordinal out of range");
  static float* wbuf[64] = {};
  if (!wbuf[dev]) DDPPO_CHECK_CUDA(cudaMalloc(&wbuf[dev], (size_t)1024 * 16 * 9 * sizeof(float)));
  cudaStream_t s = (cudaStream_t)stream;
  GConv g;
  g.N = N; g.H = H; g.W = W; g.C = C; g.cpg = C / groups; g.s = stride;
  g.Ho = (H + 2 - 3) / stride + 1; g.Wo = (W + 2 - 3) / stride + 1;
  DDPPO_TRY(launch_gconv_w_prep(w, C, g.cpg, wbuf[dev], false, s));
  return launch_gconv_fwd(g, x, wbuf[dev], z, false, s);
}

extern "C" int ddppo_squeeze_excite(int32_t N, int32_t HW, int32_t C, int32_t Cr, const float* u,
                                    const float* sc, const float* W1, const float* b1,
                                    const float* W2, const float* b2, float* m, float* a,
                                    float* gate, float* y, void* stream) {
  ARG(N >= 1 && HW >= 1 && C >= 1 && Cr >= 1 && C <= 4096, "squeeze_excite: bad sizes");
  ARG(u && W1 && b1 && W2 && b2 && m && a && gate && y, "squeeze_excite: null argument");
  SeArgs e{};
  e.N = N; e.HW = HW; e.C = C; e.Cr = Cr;
  e.u = u; e.sc = sc; e.W1 = W1; e.b1 = b1; e.W2 = W2; e.b2 = b2;
  e.m = m; e.a = a; e.gate = gate; e.y = y;
  return launch_se_fwd(e, (cudaStream_t)stream);
}

// ---- stand-alone convolution on the implicit-im2col tensor-core path ----
static int standalone_ws(GemmWorkspace* ws, int32_t* status) {
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  static float* partial[64] = {};
  ARG(dev < 64, "conv2d: device ordinal out of range");
  const size_t elems = (size_t)16 << 20;
  if (!partial[dev]) DDPPO_CHECK_CUDA(cudaMalloc(&partial[dev], elems * sizeof(float)));
  ws->partial = partial[dev];
  ws->partial_elems = elems;
  cudaDeviceGetAttribute(&ws->num_sms, cudaDevAttrMultiProcessorCount, dev);
  ws->err = status;
  return DDPPO_OK;
}

static int conv_args(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                     int32_t stride, int32_t pad, ConvShape* c) {
  ARG(N >= 1 && H >= 1 && W >= 1 && C >= 1 && Cout >= 1 && k >= 1 && stride >= 1 && pad >= 0,
      "conv2d: bad sizes");
  c->N = N; c->H = H; c->W = W; c->C = C; c->k = k; c->s = stride; c->p = pad;
  c->Ho = (H + 2 * pad - k) / stride + 1;
  c->Wo = (W + 2 * pad - k) / stride + 1;
  ARG(c->Ho >= 1 && c->Wo >= 1, "conv2d: empty output");
  return DDPPO_OK;
}

extern "C" int ddppo_conv2d(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                            int32_t stride, int32_t pad, const void* x, const void* w, float* y,
                            float beta, int32_t* status, void* stream) {
  ConvShape c;
  DDPPO_TRY(conv_args(N, H, W, C, Cout, k, stride, pad, &c));
  ARG(x && w && y, "conv2d: null argument");
  c.Cout = Cout;
  // one input channel (the encoder's stem): the contraction gathers its patches itself
  const bool c1 = C == 1 && conv_c1_tc_supported(k, Cout);
  if (!c1 && !gemm_conv_supported(c, x)) {
    set_error("conv2d: shape not covered by the implicit-im2col path");
    return DDPPO_E_CONFIG;
  }
  GemmWorkspace ws;
  DDPPO_TRY(standalone_ws(&ws, status));
  GemmDesc d;
  d.M = N * c.Ho * c.Wo; d.N = Cout; d.K = k * k * C;
  d.conv = &c; d.A = x; d.lda = d.K; d.B = w; d.ldb = d.K;
  d.C = y; d.ldc = Cout; d.beta = beta;
  return gemm(d, true, ws, (cudaStream_t)stream, nullptr);
}

extern "C" int ddppo_conv_plan(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout,
                               int32_t k, int32_t stride, int32_t pad, int32_t* plan) {
  ConvShape c;
  DDPPO_TRY(conv_args(N, H, W, C, Cout, k, stride, pad, &c));
  ARG(plan, "conv_plan: null argument");
  c.Cout = Cout;
  conv_plan(c, plan);
  return DDPPO_OK;
}

// ---- E4M3 (FP8 inference) contractions and quantisation ----
extern "C" int ddppo_quantize_e4m3(const void* x, int32_t x_bf16, int64_t n, void* q, float* scale,
                                   void* stream) {
  ARG(n >= 0, "quantize_e4m3: negative size");
  ARG(x && q && scale, "quantize_e4m3: null argument");
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  ARG(dev < 64, "quantize_e4m3: device ordinal out of range");
  static unsigned* amax[64] = {};
  if (!amax[dev]) DDPPO_CHECK_CUDA(cudaMalloc(&amax[dev], sizeof(unsigned)));
  cudaStream_t s = (cudaStream_t)stream;
  DDPPO_CHECK_CUDA(cudaMemsetAsync(amax[dev], 0, sizeof(unsigned), s));
  DDPPO_TRY(launch_amax(x, x_bf16 != 0, (size_t)n, amax[dev], s));
  return launch_quant_e4m3(x, x_bf16 != 0, (size_t)n, amax[dev], scale, (uint8_t*)q, s);
}

extern "C" int ddppo_gemm_e4m3(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                               const void* B, int32_t ldb, const float* scale_a,
                               const float* scale_b, float* C, int32_t ldc, float beta,
                               const float* bias, int32_t relu, int32_t* status, void* stream) {
  ARG(M >= 0 && N >= 0 && K >= 1, "gemm_e4m3: bad sizes");
  if (M == 0 || N == 0) return DDPPO_OK;
  ARG(A && B && C, "gemm_e4m3: null argument");
  ARG(lda >= K && ldb >= K && ldc >= N, "gemm_e4m3: leading dimension smaller than the row");
  GemmWorkspace ws;
  DDPPO_TRY(standalone_ws(&ws, status));
  GemmDesc d;
  d.M = M; d.N = N; d.K = K; d.A = A; d.lda = lda; d.B = B; d.ldb = ldb; d.C = C; d.ldc = ldc;
  d.beta = beta; d.bias = bias; d.relu = relu;
  d.fp8 = 1; d.scale_a = scale_a; d.scale_b = scale_b;
  return gemm(d, true, ws, (cudaStream_t)stream, nullptr);
}

extern "C" int ddppo_conv2d_e4m3(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout,
                                 int32_t k, int32_t stride, int32_t pad, const void* x,
                                 const void* w, const float* scale_x, const float* scale_w,
                                 float* y, float beta, int32_t* status, void* stream) {
  ConvShape c;
  DDPPO_TRY(conv_args(N, H, W, C, Cout, k, stride, pad, &c));
  ARG(x && w && y, "conv2d_e4m3: null argument");
  c.Cout = Cout;
  GemmWorkspace ws;
  DDPPO_TRY(standalone_ws(&ws, status));
  GemmDesc d;
  d.M = N * c.Ho * c.Wo; d.N = Cout; d.K = k * k * C;
  d.conv = &c; d.A = x; d.lda = d.K; d.B = w; d.ldb = d.K;
  d.C = y; d.ldc = Cout; d.beta = beta;
  d.fp8 = 1; d.scale_a = scale_x; d.scale_b = scale_w;
  return gemm(d, true, ws, (cudaStream_t)stream, nullptr);
}

extern "C" int ddppo_conv2d_wgrad(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout,
                                  int32_t k, int32_t stride, int32_t pad, const void* x,
                                  const void* dy, float* dw, float beta, int32_t* status,
                                  void* stream) {
  ConvShape c;
  DDPPO_TRY(conv_args(N, H, W, C, Cout, k, stride, pad, &c));
  ARG(x && dy && dw, "conv2d_wgrad: null argument");
  c.Cout = Cout;
  if (Cout % 8 || !(conv_wgrad_halo_ok(c, x, dy) || gemm_convw_supported(c, x, dy))) {
    set_error("conv2d_wgrad: shape not covered by the implicit weight-gradient path");
    return DDPPO_E_CONFIG;
  }
  GemmWorkspace ws;
  DDPPO_TRY(standalone_ws(&ws, status));
  GemmDesc d;
  d.M = Cout; d.N = k * k * C; d.K = N * c.Ho * c.Wo;
  d.A = dy; d.lda = Cout; d.a_t = 1;
  d.convw = &c; d.B = x;
  d.C = dw; d.ldc = d.N; d.beta = beta;
  return gemm(d, true, ws, (cudaStream_t)stream, nullptr);
}
