/*
 * ddppo.h -- C ABI of the GB300 (sm_103a) DD-PPO rollout-then-update hot path.
 *
 * DD-PPO (arXiv:1911.00357) trains a PointGoal navigation agent with PPO in a
 * synchronous collect-then-update loop (Sec. 3, Eq. 4; Fig. "distrib_rl"): each
 * worker collects a rollout with its current policy, computes GAE advantages,
 * and runs epochs x minibatches of the clipped-surrogate update (Sec. 2 Eq. 2,
 * Sec. 4 "Training"). This library is one such worker on one GPU. The
 * simulator is an occupancy-grid world with a ray-cast depth camera standing
 * in for Habitat-Sim (Sec. 4 "Simulator+Datasets"), whose scenes and renderer
 * are not available.
 *
 * Conventions for every entry point
 *   - Return value: DDPPO_OK (0) or a negative DDPPO_E_* code. Nothing aborts,
 *     throws or exits. ddppo_last_error() gives the message of the last failure
 *     on the calling thread.
 *   - Pointers marked [dev] are CUDA device pointers owned by the caller; the
 *     library never frees them and never keeps them past the call (except the
 *     buffers of a captured collect graph, see ddppo_collect). Pointers marked
 *     [host] are host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream. Work is enqueued asynchronously on it; results are ready when the
 *     stream is synchronised. Entry points that enqueue work never allocate or
 *     synchronise, so they can be captured into a CUDA graph, except where noted.
 *   - Arrays are dense, row-major, time-major where a time axis exists.
 *   - Units of the world: positions in u = 1e-4 m (int32), depth in metres.
 *   - Errors detected on the device (an index outside a buffer, a capped wait
 *     that ran out) do not trap: they set a sticky device status word that
 *     ddppo_device_status() reads.
 */
#ifndef DDPPO_H
#define DDPPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DDPPO_OK 0
#define DDPPO_E_ARG (-1)           /* null pointer, bad size, misaligned pointer        */
#define DDPPO_E_CONFIG (-2)        /* unsupported configuration or shape                 */
#define DDPPO_E_CUDA (-3)          /* a CUDA call or kernel launch failed                */
#define DDPPO_E_DEVICE_BOUNDS (-4) /* a kernel caught an out-of-range index (sticky)     */
#define DDPPO_E_TIMEOUT (-5)       /* a capped device loop ran out of iterations (sticky)*/
#define DDPPO_E_STATE (-6)         /* call order: e.g. env_step before env_reset         */

#define DDPPO_NSTATE 12   /* int32 slots of one agent state, see ddppo_env_state */
#define DDPPO_NSTATS 8    /* floats of PPO statistics per minibatch              */
#define DDPPO_NUM_ACTIONS 4

typedef struct ddppo_ctx ddppo_ctx;

/* Everything that fixes shapes and workspace sizes. Readings of the paper for
 * the values it leaves open are listed per field. */
typedef struct {
  int32_t num_envs;       /* E: parallel environments of this worker (Sec. 4 "Training") */
  /* world: procedural occupancy grids standing in for Gibson/MP3D scenes */
  int32_t gen_kind;       /* 0: border + Bernoulli walls; 1: recursive rooms and doors     */
  int32_t grid_min;       /* square grid side in cells; each episode draws a side          */
  int32_t grid_max;       /*   grid_min * 2^j <= grid_max uniformly (equal: fixed side).   */
                          /*   Sides must be multiples of 32 and at most 512.              */
  float cell_m;           /* cell side in metres (0.25 or 0.1)                             */
  float wall_density;     /* Bernoulli wall probability (gen_kind 0)                       */
  float door_m;           /* door width in metres (gen_kind 1)                              */
  int32_t min_room;       /* minimum room side in cells (gen_kind 1)                        */
  int32_t max_steps;      /* episode step cap (500)                                         */
  int32_t terminal_mode;  /* 0: +2.5 on success; 1: +2.5*SPL (Sec. 4 "Training")           */
  /* depth camera (Sec. 4 "Agent": 256x256 depth; 90 degree field of view) */
  int32_t depth_h, depth_w; /* rendered resolution; square, even, <= 1024                   */
  int32_t pool2x2;        /* 1: 2x2 average pool before the encoder (App. "Visual Encoder") */
  float cam_h_m;          /* camera height (0.88 m)                                          */
  float ceil_h_m;         /* ceiling height (2.5 m)                                          */
  float max_depth_m;      /* depth clip and normaliser (10 m)                                */
  /* agent network (App. "Agent Design") */
  int32_t net_kind;       /* 0: 3-layer conv 32/64/32 (8/4/3); 1: ResNet-18-style + GN;
                             2: blind (GPS+Compass only, Sec. 5): no visual encoder or FC;
                             3 / 4: SE-ResNeXt50 / 101 with every layer's channels halved
                             and GroupNorm (App. "Visual Encoder"; Tab. 1): bottlenecks
                             [3,4,6,3] / [3,4,23,3] of inner width 2 base 2^i (grouped 3x3,
                             32 groups, carrying the stride) and output 4 base 2^i,
                             squeeze-excite with reduction 16; 1024 x 4 x 4 at base 32    */
  int32_t base_ch;        /* ResNet base width (32 or 64); SE-ResNeXt: 16 or 32            */
  int32_t hidden;         /* LSTM hidden size and visual FC width (128 or 512)               */
  int32_t lstm_layers;    /* 1 or 2                                                          */
  int32_t precision;      /* 0: FP32 everywhere; 1: BF16 GEMM operands, FP32 accumulate;
                             2: as 1, but act-time (inference) encoder convolutions after the
                             stem take E4M3 operands with per-tensor scales (weights: amax /
                             448 at each weight refresh; activations: delayed, 2 amax / 448
                             of the previous act pass). Needs net_kind 1 and 64 | base_ch  */
  /* rollout / update shapes, used to size the workspace at creation */
  int32_t rollout_T;      /* T: frames per env per rollout (128)                             */
  int32_t minibatches;    /* PPO minibatches per epoch (E must divide evenly)                */
  int32_t encoder_chunk;  /* max frames per encoder pass in the update (0: min(all, 8192),
                             1024 for the SE-ResNeXt);
                             larger minibatches run in chunks, recomputed for the backward */
  /* task (Sec. 5 "Transfer Learning"): the reward env_step returns. Motion, episodes (stop
     or max_steps) and observations are the same for every task.
       0 PointGoal: -delta geodesic to the goal - 0.01 per step, terminal bonus (Sec. 4);
       1 Flee: r_t = 5 (D_t - D_t-1), D_t = Geo(s_t, s_0) / Max(s_0): the BFS geodesic from
         the episode's start cell, Max(s_0) the largest one reachable from it;
       2 Exploration: r_t = 0.25 (|Visited_t| - |Visited_t-1|), Visited_t the distinct
         squares of side explore_m (the paper's 1 m cubes, on the floor) occupied so far,
         the start's included. */
  int32_t task;
  float explore_m;        /* Exploration square side in metres (1.0)                        */
  uint64_t seed;          /* seeds the world (counter hash) and the initial weights          */
} ddppo_config;

/* Device views of one rollout (Sec. 4 "Training": T frames from each of E envs).
 * Slot t of obs/goal/prev_a/masks/values is the observation the policy acts on
 * at step t; slot T is the bootstrap observation. */
typedef struct {
  void* obs;            /* [dev] [T+1, E, 1, h, w]  encoder input, float (precision 0) or
                           bf16 (precision 1, 2); h = depth_h/(1+pool2x2), w likewise       */
  float* goal;          /* [dev] [T+1, E, 3]  [r (m), cos theta, sin theta]               */
  int32_t* prev_a;      /* [dev] [T+1, E]     previous action, 4 = start token             */
  uint8_t* masks;       /* [dev] [T+1, E]     0 at an episode's first frame, else 1        */
  int32_t* actions;     /* [dev] [T, E]                                                    */
  float* logp;          /* [dev] [T, E]       log pi_old(a_t | o_t)                        */
  float* values;        /* [dev] [T+1, E]     V(o_t); slot T bootstraps                    */
  float* rewards;       /* [dev] [T, E]                                                    */
  uint8_t* dones;       /* [dev] [T, E]       episode ended at step t                      */
  float* info;          /* [dev] [T, E, 4]    success, spl, collided, episode steps; NULL ok*/
  float* adv;           /* [dev] [T, E]       GAE advantages                               */
  float* ret;           /* [dev] [T, E]       returns adv + V                              */
  float* h0;            /* [dev] [L, E, hidden]  LSTM state before slot 0                  */
  float* c0;            /* [dev] [L, E, hidden]                                            */
  float* h;             /* [dev] [L, E, hidden]  running LSTM state (in/out)               */
  float* c;             /* [dev] [L, E, hidden]                                            */
  const float* uniforms;/* [dev] [T, E]  one U[0,1) draw per action sample                 */
} ddppo_rollout;

/* PPO hyper-parameters (Sec. 4 "Training": clip 0.2 by convention, 2 epochs x 2
 * minibatches, Adam lr 2.5e-4, gamma 0.99, GAE tau 0.95, no advantage
 * normalisation; value/entropy coefficients and grad clip are not stated). */
typedef struct {
  float clip;            /* epsilon of Eq. 2                          */
  float lr;              /* Adam step size                            */
  float value_coef;      /* c_v (0.5)                                 */
  float entropy_coef;    /* c_e (0.01)                                */
  float max_grad_norm;   /* global L2 clip (0.5); <= 0 disables       */
  float beta1, beta2;    /* Adam (0.9, 0.999)                         */
  float adam_eps;        /* Adam epsilon added to sqrt(v_hat) (1e-5)  */
  int32_t epochs;        /* 2                                         */
  int32_t minibatches;   /* 2; must equal the config's value          */
  int32_t norm_adv;      /* 0 (the paper's choice) or 1               */
  int32_t update_index;  /* seeds the per-epoch env permutation       */
} ddppo_ppo_hparams;

/* ---- lifetime --------------------------------------------------------------- */

/* Create a worker on the current CUDA device. Allocates (cudaMalloc) the
 * parameters (FP32, initialised from cfg->seed), Adam state, world state and all
 * workspace for the shapes in cfg. Not capturable. *out is set on success only.
 * Errors: E_ARG (null), E_CONFIG (unsupported shape), E_CUDA (allocation). */
int ddppo_create(const ddppo_config* cfg, ddppo_ctx** out);

/* The configuration checks of ddppo_create alone (the world, agent and training
 * settings of Sec. 4): host only, no CUDA call and no allocation. DDPPO_OK, or E_CONFIG with ddppo_last_error naming the first violated rule
 * (E_ARG for a null cfg). */
int ddppo_config_check(const ddppo_config* cfg);

/* Free everything ddppo_create allocated. Synchronises the device. NULL is a no-op. */
int ddppo_destroy(ddppo_ctx* ctx);

/* Message of the last failure on this thread ("" if none). Never NULL. */
const char* ddppo_last_error(void);

/* Sticky device status (DDPPO_OK or DDPPO_E_DEVICE_BOUNDS / DDPPO_E_TIMEOUT), read
 * with a device-to-host copy that synchronises `stream`. code_out: [host]. */
int ddppo_device_status(ddppo_ctx* ctx, int32_t* code_out, void* stream);

/* Cap on the level loop of the BFS geodesic field (Sec. 4 "Training": geodesic distance
 * to the goal), for tests of the device-side failure path. cap = 0 (the default) allows
 * G + 1 levels on a G-cell grid, more than any BFS needs; cap > 0 stops the loop after
 * cap levels. A BFS that still had cells to reach then sets the sticky E_TIMEOUT status,
 * leaves those cells unreachable (-1) and returns, so the launch completes and the
 * context stays usable. Takes effect for launches enqueued afterwards (a collect graph
 * keeps the value it was captured with). Host only. Errors: E_ARG (null, cap < 0). */
int ddppo_set_bfs_level_cap(ddppo_ctx* ctx, int32_t cap);

/* ---- parameters -------------------------------------------------------------- */

/* Number of FP32 parameters. The flat layout is the concatenation of the
 * tensors below in PyTorch's natural layouts (conv [Cout, Cin, kh, kw], linear
 * [out, in]), in this order:
 *   net_kind 0: c1.w [32,1,8,8] c1.b [32] c2.w [64,32,4,4] c2.b [64] c3.w [32,64,3,3] c3.b [32]
 *   net_kind 1: stem.w [c,1,7,7] stem.g [c] stem.b [c]; for each of the 8 BasicBlocks
 *               (widths c,c,2c,2c,4c,4c,8c,8c; first of each width > c has stride 2):
 *               c1.w n1.g n1.b c2.w n2.g n2.b [d.w (1x1) nd.g nd.b if it changes shape];
 *               cmp.w [128,8c,3,3] cmp.g [128] cmp.b [128]
 *   net_kind 2: nothing (no encoder)
 *   net_kind 3, 4: stem.w stem.g stem.b; for each bottleneck: c1.w [mid,cin,1,1] n1.g n1.b
 *               c2.w [mid,mid/32,3,3] n2.g n2.b c3.w [out,mid,1,1] n3.g n3.b se1.w [out/16,out]
 *               se1.b se2.w [out,out/16] se2.b [d.w [out,cin,1,1] nd.g nd.b if it changes
 *               shape]; cmp.w [128,last,3,3] cmp.g cmp.b
 *   then, except for net_kind 2, vis.w [H, F] vis.b [H] (F = flattened encoder output,
 *   C-major order); then goal.w [32,3] goal.b [32], act.emb [5,32],
 *   per LSTM layer l: w_ih [4H, In_l] w_hh [4H, H] b_ih [4H] b_hh [4H]
 *               (In_0 = H + 64, or 64 for net_kind 2; In_l = H; gate order i, f, g, o),
 *   actor.w [4,H] actor.b [4] critic.w [1,H] critic.b [1].
 * n_out: [host]. */
int ddppo_num_params(const ddppo_ctx* ctx, int64_t* n_out);

/* Copy the FP32 master parameters out of / into the worker. flat: [dev] [n].
 * n must equal ddppo_num_params. set_params also rebuilds the GEMM-layout
 * weight copies and resets the Adam moments and step count to zero. */
int ddppo_get_params(ddppo_ctx* ctx, float* flat, int64_t n, void* stream);
int ddppo_set_params(ddppo_ctx* ctx, const float* flat, int64_t n, void* stream);

/* Adam state: m, v [dev] [n] and the step count [host] (NULL to skip). */
int ddppo_get_adam(ddppo_ctx* ctx, float* m, float* v, int64_t n, int64_t* step, void* stream);

/* ---- environment (Sec. 4 "PointGoal Navigation", "Agent", "Training") -------- */

/* Start episode 0 of every env: generate the scene, draw the goal (uniform free
 * cell) and start (uniform among cells at geodesic >= 2 m; Sec. 4: random start
 * position and orientation), compute the BFS geodesic field from the goal, and
 * write the first observation: obs [dev] [E, 1, h, w] (pooled, / max_depth, in
 * the precision's dtype) and goal [dev] [E, 3]. */
int ddppo_env_reset(ddppo_ctx* ctx, void* obs, float* goal, void* stream);

/* Apply actions [dev] [E] in {0 stop, 1 forward 0.25 m, 2 left 10 deg,
 * 3 right 10 deg} (Sec. 4 "Agent"). Writes reward [dev] [E] (-delta geodesic -
 * 0.01 per step, terminal bonus on success; Sec. 4 "Training"), done [dev] [E]
 * (stop, or max_steps reached), info [dev] [E, 4] (success, SPL, collided,
 * steps; NULL ok). An env whose episode ended starts its next episode at once
 * and obs/goal [dev] are the new episode's first frame (auto-reset).
 * Errors: E_ARG; E_STATE before env_reset; out-of-range actions are caught on
 * the device (sticky E_DEVICE_BOUNDS) and treated as stop. */
int ddppo_env_step(ddppo_ctx* ctx, const int32_t* actions, void* obs, float* goal, float* reward,
                   uint8_t* done, float* info, void* stream);

/* Generate, ahead of time, the next episode of every env that has none prepared (scene,
 * geodesic field and start state, exactly as env_step's auto-reset would draw them) into
 * the env's second scene slot; an env_step that ends an episode then adopts the prepared
 * slot instead of generating it. Meant for a second stream, overlapping the policy's
 * forward pass (ddppo_collect does this); it must not overlap env_reset, env_step or
 * env_set_state of the same context. Results are identical with or without it.
 * Errors: E_STATE before env_reset. */
int ddppo_env_prefetch(ddppo_ctx* ctx, void* stream);

/* Parity / debugging views. state [dev] [E, DDPPO_NSTATE] int32: x, y (u),
 * heading (0..35, 10 deg steps counter-clockwise from +x), steps, path length
 * (u), previous geodesic (u), start geodesic l (u), goal x, goal y (u), episode,
 * grid side (cells), collided. grids [dev] [E, grid_max^2] uint8 (1 = wall) and
 * dists [dev] [E, grid_max^2] int32 (BFS cells from the goal, -1 unreachable)
 * hold each env's current episode with row stride = its grid side.
 * depth [dev] [E, depth_h, depth_w] float: the un-pooled depth image (metres) of
 * the current state. Either pointer of env_grids may be NULL. */
int ddppo_env_state(ddppo_ctx* ctx, int32_t* state, void* stream);
int ddppo_env_grids(ddppo_ctx* ctx, uint8_t* grids, int32_t* dists, void* stream);
int ddppo_env_depth(ddppo_ctx* ctx, float* depth, void* stream);

/* Overwrite the agent states [dev] [E, DDPPO_NSTATE] (same layout as env_state)
 * keeping the current scenes; for tests that place agents by hand. Discards prepared
 * next episodes (they were drawn for the replaced episode counters). */
int ddppo_env_set_state(ddppo_ctx* ctx, const int32_t* state, void* stream);

/* ---- policy (App. "Agent Design") -------------------------------------------- */

/* One inference step for all E envs: encoder -> FC -> concat(goal FC, previous
 * action embedding) -> LSTM (state reset where masks == 0) -> softmax actor +
 * critic; the action is a = min{k : CDF_k > u} for the caller's uniform u.
 * obs [dev] [E,1,h,w] (dtype of the precision), goal [dev] [E,3], prev_a [dev]
 * [E], masks [dev] [E], h/c [dev] [L,E,H] in/out, uniforms [dev] [E];
 * action [dev] [E], logp [dev] [E], value [dev] [E]. */
int ddppo_policy_act(ddppo_ctx* ctx, const void* obs, const float* goal, const int32_t* prev_a,
                     const uint8_t* masks, float* h, float* c, const float* uniforms,
                     int32_t* action, float* logp, float* value, void* stream);

/* Forward over a [T, E] segment (T <= rollout_T, T*E <= rollout_T*num_envs/minibatches)
 * from the LSTM state h0/c0 [dev] [L,E,H], keeping the activations for
 * ddppo_policy_backward. Inputs as in policy_act with a leading T axis.
 * logits [dev] [T,E,4], values [dev] [T,E]. */
int ddppo_policy_evaluate(ddppo_ctx* ctx, int32_t T, int32_t E, const void* obs, const float* goal,
                          const int32_t* prev_a, const uint8_t* masks, const float* h0,
                          const float* c0, float* logits, float* values, void* stream);

/* Backward of the last ddppo_policy_evaluate: hand-written gradients of the
 * heads, the LSTM (back-propagation through time over the segment) and the
 * encoder. dlogits [dev] [T,E,4], dvalues [dev] [T,E]; grad [dev] [n_params] is
 * overwritten with d(sum dlogits*logits + dvalues*values)/d theta in the flat
 * layout of ddppo_num_params. Errors: E_STATE without a preceding evaluate. */
int ddppo_policy_backward(ddppo_ctx* ctx, const float* dlogits, const float* dvalues, float* grad,
                          void* stream);

/* The visual encoder alone (App. "Visual Encoder"; the 3-layer conv, or the ResNet with
 * GroupNorm and the compression layer): features feat [dev] [N, F] fp32 of obs [dev]
 * [N, 1, h, w] (the precision's dtype), F = C x HW in channel-major order (feature
 * c * HW + p, the column order of vis.w), the post-ReLU output of the last layer.
 * 1 <= N <= rollout_T * num_envs / minibatches; larger N: E_CONFIG; the blind agent
 * (net_kind 2): E_CONFIG. ddppo_encoder_backward: the hand-written backward of the last
 * encoder_forward for dfeat [dev] [N, F] (same layout); grad [dev] [n_params] is
 * overwritten, nonzero only in the encoder's tensors. Any other forward of the context
 * in between (act, evaluate, collect, update, lstm_forward) invalidates it: E_STATE. */
int ddppo_encoder_forward(ddppo_ctx* ctx, int32_t N, const void* obs, float* feat, void* stream);
int ddppo_encoder_backward(ddppo_ctx* ctx, const float* dfeat, float* grad, void* stream);

/* The LSTM layers alone over a [T, E] segment (App. "Navigation Policy"; gates i, f, g, o,
 * state reset where masks == 0 before a step): in [dev] [T, E, In_0] fp32 (the layer-0
 * input [visual FC | goal FC | action embedding], rounded to the operand dtype as the
 * network does), masks [dev] [T, E], h0/c0 [dev] [L, E, H]; y [dev] [T, E, H] the top
 * layer's output. ddppo_lstm_backward: back-propagation through time of the last
 * lstm_forward for dy [dev] [T, E, H]; dx [dev] [T, E, In_0] (NULL ok) receives the
 * input gradient; grad [dev] [n_params] is overwritten, nonzero only in the LSTM's
 * tensors. Same workspace limits and invalidation as the encoder pair. */
int ddppo_lstm_forward(ddppo_ctx* ctx, int32_t T, int32_t E, const float* in, const uint8_t* masks,
                       const float* h0, const float* c0, float* y, void* stream);
int ddppo_lstm_backward(ddppo_ctx* ctx, const float* dy, float* dx, float* grad, void* stream);

/* ---- learning (Sec. 2 Eq. 1-2; Sec. 4 "Training") ----------------------------- */

/* Generalised advantage estimation, one warp-level reverse scan per env:
 *   delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t,  A_t = delta_t + gamma lam (1 - d_t) A_{t+1},
 *   R_t = A_t + V_t.
 * reward, adv, ret [dev] [T,E]; done [dev] [T,E] (nonzero = episode ended at t);
 * value [dev] [T+1,E]. Stateless: needs no ctx. */
int ddppo_gae(const float* reward, const uint8_t* done, const float* value, int32_t T, int32_t E,
              float gamma, float lam, float* adv, float* ret, void* stream);

/* PPO loss over n samples (Eq. 2 plus value and entropy terms):
 *   L = -mean(min(rho A, clip(rho, 1-eps, 1+eps) A)) + c_v 0.5 mean((R-V)^2) - c_e mean(H)
 * with rho = exp(log pi(a) - logp_old). logits [dev] [n,4], values, adv, ret,
 * logp_old [dev] [n], actions [dev] [n]. Writes stats [dev] [DDPPO_NSTATS] = loss,
 * policy loss, value loss, entropy, clip fraction, approx KL, 0, 0 and the exact
 * gradients dlogits [dev] [n,4], dvalues [dev] [n]. Reductions are in a fixed
 * order (deterministic). Stateless. */
int ddppo_ppo_loss(int32_t n, const float* logits, const float* values, const int32_t* actions,
                   const float* logp_old, const float* adv, const float* ret, float clip,
                   float value_coef, float entropy_coef, float* stats, float* dlogits,
                   float* dvalues, void* stream);

/* The PPO loss of ddppo_ppo_loss (same arguments, same outputs) for callers that cannot
 * allocate device memory where they need it, for instance inside a stream capture that
 * forbids cudaMalloc or in a process whose device memory belongs to another allocator.
 * The paper has no counterpart: this is a deployment variant. Samples are spread over
 * one thread block per 256 (ddppo_ppo_loss uses one block); the per-block partial sums
 * live in an 80 KiB array owned by the library, so nothing is allocated and no context
 * is needed. n must be at most 1,048,576 (E_CONFIG otherwise). The first call on each
 * device looks up the array's device address; make it before any stream capture. Every
 * call shares the array, so calls that overlap on the GPU race. Each call overwrites the
 * partials it uses; nothing needs clearing between calls. The looked-up address is kept
 * for the life of the process: after a cudaDeviceReset of a device, do not call this
 * entry point on that device again in the same process. */
int ddppo_ppo_loss_static(int32_t n, const float* logits, const float* values,
                          const int32_t* actions, const float* logp_old, const float* adv,
                          const float* ret, float clip, float value_coef, float entropy_coef,
                          float* stats, float* dlogits, float* dvalues, void* stream);

/* One PPO update on a collected rollout (ro->adv/ret already filled by ddppo_gae):
 * hp->epochs x hp->minibatches steps; minibatch k of epoch e holds the envs
 * perm[k*E/mb, (k+1)*E/mb) of a Fisher-Yates permutation drawn from the counter
 * hash (seed, update_index, epoch), with their full T-step sequences replayed
 * from ro->h0/c0. Each step: forward, loss, hand-written backward, global-norm
 * clip, Adam. stats [dev] [epochs*minibatches, DDPPO_NSTATS] (NULL ok): loss,
 * policy loss, value loss, entropy, clip fraction, approx KL, grad norm, 0. */
int ddppo_ppo_update(ddppo_ctx* ctx, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                     float* stats, void* stream);

/* Collect one rollout (Sec. 3: the collection stage of the synchronous loop):
 * copy slot T of the previous rollout to slot 0 (first call: env_reset), save
 * the LSTM state to h0/c0, then T times {policy_act on slot t -> env_step ->
 * slot t+1}, then the bootstrap value V(o_T). With use_graph = 1 the T-step loop
 * is captured once into a CUDA graph and replayed on later calls with the same
 * rollout pointers (the first call with new pointers captures and is not itself
 * capturable). */
int ddppo_collect(ddppo_ctx* ctx, const ddppo_rollout* ro, int32_t use_graph, void* stream);

/* ---- DD-PPO workers: step-wise collection with preemption, exchanged gradients ----- */

/* The collection stage one step at a time, for workers whose collection can be preempted
 * (Sec. 3: once p% of the workers have finished their rollout, the stragglers' collection
 * ends early, but not before one quarter of the rollout length). collect_begin is
 * ddppo_collect's prologue: slot 0 <- the previous collection's last slot (slot T, or
 * T_valid after a preempted one; the first call resets the world), h0/c0 <- h/c.
 * collect_step(t), for t = 0, 1, ... in order (t < rollout_T): act on slot t, env_step,
 * slot t + 1 (the next episodes prepared on the side stream meanwhile). collect_end
 * writes the bootstrap value of slot T_valid, T_valid = the steps taken (>= 1); a
 * following ddppo_collect or collect_begin continues from that slot. Launches directly
 * (no graph). The results of begin + rollout_T steps + end equal ddppo_collect's.
 * Errors: E_ARG (null argument or buffer), E_STATE (steps out of order, T_valid wrong). */
int ddppo_collect_begin(ddppo_ctx* ctx, const ddppo_rollout* ro, void* stream);
int ddppo_collect_step(ddppo_ctx* ctx, const ddppo_rollout* ro, int32_t t, void* stream);
int ddppo_collect_end(ddppo_ctx* ctx, const ddppo_rollout* ro, int32_t T_valid, void* stream);

/* The update one minibatch at a time, for workers that exchange gradients (Eq. 4:
 * theta <- ParamUpdate(theta, AllReduce(grad_1, ..., grad_N)), the mean over workers).
 * ddppo_ppo_grad: the gradient of minibatch k (0 <= k < minibatches) of epoch `epoch` of
 * an update with hp->update_index -- the same envs, replay, loss and hand-written
 * backward as ddppo_ppo_update -- over the first T_valid steps of the rollout (a
 * preempted worker's shorter rollout; its loss is the mean over its own samples, so every
 * worker weighs equally, as Sec. 3 states). grad [dev] [n_params] receives the unclipped
 * gradient; stats [dev] [DDPPO_NSTATS] (NULL ok) the loss statistics. ro->adv/ret must
 * hold GAE over the same T_valid steps (ddppo_gae with T = T_valid).
 * ddppo_apply_grad: ParamUpdate with grad [dev] [n_params] times `scale` (1/N for a sum
 * over N workers): global-norm clip, one Adam step (the worker's step count + 1), the
 * GEMM-layout weights refreshed; stats [dev] (NULL ok) receives the norm in slot 6.
 * Calling ppo_grad and apply_grad (scale 1) for every epoch and minibatch in order gives
 * ddppo_ppo_update's parameters bit for bit.
 * ddppo_grad_mean: out [dev] [len] = (1/n) sum_r bufs[r] [dev] [len], summed in the order
 * r = 0 .. n-1 (deterministic): the AllReduce of workers that share a GPU; bufs [host]
 * holds n <= 64 device pointers. Errors: E_ARG, E_CONFIG (shapes), E_CUDA. */
int ddppo_ppo_grad(ddppo_ctx* ctx, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                   int32_t T_valid, int32_t epoch, int32_t k, float* grad, float* stats,
                   void* stream);
int ddppo_apply_grad(ddppo_ctx* ctx, const float* grad, float scale, const ddppo_ppo_hparams* hp,
                     float* stats, void* stream);
int ddppo_grad_mean(int32_t n, const float* const* bufs, int64_t len, float* out, void* stream);

/* ---- checkpoint / resume ---------------------------------------------------------- */

/* Write / read a worker's whole learning state to / from the file `path` [host], so that
 * a run can stop and resume bit-identically (the paper trains for days under a cluster
 * scheduler that preempts and restarts jobs; Sec. 3, Sec. 4 "Training"). The file holds
 * the configuration (ddppo_load rejects a file written by a worker with another one:
 * E_CONFIG), the FP32 parameters, the Adam moments and step count, the world (both scene
 * slots of every env with their grids, wall bits and BFS fields; agent states; prepared
 * next episodes), FP8 inference's delayed activation scales and the GEMM autotuner's
 * table. With a rollout view ro (NULL ok), it also holds the state the next
 * ddppo_collect carries over: slot T of obs, goal, prev_a and masks, and the LSTM state
 * ro->h, ro->c; a file written with ro must be loaded with ro (into any rollout view of
 * the same shapes), and the next ddppo_collect then continues the saved run. Loaded
 * without rollout state, the next ddppo_collect starts from env_reset. The update index
 * (hparams) and the action uniforms stay with the caller. Both synchronise `stream`
 * and are not capturable; save reads the state once every call enqueued on `stream`
 * has finished. Errors: E_ARG (null argument, file cannot be opened or written),
 * E_CONFIG (not a checkpoint of this library and configuration, a section of the wrong
 * size, a truncated file), E_CUDA. */
int ddppo_save(ddppo_ctx* ctx, const ddppo_rollout* ro, const char* path, void* stream);
int ddppo_load(ddppo_ctx* ctx, const ddppo_rollout* ro, const char* path, void* stream);

/* ---- contraction utility --------------------------------------------------------- */

/* The GEMM every layer of the network runs on:
 *   C[M, N] = beta * C + sum_k A(m, k) B(n, k) (+ bias[N]) (then ReLU if relu)
 * A [dev] is [M, K] row-major (A(m,k) = A[m*lda + k], lda >= K) or, with a_t, stored
 * [K, M] (A(m,k) = A[k*lda + m], lda >= M); B likewise with b_t ([N, K] or [K, N]).
 * Operands are float (op_bf16 = 0, SIMT FMA) or bf16 (op_bf16 = 1; on sm_103a the
 * tcgen05 tensor-core path with fp32 accumulation when rows are 16-byte aligned). C [dev]
 * row-major fp32, or bf16 when c_bf16 (then beta must be 0). bias [dev] [N] or NULL.
 * status [dev] int32 or NULL receives the sticky timeout flag (2) of a bounded
 * tensor-core wait. The first call per device allocates a split-K workspace (not
 * capturable). */
int ddppo_gemm(int32_t M, int32_t N, int32_t K, int32_t op_bf16, const void* A, int32_t lda,
               int32_t a_t, const void* B, int32_t ldb, int32_t b_t, void* C, int32_t ldc,
               int32_t c_bf16, float beta, const float* bias, int32_t relu, int32_t* status,
               void* stream);
/* A convolution on the tensor cores without an im2col matrix (the encoder of Sec. 4):
 * y = beta y + conv(x, w). Either the GEMM kernel gathers each K-block of the input patch
 * matrix with one 4-D TMA copy of the input (filter tap shifts the box, the stride is the
 * copy's traversal stride, zero padding is the copy's out-of-bounds fill), or, for
 * stride-1 'same' convolutions of 32-channel inputs, each 128-pixel tile stages one input
 * box with its filter halo and every tap reads it through a row-shifted operand view.
 * x [dev] NHWC bf16 [N, H, W, C]; w [dev] bf16 [Cout, k*k*C] with K ordered (ky, kx, c);
 * y [dev] fp32 NHWC [N, Ho, Wo, Cout] (read when beta != 0). Requires C % 32 == 0 and an
 * output width dividing 128 (whole output rows per 128-pixel tile), or stride 1, odd k,
 * p = k / 2, C == 32, Cout <= 128 and W + 2p <= 256, or -- the encoder's stem -- C == 1,
 * k * k <= 64 and Cout 16, 32 or 64 (each 128-pixel tile's patches gathered by the CTA
 * into shared memory, the weights resident; at most 2^30 output pixels); E_CONFIG
 * otherwise. status as for ddppo_gemm. The first call per device allocates a split-K
 * workspace. */
int ddppo_conv2d(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                 int32_t stride, int32_t pad, const void* x, const void* w, float* y,
                 float beta, int32_t* status, void* stream);
/* The weight gradient of that convolution without an im2col matrix (the backward pass of
 * Sec. 4's encoder): dw[co, (ky*k + kx)*C + c] = beta dw + sum over n, oy, ox of
 * dy[n, oy, ox, co] x[n, oy*s - p + ky, ox*s - p + kx, c] (zero outside the image).
 * The GEMM's reduction runs over output pixels in 64-pixel blocks, each gathered per
 * filter tap with a 4-D TMA copy. x [dev] NHWC bf16 [N, H, W, C]; dy [dev] bf16
 * [N, Ho, Wo, Cout]; dw [dev] fp32 [Cout, k*k*C]. Requires C == 32 or C % 64 == 0,
 * Cout % 8 == 0, an output width dividing 64 and whole 64-pixel blocks (Ho*Wo a multiple
 * of 64 made of whole rows, or a divisor of 64); E_CONFIG otherwise. status and the
 * workspace as for ddppo_conv2d. */
int ddppo_conv2d_wgrad(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                       int32_t stride, int32_t pad, const void* x, const void* dy, float* dw,
                       float beta, int32_t* status, void* stream);
/* E4M3 contractions: the encoder convolutions of Sec. 4 "Agent" / App. "Visual Encoder"
 * at FP8 inference precision (E4M3 operands, per-tensor scales, fp32 accumulation).
 * ddppo_quantize_e4m3: per-tensor quantisation of n values x [dev] (fp32, or bf16 when
 * x_bf16): scale [dev] float = amax(|x|) / 448 (1 when every x is 0); q [dev] uint8 [n] =
 * e4m3(x / scale), rounded to nearest even, saturating at +-448.
 * ddppo_gemm_e4m3: C[M, N] = beta C + sa sb sum_k A[m, k] B[n, k] (+ bias) (ReLU), A and B
 * E4M3 K-major with K, lda, ldb even and 16-byte aligned rows (16 | lda, ldb), sa = *scale_a,
 * sb = *scale_b [dev] (NULL reads 1); C fp32. tcgen05 kind::f8f6f4, fp32 accumulation.
 * ddppo_conv2d_e4m3: ddppo_conv2d with E4M3 x [dev] NHWC and w [dev] [Cout, k*k*C], y =
 * beta y + sx sw conv(x, w); C a multiple of 64 (gather path) or C = 64 with stride 1 and
 * p = k / 2 (halo path). All three: E_CONFIG for unsupported shapes, status as ddppo_gemm. */
int ddppo_quantize_e4m3(const void* x, int32_t x_bf16, int64_t n, void* q, float* scale,
                        void* stream);
int ddppo_gemm_e4m3(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B,
                    int32_t ldb, const float* scale_a, const float* scale_b, float* C, int32_t ldc,
                    float beta, const float* bias, int32_t relu, int32_t* status, void* stream);
int ddppo_conv2d_e4m3(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                      int32_t stride, int32_t pad, const void* x, const void* w,
                      const float* scale_x, const float* scale_w, float* y, float beta,
                      int32_t* status, void* stream);

/* GroupNorm of the encoder (App. "Visual Encoder": GroupNorm in place of BatchNorm; C/2
 * groups of 2 channels, eps 1e-5): out = act(gn(z) gamma + beta + resid) over NHWC z [dev]
 * fp32 [N, HW, C]; gamma, beta [dev] [C]; resid [dev] [N, HW, C] or NULL; relu 0/1; mean,
 * rstd [dev] [N, C/2] receive the group statistics. N <= 8192, C even <= 1024 (E_ARG
 * otherwise). The first call per device allocates a scratch (not capturable). */
int ddppo_group_norm(int32_t N, int32_t HW, int32_t C, const float* z, const float* gamma,
                     const float* beta, const float* resid, int32_t relu, float* out, float* mean,
                     float* rstd, void* stream);
/* How the encoder's forward GroupNorms run. An image of at most 32K elements is summed by
 * one block: with at least 4 images per SM the same block then normalises it (one launch,
 * the image re-read from L2); with fewer, a second launch normalises it, spread over many
 * blocks. A larger
 * image is split over S blocks: with on = 1 (the default) the statistics and the
 * normalisation run in one cooperative launch wherever every block fits on the GPU at once
 * (the image's blocks meet at a bounded per-image barrier, then normalise the rows they
 * summed), otherwise, and with on = 0, as a statistics launch then a normalise launch.
 * Both forms use the same S, so their results are bit-identical. ddppo_group_norm follows
 * the same rules. Applies to launches enqueued afterwards. Host only. */
int ddppo_group_norm_one_launch(ddppo_ctx* ctx, int32_t on);

/* The SE-ResNeXt bottleneck's own kernels (App. "Visual Encoder"; ResNeXt's grouped
 * convolution; squeeze-and-excitation), stand-alone, fp32 NHWC:
 * ddppo_grouped_conv3x3: z [dev] [N, Ho, Wo, C] = the 3x3 convolution, padding 1, of x
 * [dev] [N, H, W, C] with `groups` groups, weights w [dev] [C, C/groups, 3, 3] (PyTorch's
 * grouped layout); C / groups <= 16, C <= 1024, stride 1 or 2 (E_ARG otherwise); the first
 * call per device allocates a weight scratch (not capturable).
 * ddppo_squeeze_excite: for u [dev] [N, HW, C]: m = mean_hw u [N, C], a = relu(W1 m + b1)
 * [N, Cr], gate = sigmoid(W2 a + b2) [N, C], y = relu(u gate + sc) [N, HW, C] (sc [dev] or
 * NULL); W1 [Cr, C], b1 [Cr], W2 [C, Cr], b2 [C]; every output [dev]. */
int ddppo_grouped_conv3x3(int32_t N, int32_t H, int32_t W, int32_t C, int32_t groups, int32_t stride,
                          const float* x, const float* w, float* z, void* stream);
int ddppo_squeeze_excite(int32_t N, int32_t HW, int32_t C, int32_t Cr, const float* u,
                         const float* sc, const float* W1, const float* b1, const float* W2,
                         const float* b2, float* m, float* a, float* gate, float* y, void* stream);

/* The paths and shared-memory staging geometry the tensor-core engine would use for a
 * bf16 convolution of this shape (the encoder of Sec. 4 "Agent") and for its weight
 * gradient. Host only: no CUDA call, no
 * device needed. plan [host] int32 [18]:
 *   [0] 4-D gather forward path usable; [1] halo forward path usable (1: anchor halo, 2:
 *   row halo -- 3x3 filters, W in {8, 16, 32}, H >= 128 / W, Cout <= 32: whole image rows
 *   per tile, the three column taps in one MMA, the default path for such shapes), then
 *   [2] anchor pitch Wp = W + 2p (row halo: W), [3] padded height Hh (row halo: H), [4]
 *   images per 128-anchor tile (0: tiles within one image), [5] tiles per image, [6] box
 *   rows per image, [7] anchor rows allocated per ring stage, [8] anchor rows the box
 *   delivers, [9] tiles;
 *   [10] 4-D gather weight gradient usable; [11] halo weight gradient usable, then [12]
 *   rows per work unit RB, [13] pitch Wp, [14] input box rows, [15] dz box rows, [16] ring
 *   depth, [17] shared memory bytes per CTA.
 * E_ARG for invalid sizes or a null plan. */
int ddppo_conv_plan(int32_t N, int32_t H, int32_t W, int32_t C, int32_t Cout, int32_t k,
                    int32_t stride, int32_t pad, int32_t* plan);

/* Whether ddppo_gemm with these operands runs on the tensor cores (1) or SIMT (0). */
int ddppo_gemm_backend(int32_t M, int32_t N, int32_t K, int32_t op_bf16, const void* A,
                       int32_t lda, const void* B, int32_t ldb, int32_t* tensor_cores);

/* The PPO update (ddppo_ppo_update) is recorded once as a CUDA graph (after its first,
 * directly launched run) and replayed while its rollout view, statistics buffer and
 * hyper-parameters other than update_index stay the same; GEMM timing, when enabled, is
 * recorded inside the graph. on = 0 launches every update directly (debugging); results
 * are bit-identical either way. */
int ddppo_update_graph(ddppo_ctx* ctx, int32_t on);

/* The LSTM recurrence (App. "Agent Design"; Sec. 4 "Training": BPTT over the rollout).
 * mode 2: in the BF16 forms the forward of each layer runs all T steps in
 * one launch on the tensor cores (tcgen05, M = 128 gate rows per CTA, the CTA's rows of
 * W_hh resident in shared memory, the cell update fused into the TMEM epilogue, one
 * bounded grid barrier per step) wherever the shape allows (H a multiple of 64, at most
 * 128 envs per segment, 64 when H = 512); the backward, the FP32 form and other shapes
 * run step by step. mode 0 (the default): a recurrent contraction and a cell kernel per
 * step, forward and backward. mode 1: forward and backward as one cooperative launch per layer on the
 * CUDA cores (recurrent weights in registers; at most 64 envs per segment); slower than
 * mode 0 at the default sizes (its per-step contraction is bound by shared-memory loads).
 * All modes compute the same arithmetic; only the recurrent contraction's fp32 summation
 * order differs. Applies to launches enqueued afterwards (a captured graph keeps the mode
 * it was captured with). E_ARG for another mode. Host only. */
int ddppo_lstm_whole_segment(ddppo_ctx* ctx, int32_t mode);

/* Launch overlap (process-wide; not a method step): every kernel of the library is
 * launched with programmatic dependent launch, so its blocks become resident and run their
 * prologue (barrier set-up, tensor-memory allocation) while the previous kernel in the
 * stream finishes; each kernel waits for that kernel's completion before it reads or
 * writes global memory, so results are bit-identical either way. on = 0 launches with
 * plain stream order. The initial state is on unless the environment variable
 * DDPPO_LAUNCH_OVERLAP is "0". Applies to launches enqueued afterwards; a graph captured
 * earlier (collect, update) keeps the form it was captured with. Host only. */
int ddppo_set_launch_overlap(int32_t on);
/* on [host]: the current state (1 on, 0 off). */
int ddppo_launch_overlap(int32_t* on);

/* Tensor-store epilogue (process-wide; not a method step): a tensor-core contraction tile
 * whose rows are whole rows of the output (plain GEMM, convolution tiles, the row halo),
 * with nothing accumulated into C and no split-K, hands its result to one tensor copy
 * (cp.async.bulk.tensor) per 32 x 32 block from shared memory instead of transposing it
 * and storing it row by row. The values are formed identically (scale, bias, ReLU, output
 * type), so results are bit-identical either way. on = 0 keeps the per-row stores. The
 * initial state is on unless the environment variable DDPPO_TMA_EPILOGUE is "0". Applies
 * to launches enqueued afterwards; a captured graph keeps the form it was captured with.
 * Host only. */
int ddppo_set_tma_epilogue(int32_t on);
/* on [host]: the current state (1 on, 0 off). */
int ddppo_tma_epilogue(int32_t* on);

/* Tile-shape autotuner of the tensor-core GEMM (precision 1): on by default. The first
 * time a contraction shape is seen outside a stream capture, each candidate (N tile 64 or
 * 128, ring depth 2-4, split-K or not) runs on a scratch output and the fastest is kept;
 * ddppo_collect runs one act step outside its capture for this. on = 0 freezes the table
 * (new shapes use the fixed heuristic). tuned_shapes [host] (NULL ok): table size. */
int ddppo_autotune(ddppo_ctx* ctx, int32_t on, int64_t* tuned_shapes);

/* Save and restore the autotuner's table (a tuning cache), so that a later process --
 * for instance one run under a profiler, whose serialised launches would distort the
 * trial timings -- launches the same configurations without re-tuning.
 * export: buf [host] (NULL: size query) of cap bytes; size [host] receives the image's
 *   byte count; DDPPO_E_CONFIG when buf is non-NULL and cap < size.
 * import: buf [host] of size bytes from an export (same library version); its entries
 *   replace equal shapes; DDPPO_E_CONFIG on a malformed image or when precision is 0
 *   (no tensor-core GEMM). The image is plain int32 words in host byte order. */
int ddppo_autotune_export(ddppo_ctx* ctx, void* buf, size_t cap, size_t* size);
int ddppo_autotune_import(ddppo_ctx* ctx, const void* buf, size_t size);

/* Per-kernel-family timing of the calls enqueued while enabled (CUDA events on
 * the launching stream). ddppo_timing_enable(ctx, 1) starts recording and
 * clears the counters; ddppo_timing_read synchronises and returns, for family
 * id (0: tensor-core / SIMT GEMM, 1: ray cast), the summed milliseconds, launch
 * count and algorithmic work (FLOPs for GEMM, output bytes for the ray cast). */
int ddppo_timing_enable(ddppo_ctx* ctx, int32_t on);
int ddppo_timing_read(ddppo_ctx* ctx, int32_t family, double* ms, int64_t* launches, double* work);
/* family 2 reports the launches and FLOPs of the contractions that ran on the tcgen05
 * tensor-core GEMM; its `ms` slot carries the FLOPs of all contractions while enabled. */

/* Per-launch records of the timed launches of a family since ddppo_timing_enable: event
 * time ms[i], work[i] (FLOPs for family 0, output bytes for 1) and the algorithmic HBM
 * bytes[i] (operands read once, result written once). Arrays [host] of cap entries (any
 * may be NULL); count [host] receives the number of records (at most 4096 per family).
 * Synchronises on the recorded events. */
int ddppo_timing_launches(ddppo_ctx* ctx, int32_t family, double* ms, double* work, double* bytes,
                          int64_t cap, int64_t* count);

/* Number of kernel launches of one steady-state iteration (collect of T steps, bootstrap
 * value, GAE, PPO update) with this rollout and hyper-parameters: the iteration is
 * captured into a CUDA graph that is counted and discarded, nothing executes. Needs a
 * preceding ddppo_collect. count: [host]. Synchronises the device. */
int ddppo_count_kernels(ddppo_ctx* ctx, const ddppo_rollout* ro, const ddppo_ppo_hparams* hp,
                        float gamma, float lam, int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* DDPPO_H */
