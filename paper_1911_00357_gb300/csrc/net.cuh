// The agent network (App. "Agent Design") held by a worker: parameters, Adam state,
// GEMM-layout weights and all workspace, sized at creation for the configured shapes.
#pragma once

#include <vector>

#include "ctx.cuh"
#include "gemm.cuh"
#include "nn_kernels.cuh"

namespace ddppo {

struct ConvL {
  int cin = 0, cout = 0, k = 0, s = 1, p = 0;
  bool bias = false;
  int64_t w_off = -1, b_off = -1;
  int Kp = 0;
  int H = 0, W = 0, Ho = 0, Wo = 0;
  void* wg = nullptr;   // [cout, Kp] op dtype
  void* wgT = nullptr;  // [Kp, cout] op dtype (dgrad through col2im)
  void* wgR = nullptr;  // [cin, k*k*cout] op dtype: flipped, channel-swapped kernel (stride-1 dgrad)
  bool dgrad_as_conv = false;
  float* dwg = nullptr; // [cout, Kp] fp32 gradient in GEMM layout
  float* z = nullptr;   // [NC, Ho, Wo, cout] conv output (fp32)
  // FP8 inference: E4M3 copy of wg with its per-tensor scale (device scalar) and absolute
  // maximum (float bits); null where the input channels are not a multiple of 64
  uint8_t* wg8 = nullptr;
  float* w8_scale = nullptr;
  unsigned* w8_amax = nullptr;
};

struct GNL {
  int C = 0;
  int64_t g_off = -1, b_off = -1;
  float* mean = nullptr;  // [NC, C/2]
  float* rstd = nullptr;
  float* out = nullptr;   // [NC, HW, C] post-activation output (when materialised)
  __nv_bfloat16* out_bf = nullptr;  // its bf16 copy (BF16 form: the next conv's TMA operand)
  uint8_t* out_f8 = nullptr;        // [E, HW, C] its E4M3 copy (FP8 inference)
  int f8_slot = -1;                 // activation scale slot of out_f8
};

struct BlockL {
  ConvL c1, c2, d;
  GNL n1, n2, nd;
  bool down = false;
  float* y = nullptr;     // block output [NC, Ho, Wo, cout]
  __nv_bfloat16* y_bf = nullptr;  // its bf16 copy (BF16 form)
  uint8_t* y_f8 = nullptr;        // [E, Ho, Wo, cout] its E4M3 copy (FP8 inference)
  int y_slot = -1;
};

// grouped 3x3 convolution of an SE-ResNeXt bottleneck (cpg = C / 32 channels per group)
struct GConvL {
  int C = 0, cpg = 0, s = 1, H = 0, W = 0, Ho = 0, Wo = 0;
  int64_t w_off = -1;    // canonical [C, cpg, 3, 3] in the flat parameters
  void* wg = nullptr;    // [C][3][3][cpg] op dtype
  float* z = nullptr;    // [NC, Ho, Wo, C] output (fp32)
};

// SE-ResNeXt bottleneck (App. "Visual Encoder"): 1x1 conv -> GN -> ReLU -> grouped 3x3
// -> GN -> ReLU -> 1x1 conv -> GN (u) -> squeeze-excite -> + shortcut -> ReLU
struct SxL {
  ConvL c1, c3, d;
  GConvL c2;
  GNL n1, n2, n3, nd;
  bool down = false;
  int C = 0, Cr = 0, HW = 0;  // output channels, squeeze width (C / 16), output pixels
  int64_t se1_w = -1, se1_b = -1, se2_w = -1, se2_b = -1;
  float* u = nullptr;     // [NC, HW, C] the branch before the excitation
  float* sc = nullptr;    // [NC, HW, C] the normalised 1x1 shortcut (when down)
  float* m = nullptr;     // [NC, C] squeeze means
  float* a = nullptr;     // [NC, Cr] squeeze FC output (after ReLU)
  float* gate = nullptr;  // [NC, C] excitation gates
  float* y = nullptr;     // [NC, HW, C] block output
  __nv_bfloat16* y_bf = nullptr;  // its bf16 copy (BF16 form)
};

struct LstmL {
  int In = 0;
  int64_t wih = -1, whh = -1, bih = -1, bhh = -1;
  void* Wih = nullptr;   // [4H, In] op
  void* WihT = nullptr;  // [In, 4H] op
  void* Whh = nullptr;   // [4H, H] op
  void* WhhT = nullptr;  // [H, 4H] op
  float* bsum = nullptr; // [4H]
  float* gates = nullptr;// [NS, 4H]
  float* c = nullptr;    // [NS, H]
  float* h = nullptr;    // [NS, H]
  void* hm = nullptr;    // [NS, H] op: masked state entering each step
  void* y = nullptr;     // [NS, H] op: layer output
};

struct Net {
  ddppo_ctx* x = nullptr;
  bool bf = false;
  // FP8 inference (precision 2): the act-time encoder convolutions after the stem take
  // E4M3 operands; training (evaluate, update) stays BF16
  bool f8 = false;
  uint8_t* pool_f8 = nullptr;  // [E, pooled HW, C] E4M3 copy of the stem output
  int pool_slot = -1;
  float* f8_scale = nullptr;   // [f8_slots] device: activation scales (delayed), weight scales
  unsigned* f8_amax = nullptr; // [f8_slots] device: absolute maxima (float bits)
  float* f8_keep = nullptr;    // [2 f8_act_slots] activation scales / maxima kept aside
  int f8_act_slots = 0, f8_slots = 0;
  int kind = 0, H = 0, L = 0, inh = 0, inw = 0;
  int F = 0, featC = 0, featHW = 0;
  int E = 0, T = 0, Emb = 0, NS = 0, NC = 0;
  int In0 = 0, InMax = 0;
  int emb_col0 = 0;  // column of the goal FC in the LSTM input (after the visual FC, if any)
  size_t pix = 0;  // encoder input elements per image
  int64_t P = 0;
  float* params = nullptr;
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  int64_t adam_t = 0;

  // encoder
  ConvL nat[3];
  ConvL stem;
  GNL stem_n;
  float* pool = nullptr;
  __nv_bfloat16* pool_bf = nullptr;
  uint8_t* pool_arg = nullptr;
  BlockL blocks[8];
  std::vector<SxL> sx;                  // SE-ResNeXt bottlenecks (net_kind 3, 4)
  float* gw_part = nullptr; size_t gw_part_elems = 0;  // grouped-conv weight-gradient partials
  float* se_dg = nullptr; float* se_dq = nullptr; float* se_dh = nullptr; float* se_dm = nullptr;
  ConvL cmp;
  GNL cmp_n;
  std::vector<ConvL*> convs;
  int max_act = 0;     // max HW*C of any encoder activation (per image)
  size_t max_col = 0;  // max Ho*Wo*Kp (per image)
  size_t max_dz = 0;   // max Ho*Wo*cout (per image)
  int max_gnC = 0;

  int64_t vis_w = -1, vis_b = -1, goal_w = -1, goal_b = -1, emb = -1;
  int64_t actor_w = -1, actor_b = -1, critic_w = -1, critic_b = -1;
  void* Wv = nullptr;
  void* WvT = nullptr;
  float* dWv = nullptr;
  LstmL lstm[4];

  // scratch
  void* col = nullptr; float* dcol = nullptr;
  void* dzop = nullptr;
  float* g0 = nullptr; float* g1 = nullptr; float* g2 = nullptr;
  float* gnp_g = nullptr; float* gnp_b = nullptr;
  GnScratch gnw;                              // GroupNorm partial sums + arrival counters
  float* gn_m1 = nullptr; float* gn_m2 = nullptr;  // [NC, C/2] backward group means
  void* featop = nullptr; float* dfeat = nullptr; void* featT = nullptr;
  void* x1 = nullptr;
  float* gx = nullptr; float* gh = nullptr;
  float* logits = nullptr; float* values = nullptr;
  float* dh_top = nullptr; float* dX[2] = {nullptr, nullptr};
  float* dg32 = nullptr; void* dgop = nullptr;
  float* dh_rec = nullptr; float* dc_carry = nullptr;
  float* dv32 = nullptr; void* dvop = nullptr;
  float* dlogits = nullptr; float* dvalues = nullptr;
  float* scratch = nullptr; size_t scratch_elems = 0;
  GemmWorkspace gws;

  // minibatch buffers
  void* obs_mb = nullptr; float* goal_mb = nullptr; int32_t* preva_mb = nullptr;
  uint8_t* masks_mb = nullptr; int32_t* act_mb = nullptr; float* logp_mb = nullptr;
  float* adv_mb = nullptr; float* ret_mb = nullptr; float* h0_mb = nullptr; float* c0_mb = nullptr;
  int32_t* perm = nullptr; float* adv_norm = nullptr; float* scal = nullptr;
  float* stats_tmp = nullptr; float* norm = nullptr;
  float* act_h = nullptr; float* act_c = nullptr;  // bootstrap state sink

  // last evaluate (inputs read again by backward)
  int ev_T = 0, ev_E = 0;
  bool ev_valid = false;
  const void* ev_obs = nullptr; const float* ev_goal = nullptr; const int32_t* ev_preva = nullptr;
  const uint8_t* ev_masks = nullptr; const float* ev_h0 = nullptr; const float* ev_c0 = nullptr;
  int ev_valid_chunk = -1;
  // last stand-alone encoder / LSTM forward (read again by their backward)
  bool enc_valid = false, lstm_valid = false;
  const void* enc_obs = nullptr; int enc_N = 0;
  int ls_T = 0, ls_E = 0;
  const uint8_t* ls_masks = nullptr; const float* ls_c0 = nullptr;

  // collect graph
  bool collect_started = false;
  int T_last = 0;      // valid steps of the last collection (its last slot is carried over)
  int step_next = -1;  // step-wise collection: the next step index (-1: none begun)
  cudaGraphExec_t graph_exec = nullptr;
  ddppo_rollout graph_ro{};
  // captured PPO update: replayed while its rollout view, statistics buffer and
  // hyper-parameters (other than the update index) are unchanged
  cudaGraphExec_t upd_exec = nullptr;
  ddppo_rollout upd_ro{};
  ddppo_ppo_hparams upd_hp{};
  const float* upd_stats = nullptr;
  bool upd_tuned = false;        // one uncaptured update has run (the autotuner saw its shapes)
  // GEMM timing captured into the graph: the timer records the graph's launches add, and
  // the first record index they use
  bool upd_timed = false;
  int upd_t_n0 = 0, upd_t_dn = 0;
  double upd_t_flops = 0.0, upd_t_flops_all = 0.0, upd_tc_flops = 0.0;
  int64_t upd_t_launches = 0, upd_tc_launches = 0;
  bool upd_no_graph = false;     // kernel census: run the update uncaptured
  bool upd_graph_on = true;      // caller's choice (ddppo_update_graph)
  int64_t* d_steps = nullptr;    // [2] device: update index, Adam steps before this update
  unsigned* lstm_bar = nullptr;  // grid-barrier counter of the whole-segment LSTM kernels
  // LSTM recurrence: 0 step by step; 1 whole segment on CUDA cores (forward and
  // backward); 2 forward on tcgen05 (whole segment, BF16), backward step by step
  int lstm_mode = 0;
  bool gn_fused_on = true;       // GroupNorm statistics + normalisation in one launch
  cudaStream_t cap_stream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  uint8_t* post_done = nullptr;

  KernelTimer timer;
  KernelTimer rc_timer;  // ray cast family
  GemmTcCount tc_count;  // tcgen05 share of the contractions
  std::vector<void*> allocs;
};

}  // namespace ddppo
