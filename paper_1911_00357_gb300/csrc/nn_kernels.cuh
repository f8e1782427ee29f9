// Launchers of the network's non-GEMM kernels (nn_kernels.cu). Activations are NHWC
// fp32; "T" buffers are GEMM operands in the precision's dtype (fp32 or bf16; FP8
// inference adds E4M3 copies of the act-time convolution inputs).
#pragma once

#include "common.cuh"

namespace ddppo {

struct ConvGeom {
  int N, H, W, C;       // input
  int Ho, Wo, Cout;     // output
  int k, s, p;          // square kernel, stride, padding
  int K, Kp;            // k*k*C and its padded row length
};

// im2col: col[m, (ky*k + kx)*C + c] (m = (n, oy, ox)); zero beyond K. x_bf16 gives the
// input's dtype, op_bf16 the output's.
int launch_im2col(const ConvGeom& g, const void* x, bool x_bf16, void* col, bool op_bf16,
                  bool transposed, cudaStream_t s);
// col2im: dx[n, iy, ix, c] (+)= sum of dcol over the (ky, kx) that read it
int launch_col2im(const ConvGeom& g, const float* dcol, float* dx, bool accumulate, cudaStream_t s);
// out[c, r] = in[r, c]
int launch_transpose(const void* in, bool in_bf16, void* out, bool out_bf16, int R, int Cc,
                     int ld_in, cudaStream_t s);
// fp32 -> op dtype copy (or plain copy)
int launch_cast(const float* in, void* out, bool out_bf16, size_t n, cudaStream_t s);

// GroupNorm with groups of 2 channels (C/2 groups), split over several blocks per image
// (gn.cu). Scratch shared by the launches of one stream: partial sums and per-image
// arrival counters (zero at allocation; every launch leaves them zero).
struct GnScratch {
  float* part = nullptr;  // gn_part_elems(max_images, max_C) floats
  size_t part_elems = 0;
  int* cnt = nullptr;     // [max_images], zeroed once
  int* cnt2 = nullptr;    // [max_images], zeroed once (the one-launch form's departures)
  int max_images = 0;
};
size_t gn_part_elems(int max_images, int max_C);
// C even, C / V <= 256 (V = 4 when C % 4 == 0, else 2): C <= 1024
int launch_gn_stats(const float* z, int N, int HW, int C, float eps, float* mean, float* rstd,
                    const GnScratch& w, cudaStream_t s);
// out = act(gn(z) + res) with res = 0, resid (fp32), or gn(zd) (a second normalised input);
// out (fp32) and out_bf (bf16) each optional
struct GNApply {
  const float* z; const float* mean; const float* rstd; const float* gamma; const float* beta;
  const float* resid;  // or null
  const float* zd; const float* mean_d; const float* rstd_d; const float* gamma_d; const float* beta_d;
  float* out; int relu;
  __nv_bfloat16* out_bf;  // optional bf16 copy of out (the next convolution's TMA operand)
  // optional E4M3 copy of out for FP8 inference: e4m3(out / *f8_scale), saturating, and
  // the largest |out| folded into *f8_amax (float bits; a max, so the order is irrelevant)
  uint8_t* out_f8; const float* f8_scale; unsigned* f8_amax;
};
int launch_gn_apply(const GNApply& a, int N, int HW, int C, cudaStream_t s);
// statistics and normalisation in one cooperative launch: a.mean/a.rstd (and a.mean_d /
// a.rstd_d with zd) receive the statistics, out as launch_gn_apply. Sets *launched = false,
// launching nothing, when an image takes one block (small images: the two launches are
// faster), when the grid cannot be resident at once (many images) or w has no departure
// counters; the caller then runs launch_gn_stats + launch_gn_apply. err: the sticky status
// word (timeout flag on a barrier run-out).
int launch_gn_fused(const GNApply& a, int N, int HW, int C, float eps, const GnScratch& w,
                    int32_t* err, cudaStream_t s, bool* launched);
// GroupNorm backward. g = dy, masked by (relu_y > 0) when relu_y is given (the ReLU that
// followed the normalisation); g_out (optional, with relu_y) receives g.
//   dz = rstd (g gamma - m1 - xhat m2), m1 / m2 the group means of gamma g and gamma g xhat;
//   dgamma_part[n, c] = sum g xhat, dbeta_part[n, c] = sum g (per image).
// m1, m2: [N, C/2] scratch. dz32 (fp32) and dzop (op dtype) each optional.
struct GNBack {
  const float* dy; const float* relu_y; float* g_out;
  const float* z; const float* mean; const float* rstd; const float* gamma;
  float* m1; float* m2;
  float* dz32; void* dzop; bool op_bf16;
  float* dgamma_part; float* dbeta_part;
  // optional: the ReLU after the normalisation was not stored; its mask is recomputed
  // from z (relu_y unused, beta = the GroupNorm shift)
  int relu_from_z; const float* beta;
};
int launch_gn_bwd(const GNBack& b, int N, int HW, int C, const GnScratch& w, cudaStream_t s);
// GroupNorm apply + ReLU + 3x3 / stride-2 / pad-1 max pool in one pass: pool (fp32),
// pool_bf (bf16, optional), arg (argmax tap) of [N, Hq, Wq, C]; the full-resolution
// activation is not written. C % 4 == 0.
int launch_gn_relu_maxpool(const GNApply& a, int N, int H, int W, int C, float* pool,
                           __nv_bfloat16* pool_bf, uint8_t* arg, cudaStream_t s);

// dz = dy * (y > 0) written as fp32 (dz32) and/or op dtype (dzop); dy may equal dz32
int launch_relu_bwd(const float* dy, const float* y, size_t n, float* dz32, void* dzop, bool op_bf16,
                    cudaStream_t s);
// dz += dy * (y > 0)   (used where a ReLU output feeds two consumers)
int launch_add(float* dst, const float* src, size_t n, cudaStream_t s);

// ---- SE-ResNeXt pieces (sx.cu) ----
// grouped 3x3 convolution, padding 1, stride s; input [N, H, W, C], output [N, Ho, Wo, C],
// cpg = C / groups channels per group; weights [C][3][3][cpg] in the operand dtype
struct GConv {
  int N, H, W, C, cpg, s, Ho, Wo;
};
int launch_gconv_fwd(const GConv& g, const void* x, const void* w, float* z, bool bf, cudaStream_t s);
int launch_gconv_dgrad(const GConv& g, const void* dz, const void* w, float* dx, bool accumulate,
                       bool bf, cudaStream_t s);
// dw canonical [C][cpg][3][3] fp32 = beta dw + the weight gradient; part: scratch of at
// least gconv_wgrad_chunks() * C * cpg * 9 floats
int gconv_wgrad_chunks(const GConv& g, int num_sms);
int launch_gconv_wgrad(const GConv& g, const void* x, const void* dz, float* part, size_t part_elems,
                       int num_sms, float* dw, float beta, bool bf, cudaStream_t s);
int launch_gconv_w_prep(const float* w, int C, int cpg, void* out, bool bf, cudaStream_t s);
// squeeze-excite of a branch u [N, HW, C] with shortcut sc (null: none) into y (+ y_bf):
//   m = mean_hw u, a = relu(W1 m + b1) [N, Cr], gate = sigmoid(W2 a + b2), y = relu(u gate + sc)
// backward (launch_se_bwd): from gy (the gradient of y): gpre = gy (y > 0) (the shortcut's
// gradient; gpre may be gy), du (the branch's), and the FC parameter gradients
// gW1/gb1/gW2/gb2 (+= when accumulate); dg, dq, dh, dm are [N, C] / [N, Cr] scratch
struct SeArgs {
  int N, HW, C, Cr;
  const float* u; const float* sc;
  const float* W1; const float* b1; const float* W2; const float* b2;
  float* m; float* a; float* gate;
  float* y; __nv_bfloat16* y_bf;
  float* dg; float* dq; float* dh; float* dm;
  float* gW1; float* gb1; float* gW2; float* gb2;
};
int launch_se_fwd(const SeArgs& e, cudaStream_t s);
int launch_se_bwd(const SeArgs& e, const float* gy, float* gpre, float* du, bool accumulate,
                  cudaStream_t s);

int launch_maxpool_fwd(const float* x, int N, int H, int W, int C, float* y, uint8_t* arg,
                       __nv_bfloat16* y_bf, cudaStream_t s);
int launch_maxpool_bwd(const float* dy, const uint8_t* arg, int N, int H, int W, int C, float* dx,
                       cudaStream_t s);

// out[c] (+)= sum_r in[r * ld + c], fixed summation order
int launch_colsum(const float* in, int R, int Cc, int ld, float* out, bool accumulate,
                  cudaStream_t s);
// the column sums of two arrays of the same shape in one launch
int launch_colsum2(const float* in0, const float* in1, int R, int Cc, int ld, float* out0,
                   float* out1, bool accumulate, cudaStream_t s);

// LSTM cell (gate order i, f, g, o). Step t of a [T, E] segment.
struct LstmStep {
  int E, H;
  const float* gx;      // [E, 4H] input projection + both biases
  const float* gh;      // [E, 4H] recurrent projection of the masked previous state
  const float* c_prev;  // [E, H] (unmasked; mask m applied here)
  const uint8_t* m;     // [E] mask of this step
  const uint8_t* m_next;// [E] mask of the next step (null at the last)
  float* gates;         // [E, 4H] post-activation i f g o
  float* c;             // [E, H]
  float* h;             // [E, H] fp32
  void* y_op;           // [E, H] op dtype (layer output for the next layer / heads) or null
  void* hm_next;        // [E, H] op dtype h * m_next (next recurrent GEMM operand) or null
  bool op_bf16;
};
int launch_lstm_fwd(const LstmStep& a, cudaStream_t s);
// hm = h0 * m (op dtype)
int launch_mask_state(const float* h0, const uint8_t* m, int E, int H, void* hm, bool op_bf16,
                      cudaStream_t s);

struct LstmBack {
  int E, H;
  const float* gates; const float* c; const float* c_prev;  // forward values of step t
  const uint8_t* m;         // mask of step t
  const uint8_t* m_next;    // mask of step t+1 (applies to dh_rec / dc_carry) or null
  const float* dh_above;    // [E, H]
  const float* dh_rec;      // [E, H] dG_{t+1} W_hh (unmasked) or null at the last step
  float* dc_carry;          // [E, H] in: dc_{t+1} f_{t+1} (unmasked); out: dc_t f_t
  float* dg32;              // [E, 4H] fp32 dgates
  void* dg_op;              // [E, 4H] op dtype dgates
  bool op_bf16;
};
int launch_lstm_bwd(const LstmBack& a, cudaStream_t s);

// The whole T-step recurrence of one LSTM layer (forward) or its back-propagation through
// time (backward) in one cooperative launch (lstm_seq.cu). Forward: gx [T, E, 4H] (input
// projection + biases), masks [T, E], h0 / c0 [E, H] -> gates [T, E, 4H], c, h [T, E, H],
// y_op [T, E, H] (op dtype, may be null), hm [T, E, H] (op dtype: the masked state entering
// each step, slot 0 included). Backward: gates, c, c0, masks, dh_above [T, E, H] ->
// dg32 / dg_op [T, E, 4H]. Whh [4H, H] op dtype. bar: one device counter (zeroed by the
// launcher); err: the sticky status word (timeout flag on a run-out barrier wait).
struct LstmSeq {
  int T, E, H;
  const float* gx; const uint8_t* m; const float* h0; const float* c0; const void* Whh;
  float* gates; float* c; float* h; void* y_op; void* hm;
  const float* dh_above; float* dg32; void* dg_op;
  unsigned* bar; int32_t* err; int op_bf16;
};
bool lstm_seq_supported(int H, int E, int num_sms);

// the forward recurrence on tcgen05 (lstm_tc.cu): BF16 operands, [T, E, *] layouts as the
// step-by-step path; hm[0] (the masked initial state) must be written beforehand
struct LstmTc {
  int T, E, H;
  const float* gx; const uint8_t* m; const float* c0; const __nv_bfloat16* Whh;
  float* gates; float* c; float* h; __nv_bfloat16* y_op; __nv_bfloat16* hm;
  unsigned* bar; int32_t* err;
};
bool lstm_tc_supported(int H, int E, int num_sms);

// single-channel convolution on tcgen05 (conv_c1_tc.cu): y [N, Ho, Wo, Cout] fp32
// (= beta y + conv) of x [N, H, W] bf16 with w [Cout, ldw] bf16 (taps (ky, kx) in its
// first k^2 columns); k^2 <= 64, Cout 16 / 32 / 64
struct ConvC1 {
  int N, H, W, k, s, p, Ho, Wo, Cout, ldw;
  const __nv_bfloat16* x; const __nv_bfloat16* w; float* y; float beta; int32_t* err;
};
bool conv_c1_tc_supported(int k, int Cout);
int launch_conv_c1_tc(const ConvC1& a, int num_sms, cudaStream_t s);
int launch_lstm_tc_fwd(const LstmTc& a, int num_sms, cudaStream_t s);
int launch_lstm_seq_fwd(const LstmSeq& a, int num_sms, cudaStream_t s);
int launch_lstm_seq_bwd(const LstmSeq& a, int num_sms, cudaStream_t s);

// heads: logits = h Wa^T + ba, value = h wv + bv (canonical fp32 weights)
struct Heads {
  int N, H;
  const float* h;        // [N, H]
  const float* Wa; const float* ba; const float* Wv; const float* bv;
  float* logits;         // [N, 4] or null
  float* value;          // [N]
  // sampling (act): uniforms -> action, logp
  const float* u; int32_t* action; float* logp;
};
int launch_heads_fwd(const Heads& a, cudaStream_t s);
// dh[n] = dlogits[n] Wa + dvalue[n] wv ; weight grads via partials
int launch_heads_bwd(int N, int H, const float* h, const float* Wa, const float* Wv,
                     const float* dlogits, const float* dvalue, float* dh, float* gWa, float* gba,
                     float* gWv, float* gbv, float* scratch, size_t scratch_elems, cudaStream_t s);

// goal FC (3 -> 32) and action embedding (5 x 32) into columns [col0, col0+64) of x (op dtype)
int launch_embed_fwd(int N, const float* goal, const int32_t* prev_a, const float* Wg,
                     const float* bg, const float* Emb, void* x, int ldx, int col0, bool op_bf16,
                     cudaStream_t s);
int launch_embed_bwd(int N, const float* goal, const int32_t* prev_a, const float* dx, int lddx,
                     int col0, float* gWg, float* gbg, float* gEmb, float* scratch,
                     size_t scratch_elems, cudaStream_t s);
// dv = dx[:, :H] * (v > 0) from the concatenated LSTM input gradient; v read from x (op dtype)
int launch_vis_relu_bwd(int N, int H, const float* dx, int lddx, const void* x, int ldx,
                        bool op_bf16, float* dv32, void* dvop, cudaStream_t s);

// rows gather: out[t, j, :] = in[t, idx[j], :], rows of `bytes` bytes; idx null = identity
int launch_gather_rows(const void* in, void* out, const int32_t* idx, int T, int Ein, int Eout,
                       size_t bytes, cudaStream_t s);

// weight preparation and gradient scatter between canonical and GEMM layouts
int launch_conv_w_prep(const float* w, int cout, int cin, int k, int Kp, void* wg, void* wgT,
                       bool op_bf16, cudaStream_t s);
// wr[ci, (ky*k + kx)*cout + co] = w[co, ci, k-1-ky, k-1-kx]: the kernel of the input
// gradient of a stride-1 'same' convolution, itself a convolution of the output gradient
int launch_conv_w_flip(const float* w, int cout, int cin, int k, void* wr, bool op_bf16,
                       cudaStream_t s);
int launch_conv_w_grad(const float* dwg, int cout, int cin, int k, int Kp, float* dw,
                       cudaStream_t s);
// vis FC: canonical column j = c*HW + hw  <->  GEMM column hw*C + c
int launch_vis_w_prep(const float* w, int H, int C, int HW, void* wg, void* wgT, bool op_bf16,
                      cudaStream_t s);
int launch_vis_w_grad(const float* dwg, int H, int C, int HW, float* dw, cudaStream_t s);
int launch_add_vec(const float* a, const float* b, float* out, int n, cudaStream_t s);

// deterministic parameter init from the counter hash
int launch_init_uniform(float* p, size_t n, float lo, float hi, uint64_t seed, uint64_t stream,
                        cudaStream_t s);
int launch_fill(float* p, size_t n, float v, cudaStream_t s);

// ---------------------------------------------------------------- E4M3 (fp8.cu)
constexpr float kE4M3Max = 448.f;  // largest finite E4M3 value

// x -> E4M3 code: round to nearest even, saturating to +-448
__device__ __forceinline__ uint8_t e4m3_sat(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// *amax = max(*amax, max |x|) over n values (fp32, or bf16 when x_bf16); *amax holds float
// bits and must start at 0 (or a previous maximum)
int launch_amax(const void* x, bool x_bf16, size_t n, unsigned* amax, cudaStream_t s);
// per-tensor quantisation: scale = amax / 448 (1 when amax = 0), q = e4m3(x / scale)
int launch_quant_e4m3(const void* x, bool x_bf16, size_t n, const unsigned* amax, float* scale,
                      uint8_t* q, cudaStream_t s);
// delayed activation scales: for every slot with amax > 0, scale = 2 amax / 448 (one binade
// of headroom for the next pass); amax is reset to 0
int launch_f8_scale_update(float* scale, unsigned* amax, int n, cudaStream_t s);

}  // namespace ddppo
