// GEMM interface used by every contraction of the agent network.
//   C[M, N] = beta * C + sum_k A(m, k) B(n, k) (+ bias[N]) (ReLU)
// A(m, k) = A[m * lda + k] (K-contiguous), or A[k * lda + m] when a_t ("MN-major": the
// weight gradients read activations and output gradients as they are stored, [rows][C]).
// B likewise with b_t. Operands are of the operand dtype (fp32 or bf16; E4M3 with the
// fp8 flag, K-major only); C is fp32, or bf16 when c_bf16 (then beta must be 0).
// Accumulation is fp32.
#pragma once

#include "common.cuh"

namespace ddppo {

// A convolution whose GEMM A operand is gathered from its NHWC bf16 input by the
// tensor-core kernel itself (implicit im2col): row m = output pixel, column
// (ky*k + kx)*C + c. K = k*k*C; B is the [Cout, K] weight matrix.
struct ConvShape {
  int N = 0, H = 0, W = 0, C = 0, Ho = 0, Wo = 0, k = 0, s = 1, p = 0;
  int Cout = 0;  // output channels (0: unknown; the halo path then stays off)
};

struct GemmDesc {
  int M = 0, N = 0, K = 0;
  const ConvShape* conv = nullptr;  // non-null: A is the convolution input (NHWC bf16)
  // non-null: the weight gradient of a convolution, dW[co, (ky, kx, c)] (+)= sum over output
  // pixels m of dz[m, co] x[m shifted by (ky, kx), c]: M = cout, N = k*k*C, K = pixels,
  // A = dz stored [K][M] (a_t = 1, lda = M), B = the convolution input (NHWC bf16)
  const ConvShape* convw = nullptr;
  const void* A = nullptr;
  int lda = 0;
  const void* B = nullptr;
  int ldb = 0;
  void* C = nullptr;
  int ldc = 0;
  int c_bf16 = 0;
  float beta = 0.f;
  const float* bias = nullptr;
  int relu = 0;
  int a_t = 0;  // A stored [K][M]
  int b_t = 0;  // B stored [K][N]
  // fp8: A and B hold E4M3 values, both K-major (K, lda, ldb and a convolution's C count
  // E4M3 elements); the product is multiplied by *scale_a * *scale_b (device scalars, null
  // reads as 1) before beta, bias and ReLU
  int fp8 = 0;
  const float* scale_a = nullptr;
  const float* scale_b = nullptr;
};

struct GemmTcCount {
  bool on = false;
  int64_t launches = 0;
  double flops = 0.0;
};

// Tile-shape autotuner of the tcgen05 GEMM: the first time a contraction shape is seen
// (outside stream capture), every candidate configuration runs into a scratch output and
// the fastest is kept for the life of the worker.
struct TcTuner;
TcTuner* tc_tuner_create(size_t scratch_bytes);
void tc_tuner_destroy(TcTuner* t);
void tc_tuner_enable(TcTuner* t, bool on);
int64_t tc_tuner_shapes(const TcTuner* t);
// serialise the table into buf (returns the bytes needed; writes only when cap suffices)
size_t tc_tuner_export(const TcTuner* t, void* buf, size_t cap);
// merge a serialised table (entries replace equal keys)
int tc_tuner_import(TcTuner* t, const void* buf, size_t size);

struct GemmWorkspace {
  float* partial = nullptr;  // split-K partial sums
  size_t partial_elems = 0;
  int num_sms = 152;
  GemmTcCount* tc = nullptr;  // counts contractions routed to tcgen05 while enabled
  int32_t* err = nullptr;      // sticky device status word (timeout flag)
  TcTuner* tuner = nullptr;    // tile-shape autotuner (null: fixed heuristic)
};

// timing of GEMM launches (family 0 of ddppo_timing_read)
struct KernelTimer {
  bool on = false;
  int n = 0;
  cudaEvent_t ev[2 * 4096];
  double work[4096];       // per timed launch: FLOPs (GEMM) or output bytes (ray cast)
  double bytes[4096];      // per timed launch: algorithmic HBM bytes
  double flops = 0.0;      // work of the launches that carry events
  int64_t launches = 0;
  double flops_all = 0.0;  // work of every launch while enabled
};

int gemm(const GemmDesc& d, bool op_bf16, const GemmWorkspace& ws, cudaStream_t s,
         KernelTimer* timer = nullptr);

// C = beta*C + sum of `splits` partial [M, N] slices (+ bias) (ReLU), fixed order
int launch_splitk_reduce(int M, int N, int splits, const float* partial, float* C, int ldc,
                         int c_bf16, float beta, const float* bias, int relu, cudaStream_t s);

// tcgen05 path (gemm_tc.cu); returns DDPPO_E_CONFIG when the shape is not supported
int gemm_tc(const GemmDesc& d, const GemmWorkspace& ws, cudaStream_t s);
// paths and staging geometry of a convolution (18 words; see gemm_tc.cu); host only
void conv_plan(const ConvShape& c, int32_t* plan);
bool gemm_tc_supported(const GemmDesc& d);
// whether the implicit-im2col path covers this convolution (C % 32 == 0, output rows that
// tile 128-pixel blocks, 16-byte aligned input)
bool gemm_conv_supported(const ConvShape& c, const void* input);
// weight gradient of a 3x3 / stride-1 / pad-1 convolution, 32 -> 32 channels, through
// staged halo boxes (gemm_tc.cu): dw[co, (ky*3+kx)*32 + c] (+)= ...; x, dz NHWC bf16
bool conv_wgrad_halo_ok(const ConvShape& c, const void* x, const void* dz);
int conv_wgrad_halo(const ConvShape& c, const void* x, const void* dz, float* dw, int ldw, float beta,
                    const GemmWorkspace& ws, cudaStream_t s);
// small-M BF16 contraction (gemm_small.cu): M <= 64, both operands K-major, K % 16 == 0
bool gemm_small_supported(const GemmDesc& d);
int gemm_small(const GemmDesc& d, cudaStream_t s);
// the implicit weight-gradient gather (64-pixel K blocks) handles this shape
bool gemm_convw_supported(const ConvShape& c, const void* input, const void* dz);

}  // namespace ddppo
