// SIMT GEMM (the plain FP32 form, and the fallback shape path of the BF16 form) with
// deterministic split-K, plus the dispatcher that routes bf16 operands to tcgen05.
#include "gemm.cuh"
#include "nn_kernels.cuh"

namespace ddppo {

template <typename T>
__device__ __forceinline__ float ld_op(const T* p);
template <>
__device__ __forceinline__ float ld_op<float>(const float* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld_op<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

constexpr int SB_M = 64, SB_N = 64, SB_K = 16;

// 256 threads; thread (tx, ty) owns rows ty + 16 i and columns tx + 16 j, i, j < 4.
template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int M, int N, int K, const T* __restrict__ A,
                                                        int lda, const T* __restrict__ B, int ldb,
                                                        float* __restrict__ C, int ldc, int c_bf16,
                                                        float beta, const float* __restrict__ bias,
                                                        int relu, int kchunk,
                                                        float* __restrict__ partial, int a_t,
                                                        int b_t) {
  DDPPO_PDL_ENTRY();
  __shared__ float As[SB_K][SB_M + 4];
  __shared__ float Bs[SB_K][SB_N + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * SB_M, n0 = blockIdx.y * SB_N;  // M tiles on x: M can exceed 65535*64
  const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
  float acc[4][4] = {};
  const int lr = tid >> 2, lk = (tid & 3) * 4;  // loader: row lr, k lk..lk+3
  for (int k0 = kbeg; k0 < kend; k0 += SB_K) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + lk + q;
      const int m = m0 + lr, n = n0 + lr;
      As[lk + q][lr] = (m < M && k < kend)
                           ? ld_op(A + (a_t ? (size_t)k * lda + m : (size_t)m * lda + k)) : 0.f;
      Bs[lk + q][lr] = (n < N && k < kend)
                           ? ld_op(B + (b_t ? (size_t)k * ldb + n : (size_t)n * ldb + k)) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < SB_K; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      if (partial) {
        partial[((size_t)blockIdx.z * M + m) * N + n] = acc[i][j];
        continue;
      }
      float v = acc[i][j];
      if (beta != 0.f) v += beta * C[(size_t)m * ldc + n];
      if (bias) v += bias[n];
      if (relu) v = fmaxf(v, 0.f);
      if (c_bf16) ((__nv_bfloat16*)C)[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
      else C[(size_t)m * ldc + n] = v;
    }
  }
}

// C = beta*C + sum_z partial[z] (+ bias) (ReLU), summed in split order.
__global__ void splitk_reduce_kernel(int M, int N, int splits, const float* __restrict__ partial,
                                     float* __restrict__ C, int ldc, int c_bf16, float beta,
                                     const float* __restrict__ bias, int relu) {
  DDPPO_PDL_ENTRY();
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)M * N) return;
  const int m = (int)(idx / N), n = (int)(idx % N);
  float v = 0.f;
  for (int z = 0; z < splits; ++z) v += partial[(size_t)z * M * N + idx];
  if (beta != 0.f) v += beta * C[(size_t)m * ldc + n];
  if (bias) v += bias[n];
  if (relu) v = fmaxf(v, 0.f);
  if (c_bf16) ((__nv_bfloat16*)C)[(size_t)m * ldc + n] = __float2bfloat16_rn(v);
  else C[(size_t)m * ldc + n] = v;
}

static int gemm_simt(const GemmDesc& d, bool op_bf16, const GemmWorkspace& ws, cudaStream_t s) {
  const int gm = (d.M + SB_M - 1) / SB_M, gn = (d.N + SB_N - 1) / SB_N;
  int splits = 1;
  const int tiles = gm * gn;
  const int target = 2 * ws.num_sms;
  if (tiles < target && d.K >= 4 * SB_K * 8) {
    splits = (target + tiles - 1) / tiles;
    splits = min(splits, d.K / (SB_K * 8));
    const size_t per = (size_t)d.M * d.N;
    if (per > 0) splits = (int)min((size_t)splits, ws.partial_elems / per);
    if (splits < 2) splits = 1;
  }
  int kchunk = (d.K + splits - 1) / splits;
  kchunk = (kchunk + SB_K - 1) / SB_K * SB_K;
  splits = (d.K + kchunk - 1) / kchunk;
  if (splits < 1) splits = 1;
  float* partial = splits > 1 ? ws.partial : nullptr;
  dim3 grid(gm, gn, splits);
  if (op_bf16)
    ::ddppo::launch_k(gemm_simt_kernel<__nv_bfloat16>, grid, 256, 0, s,
        d.M, d.N, d.K, (const __nv_bfloat16*)d.A, d.lda, (const __nv_bfloat16*)d.B, d.ldb,
        (float*)d.C, d.ldc, d.c_bf16, d.beta, d.bias, d.relu, kchunk, partial, d.a_t, d.b_t);
  else
    ::ddppo::launch_k(gemm_simt_kernel<float>, grid, 256, 0, s, d.M, d.N, d.K, (const float*)d.A, d.lda,
                                                 (const float*)d.B, d.ldb, (float*)d.C, d.ldc,
                                                 d.c_bf16, d.beta, d.bias, d.relu, kchunk, partial,
                                                 d.a_t, d.b_t);
  DDPPO_CHECK_LAUNCH();
  if (partial)
    DDPPO_TRY(launch_splitk_reduce(d.M, d.N, splits, partial, (float*)d.C, d.ldc, d.c_bf16, d.beta,
                                   d.bias, d.relu, s));
  return DDPPO_OK;
}

int launch_splitk_reduce(int M, int N, int splits, const float* partial, float* C, int ldc,
                         int c_bf16, float beta, const float* bias, int relu, cudaStream_t s) {
  const size_t n = (size_t)M * N;
  ::ddppo::launch_k(splitk_reduce_kernel, (unsigned)((n + 255) / 256), 256, 0, s, M, N, splits, partial, C, ldc,
                                                                   c_bf16, beta, bias, relu);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// E4M3 operands on the tensor cores. The kernel's layouts are byte layouts (a 128-byte
// operand row is 64 bf16 or 128 E4M3 values, and one MMA consumes 32 bytes of K either
// way), so the contraction runs on the 16-bit view of its operands: K, the leading
// dimensions and a convolution's channels count E4M3 pairs, and only the MMA kind and the
// epilogue's scale differ from the bf16 form.
static int gemm_fp8(const GemmDesc& d, const GemmWorkspace& ws, cudaStream_t s) {
  if (d.convw || d.a_t || d.b_t || (d.K % 2) || (d.lda % 2) || (d.ldb % 2) ||
      (d.conv && (d.conv->C % 2))) {
    set_error("gemm: E4M3 operands must be K-major with even K, leading dimensions and channels");
    return DDPPO_E_CONFIG;
  }
  GemmDesc p = d;
  p.K = d.K / 2;
  p.lda = d.lda / 2;
  p.ldb = d.ldb / 2;
  ConvShape cp;
  if (d.conv) {
    cp = *d.conv;
    cp.C = d.conv->C / 2;
    p.conv = &cp;
    if (!gemm_conv_supported(cp, p.A)) {
      set_error("gemm: E4M3 convolution needs 64 | C (or C = 64 on the halo path)");
      return DDPPO_E_CONFIG;
    }
  } else if (!gemm_tc_supported(p)) {
    set_error("gemm: E4M3 operands need 16-byte aligned rows and K >= 32");
    return DDPPO_E_CONFIG;
  }
  return gemm_tc(p, ws, s);
}

// the single-channel convolution kernel covers this contraction: an implicit convolution
// of a 1-channel input into fp32 rows of Cout (no bias, ReLU or bf16 output)
static bool conv_c1_ok(const GemmDesc& d) {
  return d.conv && d.conv->C == 1 && conv_c1_tc_supported(d.conv->k, d.conv->Cout) &&
         d.N == d.conv->Cout && d.ldc == d.N && !d.c_bf16 && !d.bias && !d.relu && !d.fp8 &&
         d.ldb >= d.conv->k * d.conv->k;
}

int gemm(const GemmDesc& d, bool op_bf16, const GemmWorkspace& ws, cudaStream_t s,
         KernelTimer* timer) {
  if (d.M <= 0 || d.N <= 0) return DDPPO_OK;
  if (d.K <= 0) {
    set_error("gemm: K must be positive");
    return DDPPO_E_CONFIG;
  }
  if (d.fp8 && (!op_bf16 || d.c_bf16)) {
    set_error("gemm: E4M3 operands need the tensor-core path and an fp32 output");
    return DDPPO_E_CONFIG;
  }
  if (d.c_bf16 && d.beta != 0.f) {
    set_error("gemm: bf16 output cannot accumulate");
    return DDPPO_E_CONFIG;
  }
  if (d.conv && !d.fp8 && !(op_bf16 && (gemm_conv_supported(*d.conv, d.A) || conv_c1_ok(d)))) {
    set_error("gemm: implicit convolution not supported for this shape");
    return DDPPO_E_CONFIG;
  }
  if (d.convw && !(op_bf16 && !d.conv && d.a_t && d.lda == d.M && d.lda % 8 == 0 && !d.c_bf16 && !d.bias && !d.relu &&
                   d.N == d.convw->k * d.convw->k * d.convw->C &&
                   d.K == d.convw->N * d.convw->Ho * d.convw->Wo &&
                   (conv_wgrad_halo_ok(*d.convw, d.B, d.A) ||
                    gemm_convw_supported(*d.convw, d.B, d.A)))) {
    set_error("gemm: implicit weight gradient not supported for this shape");
    return DDPPO_E_CONFIG;
  }
  const bool rec = timer && timer->on && timer->n + 2 <= 2 * 4096;
  if (timer && timer->on) timer->flops_all += 2.0 * d.M * d.N * d.K;
  // inside a stream capture the records are external: they become event nodes of the graph
  unsigned rec_flags = cudaEventRecordDefault;
  if (rec) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      rec_flags = cudaEventRecordExternal;
    cudaEventRecordWithFlags(timer->ev[timer->n], s, rec_flags);
  }
  int rc;
  if (d.fp8) {
    rc = gemm_fp8(d, ws, s);
    if (ws.tc && ws.tc->on) {
      ws.tc->launches += 1;
      ws.tc->flops += 2.0 * d.M * d.N * d.K;
    }
  } else if (op_bf16 && conv_c1_ok(d)) {
    // a single-channel convolution (the stem): patches gathered in shared memory
    const ConvShape& c = *d.conv;
    ConvC1 a{};
    a.N = c.N; a.H = c.H; a.W = c.W; a.k = c.k; a.s = c.s; a.p = c.p; a.Ho = c.Ho; a.Wo = c.Wo;
    a.Cout = c.Cout; a.ldw = d.ldb;
    a.x = (const __nv_bfloat16*)d.A; a.w = (const __nv_bfloat16*)d.B; a.y = (float*)d.C;
    a.beta = d.beta; a.err = ws.err;
    rc = launch_conv_c1_tc(a, ws.num_sms, s);
    if (ws.tc && ws.tc->on) {
      ws.tc->launches += 1;
      ws.tc->flops += 2.0 * d.M * d.N * d.K;
    }
  } else if (op_bf16 && gemm_small_supported(d)) {
    rc = gemm_small(d, s);  // latency-bound small-M shapes: no tensor-memory pipeline
  } else if (op_bf16 && d.convw && conv_wgrad_halo_ok(*d.convw, d.B, d.A)) {
    rc = conv_wgrad_halo(*d.convw, d.B, d.A, (float*)d.C, d.ldc, d.beta, ws, s);
  } else if (op_bf16 && (d.conv || d.convw || gemm_tc_supported(d))) {
    rc = gemm_tc(d, ws, s);
    if (ws.tc && ws.tc->on) {
      ws.tc->launches += 1;
      ws.tc->flops += 2.0 * d.M * d.N * d.K;
    }
  } else {
    rc = gemm_simt(d, op_bf16, ws, s);
  }
  if (rec) {
    cudaEventRecordWithFlags(timer->ev[timer->n + 1], s, rec_flags);
    const double es = d.fp8 ? 1.0 : op_bf16 ? 2.0 : 4.0, cs = d.c_bf16 ? 2.0 : 4.0;
    timer->work[timer->n / 2] = 2.0 * d.M * d.N * d.K;
    // operands read once, result written once (and read when accumulating); an implicit
    // convolution reads its input tensor, not the M x K patch matrix
    const ConvShape* cv = d.conv ? d.conv : d.convw;
    const double in_elems = cv ? (double)cv->N * cv->H * cv->W * cv->C : 0.0;
    const double a_elems = d.conv ? in_elems : (double)d.M * d.K;
    const double b_elems = d.convw ? in_elems : (double)d.N * d.K;
    timer->bytes[timer->n / 2] = (a_elems + b_elems) * es +
                                 (double)d.M * d.N * cs * (d.beta != 0.f ? 2.0 : 1.0);
    timer->n += 2;
    timer->flops += 2.0 * d.M * d.N * d.K;
    timer->launches += 1;
  }
  return rc;
}

}  // namespace ddppo
