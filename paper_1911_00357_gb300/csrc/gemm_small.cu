// Small-M BF16 contraction: C[M, N] (+)= A[M, K] B[N, K]^T for M <= 64, both operands
// K-major (the per-step LSTM recurrences: M = envs, N = 4H or H, K = H or 4H, and the
// per-step input projections of a rollout step).
//
// These shapes are latency-bound (a few MFLOP, weights L2-resident), so the kernel has no
// pipeline set-up: each CTA owns 32 output columns, its 8 warps split K into eight
// slices, and every warp issues warp-level MMAs (m16n8k16, bf16 in, fp32 accumulate)
// on fragments loaded straight from global memory. The eight partial tiles are summed in
// warp order through shared memory (deterministic), then beta, bias and ReLU are applied.
#include "gemm.cuh"

namespace ddppo {

namespace {

constexpr int SM_NB = 32;       // output columns per CTA (four n8 tiles)
constexpr int SM_WARPS = 8;     // K slices per CTA

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p, bool ok) {
  return ok ? *reinterpret_cast<const uint32_t*>(p) : 0u;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// MT: 16-row tiles of M (M <= 16 MT)
template <int MT>
__global__ void __launch_bounds__(SM_WARPS * 32)
    gemm_small_kernel(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                      const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                      int c_bf16, float beta, const float* __restrict__ bias, int relu) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float red[];  // [SM_WARPS][16 MT][SM_NB]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int n0 = blockIdx.x * SM_NB;
  // this warp's K slice, in whole 16-element steps
  const int ksteps = K / 16;
  const int per = (ksteps + SM_WARPS - 1) / SM_WARPS;
  const int kb = warp * per, ke = min(ksteps, kb + per);
  float acc[MT][4][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int ks = kb; ks < ke; ++ks) {
    const int k0 = ks * 16 + 2 * t;
    uint32_t a[MT][4], b[4][2];
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int r0 = i * 16 + g, r1 = r0 + 8;
      a[i][0] = ld_pair(A + (size_t)r0 * lda + k0, r0 < M);
      a[i][1] = ld_pair(A + (size_t)r1 * lda + k0, r1 < M);
      a[i][2] = ld_pair(A + (size_t)r0 * lda + k0 + 8, r0 < M);
      a[i][3] = ld_pair(A + (size_t)r1 * lda + k0 + 8, r1 < M);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + j * 8 + g;
      b[j][0] = ld_pair(B + (size_t)n * ldb + k0, n < N);
      b[j][1] = ld_pair(B + (size_t)n * ldb + k0 + 8, n < N);
    }
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j][0], b[j][1]);
  }
  // partial tiles to shared memory: D fragment rows g / g + 8, columns 2t, 2t + 1
  float* mine = red + (size_t)warp * 16 * MT * SM_NB;
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i * 16 + g, c = j * 8 + 2 * t;
      mine[r * SM_NB + c] = acc[i][j][0];
      mine[r * SM_NB + c + 1] = acc[i][j][1];
      mine[(r + 8) * SM_NB + c] = acc[i][j][2];
      mine[(r + 8) * SM_NB + c + 1] = acc[i][j][3];
    }
  __syncthreads();
  // sum the warps' partials in warp order; epilogue
  for (int e = threadIdx.x; e < 16 * MT * SM_NB; e += blockDim.x) {
    const int r = e / SM_NB, c = e - r * SM_NB, col = n0 + c;
    if (r >= M || col >= N) continue;
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < SM_WARPS; ++w) v += red[(size_t)w * 16 * MT * SM_NB + e];
    const size_t o = (size_t)r * ldc + col;
    if (beta != 0.f) v += beta * C[o];
    if (bias) v += bias[col];
    if (relu) v = fmaxf(v, 0.f);
    if (c_bf16) ((__nv_bfloat16*)C)[o] = __float2bfloat16_rn(v);
    else C[o] = v;
  }
}

template <int MT>
int launch_small(const GemmDesc& d, cudaStream_t s) {
  const size_t smem = (size_t)SM_WARPS * 16 * MT * SM_NB * sizeof(float);
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    DDPPO_CHECK_CUDA(cudaFuncSetAttribute(gemm_small_kernel<MT>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_done[dev] = true;
  }
  const unsigned grid = (unsigned)((d.N + SM_NB - 1) / SM_NB);
  ::ddppo::launch_k(gemm_small_kernel<MT>, grid, SM_WARPS * 32, smem, s,
      d.M, d.N, d.K, (const __nv_bfloat16*)d.A, d.lda, (const __nv_bfloat16*)d.B, d.ldb,
      (float*)d.C, d.ldc, d.c_bf16, d.beta, d.bias, d.relu);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace

bool gemm_small_supported(const GemmDesc& d) {
  return !d.conv && !d.convw && !d.a_t && !d.b_t && d.M >= 1 && d.M <= 64 && d.N >= 1 &&
         d.K >= 16 && d.K % 16 == 0 && d.lda % 2 == 0 && d.ldb % 2 == 0 &&
         ((uintptr_t)d.A & 3) == 0 && ((uintptr_t)d.B & 3) == 0 && d.N <= 65535 * SM_NB;
}

int gemm_small(const GemmDesc& d, cudaStream_t s) {
  if (d.M <= 16) return launch_small<1>(d, s);
  if (d.M <= 32) return launch_small<2>(d, s);
  return launch_small<4>(d, s);
}

}  // namespace ddppo
