// E4M3 quantisation for FP8 inference: per-tensor absolute maxima, per-tensor scales and
// the saturating conversion. Scales follow the usual per-tensor convention: a tensor x is
// carried as q = e4m3(x / s) with s = amax(x) / 448, so that q * s reproduces x to E4M3
// precision (3 mantissa bits) over the whole range of the tensor.
#include <algorithm>

#include "nn_kernels.cuh"

namespace ddppo {

namespace {

constexpr int kQThreads = 256;

template <bool BF>
__device__ __forceinline__ float ld_any(const void* x, size_t i) {
  if (BF) return __bfloat162float(((const __nv_bfloat16*)x)[i]);
  return ((const float*)x)[i];
}

template <bool BF>
__global__ void __launch_bounds__(kQThreads) amax_kernel(const void* __restrict__ x, size_t n,
                                                         unsigned* __restrict__ amax) {
  DDPPO_PDL_ENTRY();
  __shared__ float wmax[kQThreads / 32];
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(ld_any<BF>(x, i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < kQThreads / 32; ++w) b = fmaxf(b, wmax[w]);
    atomicMax(amax, __float_as_uint(b));
  }
}

template <bool BF>
__global__ void __launch_bounds__(kQThreads) quant_kernel(const void* __restrict__ x, size_t n,
                                                          const unsigned* __restrict__ amax,
                                                          float* __restrict__ scale,
                                                          uint8_t* __restrict__ q) {
  DDPPO_PDL_ENTRY();
  const float a = __uint_as_float(*amax);
  const float sc = a > 0.f ? a / kE4M3Max : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = sc;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    q[i] = e4m3_sat(ld_any<BF>(x, i) / sc);
}

__global__ void f8_scale_update_kernel(float* __restrict__ scale, unsigned* __restrict__ amax, int n) {
  DDPPO_PDL_ENTRY();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float a = __uint_as_float(amax[i]);
  if (a > 0.f) scale[i] = 2.f * a / kE4M3Max;
  amax[i] = 0u;
}

unsigned qgrid(size_t n) {
  const size_t b = (n + kQThreads - 1) / kQThreads;
  return (unsigned)std::min<size_t>(std::max<size_t>(b, 1), 8 * 1024);
}

}  // namespace

int launch_amax(const void* x, bool x_bf16, size_t n, unsigned* amax, cudaStream_t s) {
  if (!n) return DDPPO_OK;
  if (x_bf16) ::ddppo::launch_k(amax_kernel<true>, qgrid(n), kQThreads, 0, s, x, n, amax);
  else ::ddppo::launch_k(amax_kernel<false>, qgrid(n), kQThreads, 0, s, x, n, amax);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_quant_e4m3(const void* x, bool x_bf16, size_t n, const unsigned* amax, float* scale,
                      uint8_t* q, cudaStream_t s) {
  if (x_bf16) ::ddppo::launch_k(quant_kernel<true>, qgrid(n), kQThreads, 0, s, x, n, amax, scale, q);
  else ::ddppo::launch_k(quant_kernel<false>, qgrid(n), kQThreads, 0, s, x, n, amax, scale, q);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_f8_scale_update(float* scale, unsigned* amax, int n, cudaStream_t s) {
  if (n <= 0) return DDPPO_OK;
  ::ddppo::launch_k(f8_scale_update_kernel, (n + 127) / 128, 128, 0, s, scale, amax, n);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
