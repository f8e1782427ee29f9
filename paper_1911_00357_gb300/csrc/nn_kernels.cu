// Non-GEMM kernels of the agent network (App. "Agent Design"): convolution layout
// transforms, GroupNorm (Wu & He 2018) with C/2 groups, max pool, the LSTM cell and its
// backward, actor/critic heads with inverse-CDF sampling, goal/action embeddings, and the
// canonical <-> GEMM weight layouts. All reductions run in a fixed order.
#include <algorithm>

#include "nn_kernels.cuh"

namespace ddppo {

static inline unsigned nblk(size_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <typename T> __device__ __forceinline__ T from_f(float v);
template <> __device__ __forceinline__ float from_f<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}
__device__ __forceinline__ void st_op(void* p, size_t i, float v, bool bf) {
  if (bf) ((__nv_bfloat16*)p)[i] = __float2bfloat16_rn(v);
  else ((float*)p)[i] = v;
}
__device__ __forceinline__ float ld_any(const void* p, size_t i, bool bf) {
  return bf ? __bfloat162float(((const __nv_bfloat16*)p)[i]) : ((const float*)p)[i];
}

// ---------------------------------------------------------------- im2col / col2im
template <typename Ti, typename To>
__global__ void im2col_kernel(ConvGeom g, const Ti* __restrict__ x, To* __restrict__ col) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)g.N * g.Ho * g.Wo * g.Kp;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kk = (int)(idx % g.Kp);
    const size_t m = idx / g.Kp;
    float v = 0.f;
    if (kk < g.K) {
      const int c = kk % g.C, kx = (kk / g.C) % g.k, ky = kk / (g.C * g.k);
      const int ox = (int)(m % g.Wo), oy = (int)((m / g.Wo) % g.Ho), n = (int)(m / ((size_t)g.Wo * g.Ho));
      const int iy = oy * g.s - g.p + ky, ix = ox * g.s - g.p + kx;
      if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W)
        v = to_f(x[(((size_t)n * g.H + iy) * g.W + ix) * g.C + c]);
    }
    col[idx] = from_f<To>(v);
  }
}

// colT[kk, m]
template <typename Ti, typename To>
__global__ void im2colT_kernel(ConvGeom g, const Ti* __restrict__ x, To* __restrict__ colT) {
  DDPPO_PDL_ENTRY();
  const size_t M = (size_t)g.N * g.Ho * g.Wo;
  const size_t total = M * g.Kp;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t m = idx % M;
    const int kk = (int)(idx / M);
    float v = 0.f;
    if (kk < g.K) {
      const int c = kk % g.C, kx = (kk / g.C) % g.k, ky = kk / (g.C * g.k);
      const int ox = (int)(m % g.Wo), oy = (int)((m / g.Wo) % g.Ho), n = (int)(m / ((size_t)g.Wo * g.Ho));
      const int iy = oy * g.s - g.p + ky, ix = ox * g.s - g.p + kx;
      if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W)
        v = to_f(x[(((size_t)n * g.H + iy) * g.W + ix) * g.C + c]);
    }
    colT[idx] = from_f<To>(v);
  }
}

static unsigned grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  if (b > 152u * 64u) b = 152u * 64u;
  if (b < 1) b = 1;
  return (unsigned)b;
}

// Vectorised forward-layout im2col for C % 8 == 0: one thread per (row m, tap, 8-channel
// group); 8 channels are read (two float4 or one 16-byte bf16 load) and written with one
// 16-byte (bf16) or two (fp32) stores, so index decoding happens once per 8 elements and
// consecutive threads touch consecutive bytes.
template <typename Ti, typename To>
__global__ void im2col_vec_kernel(ConvGeom g, const Ti* __restrict__ x, To* __restrict__ col) {
  DDPPO_PDL_ENTRY();
  const int C8 = g.C >> 3, taps = g.k * g.k;
  const size_t total = (size_t)g.N * g.Ho * g.Wo * taps * C8;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(idx % C8);
    const size_t q = idx / C8;
    const int tap = (int)(q % taps);
    const size_t m = q / taps;
    const int ky = tap / g.k, kx = tap - ky * g.k;
    const int ox = (int)(m % g.Wo), oy = (int)((m / g.Wo) % g.Ho), n = (int)(m / ((size_t)g.Wo * g.Ho));
    const int iy = oy * g.s - g.p + ky, ix = ox * g.s - g.p + kx;
    float v[8];
    if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W) {
      const Ti* src = x + (((size_t)n * g.H + iy) * g.W + ix) * g.C + c8 * 8;
      if constexpr (sizeof(Ti) == 4) {
        const float4 a = *(const float4*)src, b = *(const float4*)(src + 4);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
      } else {
        const uint4 u = *(const uint4*)src;
        const __nv_bfloat16* h = (const __nv_bfloat16*)&u;
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __bfloat162float(h[i]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = 0.f;
    }
    To* dst = col + m * g.Kp + (size_t)tap * g.C + c8 * 8;
    if constexpr (sizeof(To) == 2) {
      uint4 u;
      __nv_bfloat16* h = (__nv_bfloat16*)&u;
#pragma unroll
      for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
      *(uint4*)dst = u;
    } else {
      *(float4*)dst = make_float4(v[0], v[1], v[2], v[3]);
      *(float4*)(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
}

// Single-channel input (the first convolution on the depth image): one thread per output
// row, assembling 8 taps at a time into one 16-byte (bf16) or two (fp32) stores; adjacent
// threads write adjacent rows, so a warp writes one contiguous stretch of the col matrix.
template <typename Ti, typename To>
__global__ void im2col_c1_kernel(ConvGeom g, const Ti* __restrict__ x, To* __restrict__ col) {
  DDPPO_PDL_ENTRY();
  const int nck = g.Kp / 8;                     // 8-tap chunks per row
  const int per_img = g.Ho * g.Wo * nck;        // chunks of one image
  const int n = blockIdx.y;
  const Ti* img = x + (size_t)n * g.H * g.W;
  To* dst_img = col + (size_t)n * g.Ho * g.Wo * g.Kp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per_img; i += gridDim.x * blockDim.x) {
    const int ck = i % nck, m = i / nck;
    const int ox = m % g.Wo, oy = m / g.Wo;
    const int k0 = ck * 8;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = k0 + q;
      float t = 0.f;
      if (kk < g.K) {
        const int ky = kk / g.k, kx = kk - ky * g.k;
        const int iy = oy * g.s - g.p + ky, ix = ox * g.s - g.p + kx;
        if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W) t = to_f(img[iy * g.W + ix]);
      }
      v[q] = t;
    }
    To* dst = dst_img + (size_t)m * g.Kp + k0;
    if constexpr (sizeof(To) == 2) {
      uint4 u;
      __nv_bfloat16* h = (__nv_bfloat16*)&u;
#pragma unroll
      for (int q = 0; q < 8; ++q) h[q] = __float2bfloat16_rn(v[q]);
      *(uint4*)dst = u;
    } else {
      *(float4*)dst = make_float4(v[0], v[1], v[2], v[3]);
      *(float4*)(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
}

// Single-channel im2col with compile-time filter geometry (the 7x7 / stride 2 / pad 3
// stem): one block per (image, RB output rows). The input rows those outputs read are
// staged once in shared memory with the zero padding materialised, then every thread
// assembles 8 consecutive taps of one output pixel and writes them with one 16-byte
// (bf16) or two (fp32) stores; consecutive threads write consecutive bytes.
template <typename Ti, typename To, int KS, int S, int P, int RB>
__global__ void __launch_bounds__(256) im2col_stem_kernel(ConvGeom g, const Ti* __restrict__ x,
                                                          To* __restrict__ col) {
  DDPPO_PDL_ENTRY();
  constexpr int KK = KS * KS, KP = (KK + 7) / 8 * 8, NCK = KP / 8, ROWS = (RB - 1) * S + KS;
  extern __shared__ float tile[];  // [ROWS][W + 2P]
  const int n = blockIdx.y, oy0 = blockIdx.x * RB;
  const int Wp = g.W + 2 * P;
  const Ti* img = x + (size_t)n * g.H * g.W;
  const int iy0 = oy0 * S - P;
  for (int i = threadIdx.x; i < ROWS * Wp; i += blockDim.x) {
    const int r = i / Wp, c = i - r * Wp;
    const int iy = iy0 + r, ix = c - P;
    tile[i] = (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W) ? to_f(img[iy * g.W + ix]) : 0.f;
  }
  __syncthreads();
  const int rows = min(RB, g.Ho - oy0);
  const int items = rows * g.Wo * NCK;
  To* dst0 = col + ((size_t)n * g.Ho + oy0) * g.Wo * KP;
  for (int i = threadIdx.x; i < items; i += blockDim.x) {
    const int ck = i % NCK, px = i / NCK;
    const int r = px / g.Wo, ox = px - r * g.Wo;
    const float* base = tile + (r * S) * Wp + ox * S;
    float v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int kk = ck * 8 + q;
      const int ky = kk / KS, kx = kk - ky * KS;
      v[q] = kk < KK ? base[ky * Wp + kx] : 0.f;
    }
    To* dst = dst0 + (size_t)px * KP + ck * 8;
    if constexpr (sizeof(To) == 2) {
      uint4 u;
      __nv_bfloat16* h = (__nv_bfloat16*)&u;
#pragma unroll
      for (int q = 0; q < 8; ++q) h[q] = __float2bfloat16_rn(v[q]);
      *(uint4*)dst = u;
    } else {
      *(float4*)dst = make_float4(v[0], v[1], v[2], v[3]);
      *(float4*)(dst + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
  }
}

int launch_im2col(const ConvGeom& g, const void* x, bool x_bf16, void* col, bool op_bf16,
                  bool transposed, cudaStream_t s) {
  const size_t total = (size_t)g.N * g.Ho * g.Wo * g.Kp;
  if (total == 0) return DDPPO_OK;
  if (!transposed && g.C == 1 && g.k == 7 && g.s == 2 && g.p == 3 && g.Kp == 56 &&
      ((uintptr_t)col & 15) == 0 && g.N <= 65535 && g.W <= 900) {
    constexpr int RB = 4;  // 16 rows per block measured slower at the 64-image act batch
    const dim3 gb((unsigned)((g.Ho + RB - 1) / RB), (unsigned)g.N);
    const size_t smem = (size_t)((RB - 1) * 2 + 7) * (g.W + 6) * sizeof(float);
#define STEM_CASE(TI, TO) \
    ::ddppo::launch_k(im2col_stem_kernel<TI, TO, 7, 2, 3, RB>, gb, 256, smem, s, g, (const TI*)x, (TO*)col);
    if (x_bf16 && op_bf16) { STEM_CASE(__nv_bfloat16, __nv_bfloat16) }
    else if (x_bf16) { STEM_CASE(__nv_bfloat16, float) }
    else if (op_bf16) { STEM_CASE(float, __nv_bfloat16) }
    else { STEM_CASE(float, float) }
#undef STEM_CASE
    DDPPO_CHECK_LAUNCH();
    return DDPPO_OK;
  }
  if (!transposed && g.C == 1 && g.Kp % 8 == 0 && ((uintptr_t)col & 15) == 0 && g.N <= 65535 &&
      (int64_t)g.Ho * g.Wo * g.Kp < (1ll << 31) && (int64_t)g.H * g.W < (1ll << 31)) {
    const long per = (long)g.Ho * g.Wo * (g.Kp / 8);
    const dim3 gb((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256,
                                                             (8l * 152 + g.N - 1) / g.N)), g.N);
    if (x_bf16 && op_bf16)
      ::ddppo::launch_k(im2col_c1_kernel<__nv_bfloat16, __nv_bfloat16>, gb, 256, 0, s, g, (const __nv_bfloat16*)x, (__nv_bfloat16*)col);
    else if (x_bf16)
      ::ddppo::launch_k(im2col_c1_kernel<__nv_bfloat16, float>, gb, 256, 0, s, g, (const __nv_bfloat16*)x, (float*)col);
    else if (op_bf16)
      ::ddppo::launch_k(im2col_c1_kernel<float, __nv_bfloat16>, gb, 256, 0, s, g, (const float*)x, (__nv_bfloat16*)col);
    else
      ::ddppo::launch_k(im2col_c1_kernel<float, float>, gb, 256, 0, s, g, (const float*)x, (float*)col);
    DDPPO_CHECK_LAUNCH();
    return DDPPO_OK;
  }
  const bool vec = !transposed && g.C % 8 == 0 && g.Kp == g.K && g.Kp % 8 == 0 &&
                   ((uintptr_t)x & 15) == 0 && ((uintptr_t)col & 15) == 0;
  const unsigned gb = grid_for(vec ? total / 8 : total);
#define IM2COL_CASE(TI, TO)                                                                   \
  if (vec) ::ddppo::launch_k(im2col_vec_kernel<TI, TO>, gb, 256, 0, s, g, (const TI*)x, (TO*)col);           \
  else if (transposed) ::ddppo::launch_k(im2colT_kernel<TI, TO>, gb, 256, 0, s, g, (const TI*)x, (TO*)col);  \
  else ::ddppo::launch_k(im2col_kernel<TI, TO>, gb, 256, 0, s, g, (const TI*)x, (TO*)col);
  if (x_bf16 && op_bf16) { IM2COL_CASE(__nv_bfloat16, __nv_bfloat16) }
  else if (x_bf16) { IM2COL_CASE(__nv_bfloat16, float) }
  else if (op_bf16) { IM2COL_CASE(float, __nv_bfloat16) }
  else { IM2COL_CASE(float, float) }
#undef IM2COL_CASE
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void col2im_kernel(ConvGeom g, const float* __restrict__ dcol, float* __restrict__ dx,
                              int accumulate) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)g.N * g.H * g.W * g.C;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.C);
    const int ix = (int)((idx / g.C) % g.W), iy = (int)((idx / ((size_t)g.C * g.W)) % g.H);
    const int n = (int)(idx / ((size_t)g.C * g.W * g.H));
    float acc = 0.f;
    for (int ky = 0; ky < g.k; ++ky) {
      const int ty = iy + g.p - ky;
      if (ty < 0 || ty % g.s) continue;
      const int oy = ty / g.s;
      if (oy >= g.Ho) continue;
      for (int kx = 0; kx < g.k; ++kx) {
        const int tx = ix + g.p - kx;
        if (tx < 0 || tx % g.s) continue;
        const int ox = tx / g.s;
        if (ox >= g.Wo) continue;
        const size_t m = ((size_t)n * g.Ho + oy) * g.Wo + ox;
        acc += dcol[m * g.Kp + (ky * g.k + kx) * g.C + c];
      }
    }
    dx[idx] = accumulate ? dx[idx] + acc : acc;
  }
}

// vectorised col2im for C % 8 == 0: one thread per (pixel, 8-channel group)
__global__ void col2im_vec_kernel(ConvGeom g, const float* __restrict__ dcol, float* __restrict__ dx,
                                  int accumulate) {
  DDPPO_PDL_ENTRY();
  const int C8 = g.C >> 3;
  const size_t total = (size_t)g.N * g.H * g.W * C8;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c8 = (int)(idx % C8);
    const size_t pix = idx / C8;
    const int ix = (int)(pix % g.W), iy = (int)((pix / g.W) % g.H), n = (int)(pix / ((size_t)g.W * g.H));
    float a[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int ky = 0; ky < g.k; ++ky) {
      const int ty = iy + g.p - ky;
      if (ty < 0 || ty % g.s) continue;
      const int oy = ty / g.s;
      if (oy >= g.Ho) continue;
      for (int kx = 0; kx < g.k; ++kx) {
        const int tx = ix + g.p - kx;
        if (tx < 0 || tx % g.s) continue;
        const int ox = tx / g.s;
        if (ox >= g.Wo) continue;
        const float* src = dcol + (((size_t)n * g.Ho + oy) * g.Wo + ox) * g.Kp +
                           (size_t)(ky * g.k + kx) * g.C + c8 * 8;
        const float4 u = *(const float4*)src, w = *(const float4*)(src + 4);
        a[0] += u.x; a[1] += u.y; a[2] += u.z; a[3] += u.w;
        a[4] += w.x; a[5] += w.y; a[6] += w.z; a[7] += w.w;
      }
    }
    float* d = dx + pix * g.C + c8 * 8;
    if (accumulate) {
      const float4 u = *(const float4*)d, w = *(const float4*)(d + 4);
      a[0] += u.x; a[1] += u.y; a[2] += u.z; a[3] += u.w;
      a[4] += w.x; a[5] += w.y; a[6] += w.z; a[7] += w.w;
    }
    *(float4*)d = make_float4(a[0], a[1], a[2], a[3]);
    *(float4*)(d + 4) = make_float4(a[4], a[5], a[6], a[7]);
  }
}

int launch_col2im(const ConvGeom& g, const float* dcol, float* dx, bool accumulate, cudaStream_t s) {
  const size_t total = (size_t)g.N * g.H * g.W * g.C;
  if (total == 0) return DDPPO_OK;
  if (g.C % 8 == 0 && g.Kp % 4 == 0 && ((uintptr_t)dcol & 15) == 0 && ((uintptr_t)dx & 15) == 0)
    ::ddppo::launch_k(col2im_vec_kernel, grid_for(total / 8), 256, 0, s, g, dcol, dx, accumulate ? 1 : 0);
  else
    ::ddppo::launch_k(col2im_kernel, grid_for(total), 256, 0, s, g, dcol, dx, accumulate ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- transpose / cast
template <typename Ti, typename To>
__global__ void transpose_kernel(const Ti* __restrict__ in, To* __restrict__ out, int R, int Cc,
                                 int ld_in) {
  DDPPO_PDL_ENTRY();
  __shared__ float tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;  // rows on x: R can be in the millions
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = r0 + j, c = c0 + threadIdx.x;
    tile[j][threadIdx.x] = (r < R && c < Cc) ? to_f(in[(size_t)r * ld_in + c]) : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j, r = r0 + threadIdx.x;
    if (c < Cc && r < R) out[(size_t)c * R + r] = from_f<To>(tile[threadIdx.x][j]);
  }
}

int launch_transpose(const void* in, bool in_bf16, void* out, bool out_bf16, int R, int Cc,
                     int ld_in, cudaStream_t s) {
  if (R == 0 || Cc == 0) return DDPPO_OK;
  dim3 grid((R + 31) / 32, (Cc + 31) / 32), blk(32, 8);
  if (in_bf16 && out_bf16)
    ::ddppo::launch_k(transpose_kernel<__nv_bfloat16, __nv_bfloat16>, grid, blk, 0, s, (const __nv_bfloat16*)in, (__nv_bfloat16*)out, R, Cc, ld_in);
  else if (in_bf16)
    ::ddppo::launch_k(transpose_kernel<__nv_bfloat16, float>, grid, blk, 0, s, (const __nv_bfloat16*)in, (float*)out, R, Cc, ld_in);
  else if (out_bf16)
    ::ddppo::launch_k(transpose_kernel<float, __nv_bfloat16>, grid, blk, 0, s, (const float*)in, (__nv_bfloat16*)out, R, Cc, ld_in);
  else
    ::ddppo::launch_k(transpose_kernel<float, float>, grid, blk, 0, s, (const float*)in, (float*)out, R, Cc, ld_in);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void cast_kernel(const float* __restrict__ in, void* out, int bf, size_t n) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    st_op(out, i, in[i], bf);
}
int launch_cast(const float* in, void* out, bool out_bf16, size_t n, cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(cast_kernel, grid_for(n), 256, 0, s, in, out, out_bf16 ? 1 : 0, n);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- GroupNorm (2 channels / group)
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One block per image; blockDim = max(256, C) with C | blockDim, so thread t owns channel
// t % C and reads pixels t / C, t / C + blockDim / C, ... -- consecutive threads read
// consecutive channels of a pixel (coalesced). Two passes (mean, then the centred second
// moment); per-channel sums combine in shared memory in a fixed order.


// ---------------------------------------------------------------- ReLU backward, add
__global__ void relu_bwd_kernel(const float* dy, const float* __restrict__ y, size_t n, float* dz32,
                                void* dzop, int bf) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float v = y[i] > 0.f ? dy[i] : 0.f;
    if (dz32) dz32[i] = v;
    if (dzop) st_op(dzop, i, v, bf);
  }
}
int launch_relu_bwd(const float* dy, const float* y, size_t n, float* dz32, void* dzop, bool op_bf16,
                    cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(relu_bwd_kernel, grid_for(n), 256, 0, s, dy, y, n, dz32, dzop, op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void add_kernel(float* dst, const float* __restrict__ src, size_t n) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] += src[i];
}
int launch_add(float* dst, const float* src, size_t n, cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(add_kernel, grid_for(n), 256, 0, s, dst, src, n);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- max pool 3x3 / 2, pad 1
__global__ void maxpool_fwd_kernel(const float* __restrict__ x, int N, int H, int W, int C,
                                   float* __restrict__ y, uint8_t* __restrict__ arg,
                                   __nv_bfloat16* __restrict__ y_bf) {
  DDPPO_PDL_ENTRY();
  const int Ho = (H + 2 - 3) / 2 + 1, Wo = (W + 2 - 3) / 2 + 1;
  const size_t total = (size_t)N * Ho * Wo * C;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    const int ox = (int)((idx / C) % Wo), oy = (int)((idx / ((size_t)C * Wo)) % Ho);
    const int n = (int)(idx / ((size_t)C * Wo * Ho));
    float best = -INFINITY;
    int bi = 0;
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = oy * 2 - 1 + ky;
      if (iy < 0 || iy >= H) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = ox * 2 - 1 + kx;
        if (ix < 0 || ix >= W) continue;
        const float v = x[(((size_t)n * H + iy) * W + ix) * C + c];
        if (v > best) { best = v; bi = ky * 3 + kx; }
      }
    }
    y[idx] = best;
    if (y_bf) y_bf[idx] = __float2bfloat16_rn(best);
    arg[idx] = (uint8_t)bi;
  }
}
// 4 channels per thread (C % 4 == 0): float4 loads and stores, 32-bit index decoding
__global__ void maxpool_fwd4_kernel(const float* __restrict__ x, int H, int W, int C,
                                    float* __restrict__ y, uint8_t* __restrict__ arg,
                                    __nv_bfloat16* __restrict__ y_bf) {
  DDPPO_PDL_ENTRY();
  const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1, C4 = C / 4;
  const int n = blockIdx.y, per = Ho * Wo * C4;
  const float* xi = x + (size_t)n * H * W * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
    const int c4 = i % C4, pix = i / C4;
    const int ox = pix % Wo, oy = pix / Wo;
    float b[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int bi[4] = {0, 0, 0, 0};
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = oy * 2 - 1 + ky;
      if (iy < 0 || iy >= H) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = ox * 2 - 1 + kx;
        if (ix < 0 || ix >= W) continue;
        const float4 v = *reinterpret_cast<const float4*>(xi + ((size_t)iy * W + ix) * C + c4 * 4);
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (vv[q] > b[q]) { b[q] = vv[q]; bi[q] = ky * 3 + kx; }
      }
    }
    const size_t o = (size_t)n * per * 4 + (size_t)i * 4;
    *reinterpret_cast<float4*>(y + o) = make_float4(b[0], b[1], b[2], b[3]);
    if (y_bf) {
      __nv_bfloat162 h0 = __floats2bfloat162_rn(b[0], b[1]), h1 = __floats2bfloat162_rn(b[2], b[3]);
      *reinterpret_cast<uint2*>(y_bf + o) =
          make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1));
    }
    *reinterpret_cast<uchar4*>(arg + o) = make_uchar4(bi[0], bi[1], bi[2], bi[3]);
  }
}

int launch_maxpool_fwd(const float* x, int N, int H, int W, int C, float* y, uint8_t* arg,
                       __nv_bfloat16* y_bf, cudaStream_t s) {
  const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
  const size_t total = (size_t)N * Ho * Wo * C;
  if (!total) return DDPPO_OK;
  if (C % 4 == 0 && N <= 65535 && (int64_t)Ho * Wo * C < (1ll << 31)) {
    const long per = (long)Ho * Wo * (C / 4);
    const dim3 gb((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256, (8l * 152 + N - 1) / N)), N);
    ::ddppo::launch_k(maxpool_fwd4_kernel, gb, 256, 0, s, x, H, W, C, y, arg, y_bf);
  } else {
    ::ddppo::launch_k(maxpool_fwd_kernel, grid_for(total), 256, 0, s, x, N, H, W, C, y, arg, y_bf);
  }
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void maxpool_bwd_kernel(const float* __restrict__ dy, const uint8_t* __restrict__ arg,
                                   int N, int H, int W, int C, float* __restrict__ dx) {
  DDPPO_PDL_ENTRY();
  const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1;
  const size_t total = (size_t)N * H * W * C;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % C);
    const int ix = (int)((idx / C) % W), iy = (int)((idx / ((size_t)C * W)) % H);
    const int n = (int)(idx / ((size_t)C * W * H));
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int ty = iy + 1 - ky;
      if (ty < 0 || (ty & 1)) continue;
      const int oy = ty >> 1;
      if (oy >= Ho) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int tx = ix + 1 - kx;
        if (tx < 0 || (tx & 1)) continue;
        const int ox = tx >> 1;
        if (ox >= Wo) continue;
        const size_t o = (((size_t)n * Ho + oy) * Wo + ox) * C + c;
        if (arg[o] == ky * 3 + kx) acc += dy[o];
      }
    }
    dx[idx] = acc;
  }
}
__global__ void maxpool_bwd4_kernel(const float* __restrict__ dy, const uint8_t* __restrict__ arg,
                                    int H, int W, int C, float* __restrict__ dx) {
  DDPPO_PDL_ENTRY();
  const int Ho = (H - 1) / 2 + 1, Wo = (W - 1) / 2 + 1, C4 = C / 4;
  const int n = blockIdx.y, per = H * W * C4;
  const size_t ob = (size_t)n * Ho * Wo * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
    const int c4 = i % C4, pix = i / C4;
    const int ix = pix % W, iy = pix / W;
    // the (at most 2 x 2) windows covering this pixel: filter row ky covers it when
    // iy + 1 - ky is even and in range, i.e. ky = (iy + 1) & 1 and that + 2 (the same for
    // kx); the four candidate loads are issued first, then added in (ky, kx) order
    const int ky0 = (iy + 1) & 1, kx0 = (ix + 1) & 1;
    uchar4 a4[4];
    float4 d4[4];
    bool cov[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int ky = ky0 + 2 * (j >> 1), kx = kx0 + 2 * (j & 1);
      const int ty = iy + 1 - ky, tx = ix + 1 - kx;
      cov[j] = ky <= 2 && kx <= 2 && ty >= 0 && (ty >> 1) < Ho && tx >= 0 && (tx >> 1) < Wo;
      if (cov[j]) {
        const size_t o = ob + ((size_t)(ty >> 1) * Wo + (tx >> 1)) * C + c4 * 4;
        a4[j] = *reinterpret_cast<const uchar4*>(arg + o);
        d4[j] = *reinterpret_cast<const float4*>(dy + o);
      }
    }
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!cov[j]) continue;
      const int t = (ky0 + 2 * (j >> 1)) * 3 + kx0 + 2 * (j & 1);
      if (a4[j].x == t) acc[0] += d4[j].x;
      if (a4[j].y == t) acc[1] += d4[j].y;
      if (a4[j].z == t) acc[2] += d4[j].z;
      if (a4[j].w == t) acc[3] += d4[j].w;
    }
    *reinterpret_cast<float4*>(dx + (size_t)n * per * 4 + (size_t)i * 4) =
        make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
}

int launch_maxpool_bwd(const float* dy, const uint8_t* arg, int N, int H, int W, int C, float* dx,
                       cudaStream_t s) {
  const size_t total = (size_t)N * H * W * C;
  if (!total) return DDPPO_OK;
  if (C % 4 == 0 && N <= 65535 && (int64_t)H * W * C < (1ll << 31)) {
    const long per = (long)H * W * (C / 4);
    const dim3 gb((unsigned)std::max<long>(1, std::min<long>((per + 255) / 256, (8l * 152 + N - 1) / N)), N);
    ::ddppo::launch_k(maxpool_bwd4_kernel, gb, 256, 0, s, dy, arg, H, W, C, dx);
  } else {
    ::ddppo::launch_k(maxpool_bwd_kernel, grid_for(total), 256, 0, s, dy, arg, N, H, W, C, dx);
  }
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- column sums
// block (32, 8): column c = blockIdx.x*32 + tx; row lanes ty; fixed-order combine.
// out[c] (+)= sum over rows r of in[r * ld + c]. Block (32, 32): column c = blockIdx.x * 32
// + tx; row lane ty sums rows ty, ty + 32, ... (eight loads in flight); then a fixed-order
// combine over the 32 lanes. Two arrays of the same shape in one launch (blockIdx.y).
__global__ void __launch_bounds__(1024) colsum_kernel(const float* __restrict__ in0,
                                                      const float* __restrict__ in1, int R,
                                                      int Cc, int ld, float* __restrict__ out0,
                                                      float* __restrict__ out1, int accumulate) {
  DDPPO_PDL_ENTRY();
  __shared__ float sh[32][33];
  const float* in = blockIdx.y ? in1 : in0;
  float* out = blockIdx.y ? out1 : out0;
  const int c = blockIdx.x * 32 + threadIdx.x;
  float s = 0.f;
  if (c < Cc) {
#pragma unroll 8
    for (int r = threadIdx.y; r < R; r += 32) s += in[(size_t)r * ld + c];
  }
  sh[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && c < Cc) {
    float t = 0.f;
    for (int k = 0; k < 32; ++k) t += sh[k][threadIdx.x];
    out[c] = accumulate ? out[c] + t : t;
  }
}
int launch_colsum(const float* in, int R, int Cc, int ld, float* out, bool accumulate,
                  cudaStream_t s) {
  if (Cc == 0) return DDPPO_OK;
  ::ddppo::launch_k(colsum_kernel, dim3((Cc + 31) / 32, 1), dim3(32, 32), 0, s, in, in, R, Cc, ld, out, out,
                                                                 accumulate ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
int launch_colsum2(const float* in0, const float* in1, int R, int Cc, int ld, float* out0,
                   float* out1, bool accumulate, cudaStream_t s) {
  if (Cc == 0) return DDPPO_OK;
  ::ddppo::launch_k(colsum_kernel, dim3((Cc + 31) / 32, 2), dim3(32, 32), 0, s, in0, in1, R, Cc, ld, out0, out1,
                                                                 accumulate ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- LSTM cell
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

__global__ void lstm_fwd_kernel(LstmStep a) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)a.E * a.H;
  const int bf = a.op_bf16 ? 1 : 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / a.H), j = (int)(idx % a.H);
    const size_t gb = (size_t)e * 4 * a.H;
    const float zi = a.gx[gb + j] + a.gh[gb + j];
    const float zf = a.gx[gb + a.H + j] + a.gh[gb + a.H + j];
    const float zg = a.gx[gb + 2 * a.H + j] + a.gh[gb + 2 * a.H + j];
    const float zo = a.gx[gb + 3 * a.H + j] + a.gh[gb + 3 * a.H + j];
    const float i = sigm(zi), f = sigm(zf), g = tanhf(zg), o = sigm(zo);
    const float cp = a.m[e] ? a.c_prev[idx] : 0.f;
    const float c = f * cp + i * g;
    const float h = o * tanhf(c);
    a.gates[gb + j] = i; a.gates[gb + a.H + j] = f;
    a.gates[gb + 2 * a.H + j] = g; a.gates[gb + 3 * a.H + j] = o;
    a.c[idx] = c;
    a.h[idx] = h;
    if (a.y_op) st_op(a.y_op, idx, h, bf);
    if (a.hm_next) st_op(a.hm_next, idx, a.m_next[e] ? h : 0.f, bf);
  }
}
int launch_lstm_fwd(const LstmStep& a, cudaStream_t s) {
  const size_t total = (size_t)a.E * a.H;
  if (!total) return DDPPO_OK;
  ::ddppo::launch_k(lstm_fwd_kernel, grid_for(total), 256, 0, s, a);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void mask_state_kernel(const float* __restrict__ h0, const uint8_t* __restrict__ m,
                                  int E, int H, void* hm, int bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)E * H;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x)
    st_op(hm, idx, m[idx / H] ? h0[idx] : 0.f, bf);
}
int launch_mask_state(const float* h0, const uint8_t* m, int E, int H, void* hm, bool op_bf16,
                      cudaStream_t s) {
  const size_t total = (size_t)E * H;
  if (!total) return DDPPO_OK;
  ::ddppo::launch_k(mask_state_kernel, grid_for(total), 256, 0, s, h0, m, E, H, hm, op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// Backward of step t: the state entering t was (h, c)_{t-1} * m_t.
//   dh = dh_above + m_{t+1} dh_rec ; dc = dh o (1 - tanh^2 c) + m_{t+1} dc_carry
//   dz_i = dc g i(1-i), dz_f = dc c_prev_m f(1-f), dz_g = dc i (1-g^2), dz_o = dh tanh(c) o(1-o)
//   dc_carry <- dc f  (the caller's next step applies m_t)
__global__ void lstm_bwd_kernel(LstmBack a) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)a.E * a.H;
  const int bf = a.op_bf16 ? 1 : 0;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int e = (int)(idx / a.H), j = (int)(idx % a.H);
    const size_t gb = (size_t)e * 4 * a.H;
    const float i = a.gates[gb + j], f = a.gates[gb + a.H + j];
    const float g = a.gates[gb + 2 * a.H + j], o = a.gates[gb + 3 * a.H + j];
    const float c = a.c[idx];
    const float cp = (a.m[e] && a.c_prev) ? a.c_prev[idx] : 0.f;
    const bool carry = a.m_next && a.m_next[e];
    float dh = a.dh_above[idx];
    if (carry && a.dh_rec) dh += a.dh_rec[idx];
    const float tc = tanhf(c);
    float dc = dh * o * (1.f - tc * tc);
    if (carry) dc += a.dc_carry[idx];
    const float dzi = dc * g * i * (1.f - i);
    const float dzf = dc * cp * f * (1.f - f);
    const float dzg = dc * i * (1.f - g * g);
    const float dzo = dh * tc * o * (1.f - o);
    a.dc_carry[idx] = dc * f;
    a.dg32[gb + j] = dzi; a.dg32[gb + a.H + j] = dzf;
    a.dg32[gb + 2 * a.H + j] = dzg; a.dg32[gb + 3 * a.H + j] = dzo;
    if (a.dg_op) {
      st_op(a.dg_op, gb + j, dzi, bf); st_op(a.dg_op, gb + a.H + j, dzf, bf);
      st_op(a.dg_op, gb + 2 * a.H + j, dzg, bf); st_op(a.dg_op, gb + 3 * a.H + j, dzo, bf);
    }
  }
}
int launch_lstm_bwd(const LstmBack& a, cudaStream_t s) {
  const size_t total = (size_t)a.E * a.H;
  if (!total) return DDPPO_OK;
  ::ddppo::launch_k(lstm_bwd_kernel, grid_for(total), 256, 0, s, a);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- heads
// one warp per sample
__global__ void heads_fwd_kernel(Heads a) {
  DDPPO_PDL_ENTRY();
  const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (n >= a.N) return;
  const float* h = a.h + (size_t)n * a.H;
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int k = lane; k < a.H; k += 32) {
    const float hv = h[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += hv * a.Wa[q * a.H + k];
    s[4] += hv * a.Wv[k];
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) s[q] = warp_sum(s[q]);
  if (lane != 0) return;
  float lg[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) lg[q] = s[q] + a.ba[q];
  if (a.logits)
    for (int q = 0; q < 4; ++q) a.logits[(size_t)n * 4 + q] = lg[q];
  a.value[n] = s[4] + a.bv[0];
  if (a.action) {
    const float mx = fmaxf(fmaxf(lg[0], lg[1]), fmaxf(lg[2], lg[3]));
    float ex[4], z = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) { ex[q] = expf(lg[q] - mx); z += ex[q]; }
    const float u = a.u[n];
    float cdf = 0.f;
    int act = 3;
    for (int q = 0; q < 4; ++q) {
      cdf += ex[q] / z;
      if (cdf > u) { act = q; break; }
    }
    a.action[n] = act;
    a.logp[n] = lg[act] - mx - logf(z);
  }
}
int launch_heads_fwd(const Heads& a, cudaStream_t s) {
  if (!a.N) return DDPPO_OK;
  ::ddppo::launch_k(heads_fwd_kernel, nblk((size_t)a.N * 32, 256), 256, 0, s, a);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void heads_dh_kernel(int N, int H, const float* __restrict__ Wa,
                                const float* __restrict__ Wv, const float* __restrict__ dl,
                                const float* __restrict__ dv, float* __restrict__ dh) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * H;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(idx / H), k = (int)(idx % H);
    float v = dv[n] * Wv[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) v += dl[(size_t)n * 4 + q] * Wa[q * H + k];
    dh[idx] = v;
  }
}
// partial[chunk, q, k] = sum over the chunk's samples of d_q[n] * h[n, k]  (q: 4 logits + value)
__global__ void heads_wgrad_partial(int N, int H, int chunk, const float* __restrict__ h,
                                    const float* __restrict__ dl, const float* __restrict__ dv,
                                    float* __restrict__ part) {
  DDPPO_PDL_ENTRY();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int ch = blockIdx.y;
  if (k >= H) return;
  float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  const int n0 = ch * chunk, n1 = min(N, n0 + chunk);
  for (int n = n0; n < n1; ++n) {
    const float hv = h[(size_t)n * H + k];
#pragma unroll
    for (int q = 0; q < 4; ++q) s[q] += dl[(size_t)n * 4 + q] * hv;
    s[4] += dv[n] * hv;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) part[((size_t)ch * 5 + q) * H + k] = s[q];
}
__global__ void heads_wgrad_final(int H, int nch, const float* __restrict__ part, float* gWa,
                                  float* gWv) {
  DDPPO_PDL_ENTRY();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 5 * H) return;
  float s = 0.f;
#pragma unroll 8
  for (int c = 0; c < nch; ++c) s += part[(size_t)c * 5 * H + idx];
  const int q = idx / H, k = idx % H;
  if (q < 4) gWa[q * H + k] = s;
  else gWv[k] = s;
}
int launch_heads_bwd(int N, int H, const float* h, const float* Wa, const float* Wv,
                     const float* dlogits, const float* dvalue, float* dh, float* gWa, float* gba,
                     float* gWv, float* gbv, float* scratch, size_t scratch_elems, cudaStream_t s) {
  if (!N) return DDPPO_OK;
  ::ddppo::launch_k(heads_dh_kernel, grid_for((size_t)N * H), 256, 0, s, N, H, Wa, Wv, dlogits, dvalue, dh);
  DDPPO_CHECK_LAUNCH();
  int nch = (int)min((size_t)((N + 63) / 64), scratch_elems / (5 * (size_t)H));
  if (nch < 1) { set_error("heads_bwd: scratch too small"); return DDPPO_E_CONFIG; }
  const int chunk = (N + nch - 1) / nch;
  nch = (N + chunk - 1) / chunk;
  ::ddppo::launch_k(heads_wgrad_partial, dim3((H + 127) / 128, nch), 128, 0, s, N, H, chunk, h, dlogits, dvalue, scratch);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(heads_wgrad_final, nblk(5 * (size_t)H, 256), 256, 0, s, H, nch, scratch, gWa, gWv);
  DDPPO_CHECK_LAUNCH();
  DDPPO_TRY(launch_colsum(dlogits, N, 4, 4, gba, false, s));
  DDPPO_TRY(launch_colsum(dvalue, N, 1, 1, gbv, false, s));
  return DDPPO_OK;
}

// ---------------------------------------------------------------- goal / action embedding
__global__ void embed_fwd_kernel(int N, const float* __restrict__ goal,
                                 const int32_t* __restrict__ prev_a, const float* __restrict__ Wg,
                                 const float* __restrict__ bg, const float* __restrict__ Emb,
                                 void* x, int ldx, int col0, int bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * 64;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(idx / 64), j = (int)(idx % 64);
    float v;
    if (j < 32) {
      v = bg[j] + goal[3 * n] * Wg[3 * j] + goal[3 * n + 1] * Wg[3 * j + 1] +
          goal[3 * n + 2] * Wg[3 * j + 2];
    } else {
      int a = prev_a[n];
      a = a < 0 ? 0 : (a > 4 ? 4 : a);
      v = Emb[a * 32 + (j - 32)];
    }
    st_op(x, (size_t)n * ldx + col0 + j, v, bf);
  }
}
int launch_embed_fwd(int N, const float* goal, const int32_t* prev_a, const float* Wg,
                     const float* bg, const float* Emb, void* x, int ldx, int col0, bool op_bf16,
                     cudaStream_t s) {
  if (!N) return DDPPO_OK;
  ::ddppo::launch_k(embed_fwd_kernel, grid_for((size_t)N * 64), 256, 0, s, N, goal, prev_a, Wg, bg, Emb, x, ldx,
                                                            col0, op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
// warp per output weight: gWg[j, i] (96), gbg[j] (32), gEmb[a, j] (160). Lane l sums rows
// l, l + 32, ... (eight loads in flight); a fixed xor tree combines the lanes.
__global__ void __launch_bounds__(256) embed_bwd_kernel(int N, const float* __restrict__ goal,
                                                        const int32_t* __restrict__ prev_a,
                                                        const float* __restrict__ dx, int lddx,
                                                        int col0, float* gWg, float* gbg,
                                                        float* gEmb) {
  DDPPO_PDL_ENTRY();
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (t >= 96 + 32 + 160) return;
  float s = 0.f;
  if (t < 96) {
    const int j = t / 3, i = t % 3;
#pragma unroll 8
    for (int n = lane; n < N; n += 32) s += dx[(size_t)n * lddx + col0 + j] * goal[3 * n + i];
  } else if (t < 128) {
    const int j = t - 96;
#pragma unroll 8
    for (int n = lane; n < N; n += 32) s += dx[(size_t)n * lddx + col0 + j];
  } else {
    const int a = (t - 128) / 32, j = (t - 128) % 32;
#pragma unroll 8
    for (int n = lane; n < N; n += 32) {
      int pa = prev_a[n];
      pa = pa < 0 ? 0 : (pa > 4 ? 4 : pa);
      if (pa == a) s += dx[(size_t)n * lddx + col0 + 32 + j];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane != 0) return;
  if (t < 96) gWg[t] = s;
  else if (t < 128) gbg[t - 96] = s;
  else gEmb[t - 128] = s;
}
int launch_embed_bwd(int N, const float* goal, const int32_t* prev_a, const float* dx, int lddx,
                     int col0, float* gWg, float* gbg, float* gEmb, float*, size_t, cudaStream_t s) {
  ::ddppo::launch_k(embed_bwd_kernel, (288 + 7) / 8, 256, 0, s, N, goal, prev_a, dx, lddx, col0, gWg, gbg, gEmb);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void vis_relu_bwd_kernel(int N, int H, const float* __restrict__ dx, int lddx,
                                    const void* x, int ldx, int bf, float* dv32, void* dvop) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * H;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int n = (int)(idx / H), k = (int)(idx % H);
    const float xv = ld_any(x, (size_t)n * ldx + k, bf);
    const float v = xv > 0.f ? dx[(size_t)n * lddx + k] : 0.f;
    if (dv32) dv32[idx] = v;
    if (dvop) st_op(dvop, idx, v, bf);
  }
}
int launch_vis_relu_bwd(int N, int H, const float* dx, int lddx, const void* x, int ldx,
                        bool op_bf16, float* dv32, void* dvop, cudaStream_t s) {
  if (!N) return DDPPO_OK;
  ::ddppo::launch_k(vis_relu_bwd_kernel, grid_for((size_t)N * H), 256, 0, s, N, H, dx, lddx, x, ldx,
                                                              op_bf16 ? 1 : 0, dv32, dvop);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- gather rows
__global__ void gather_rows_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                   const int32_t* __restrict__ idx, int T, int Ein, int Eout,
                                   size_t words) {  // rows of `words` 4-byte words
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)T * Eout * words;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t w = i % words;
    const int j = (int)((i / words) % Eout), t = (int)(i / (words * Eout));
    const int src = idx ? idx[j] : j;
    ((uint32_t*)out)[i] = ((const uint32_t*)in)[((size_t)t * Ein + src) * words + w];
  }
}
__global__ void gather_rows_bytes_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                                         const int32_t* __restrict__ idx, int T, int Ein, int Eout,
                                         size_t bytes) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)T * Eout * bytes;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t w = i % bytes;
    const int j = (int)((i / bytes) % Eout), t = (int)(i / (bytes * Eout));
    const int src = idx ? idx[j] : j;
    out[i] = in[((size_t)t * Ein + src) * bytes + w];
  }
}
int launch_gather_rows(const void* in, void* out, const int32_t* idx, int T, int Ein, int Eout,
                       size_t bytes, cudaStream_t s) {
  const size_t total = (size_t)T * Eout * bytes;
  if (!total) return DDPPO_OK;
  if (bytes % 4 == 0 && ((uintptr_t)in & 3) == 0 && ((uintptr_t)out & 3) == 0)
    ::ddppo::launch_k(gather_rows_kernel, grid_for(total / 4), 256, 0, s, (const uint8_t*)in, (uint8_t*)out, idx,
                                                           T, Ein, Eout, bytes / 4);
  else
    ::ddppo::launch_k(gather_rows_bytes_kernel, grid_for(total), 256, 0, s, (const uint8_t*)in, (uint8_t*)out, idx,
                                                             T, Ein, Eout, bytes);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- weight layouts
// canonical w[co, ci, ky, kx] -> wg[co, (ky*k + kx)*cin + ci] and wgT[(..), co]; pad zero
__global__ void conv_w_prep_kernel(const float* __restrict__ w, int cout, int cin, int k, int Kp,
                                   void* wg, void* wgT, int bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)cout * Kp;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(idx / Kp), kk = (int)(idx % Kp);
    float v = 0.f;
    if (kk < k * k * cin) {
      const int ci = kk % cin, kx = (kk / cin) % k, ky = kk / (cin * k);
      v = w[(((size_t)co * cin + ci) * k + ky) * k + kx];
    }
    st_op(wg, idx, v, bf);
    if (wgT) st_op(wgT, (size_t)kk * cout + co, v, bf);
  }
}
int launch_conv_w_prep(const float* w, int cout, int cin, int k, int Kp, void* wg, void* wgT,
                       bool op_bf16, cudaStream_t s) {
  ::ddppo::launch_k(conv_w_prep_kernel, grid_for((size_t)cout * Kp), 256, 0, s, w, cout, cin, k, Kp, wg, wgT,
                                                                 op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void conv_w_flip_kernel(const float* __restrict__ w, int cout, int cin, int k, void* wr,
                                   int bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)cin * k * k * cout;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(idx % cout);
    const int tap = (int)((idx / cout) % (k * k));
    const int ci = (int)(idx / ((size_t)cout * k * k));
    const int ky = tap / k, kx = tap % k;
    st_op(wr, idx, w[(((size_t)co * cin + ci) * k + (k - 1 - ky)) * k + (k - 1 - kx)], bf);
  }
}
int launch_conv_w_flip(const float* w, int cout, int cin, int k, void* wr, bool op_bf16,
                       cudaStream_t s) {
  ::ddppo::launch_k(conv_w_flip_kernel, grid_for((size_t)cin * k * k * cout), 256, 0, s, w, cout, cin, k, wr,
                                                                          op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void conv_w_grad_kernel(const float* __restrict__ dwg, int cout, int cin, int k, int Kp,
                                   float* __restrict__ dw) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)cout * cin * k * k;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(idx % k), ky = (int)((idx / k) % k), ci = (int)((idx / (k * k)) % cin);
    const int co = (int)(idx / ((size_t)k * k * cin));
    dw[idx] = dwg[(size_t)co * Kp + (ky * k + kx) * cin + ci];
  }
}
int launch_conv_w_grad(const float* dwg, int cout, int cin, int k, int Kp, float* dw,
                       cudaStream_t s) {
  ::ddppo::launch_k(conv_w_grad_kernel, grid_for((size_t)cout * cin * k * k), 256, 0, s, dwg, cout, cin, k, Kp, dw);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void vis_w_prep_kernel(const float* __restrict__ w, int H, int C, int HW, void* wg,
                                  void* wgT, int bf) {
  DDPPO_PDL_ENTRY();
  const int F = C * HW;
  const size_t total = (size_t)H * F;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(idx / F), jg = (int)(idx % F);
    const int c = jg % C, hw = jg / C;
    const float v = w[(size_t)h * F + (size_t)c * HW + hw];
    st_op(wg, idx, v, bf);
    if (wgT) st_op(wgT, (size_t)jg * H + h, v, bf);
  }
}
int launch_vis_w_prep(const float* w, int H, int C, int HW, void* wg, void* wgT, bool op_bf16,
                      cudaStream_t s) {
  ::ddppo::launch_k(vis_w_prep_kernel, grid_for((size_t)H * C * HW), 256, 0, s, w, H, C, HW, wg, wgT, op_bf16 ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void vis_w_grad_kernel(const float* __restrict__ dwg, int H, int C, int HW,
                                  float* __restrict__ dw) {
  DDPPO_PDL_ENTRY();
  const int F = C * HW;
  const size_t total = (size_t)H * F;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(idx / F), j = (int)(idx % F);
    const int c = j / HW, hw = j % HW;
    dw[idx] = dwg[(size_t)h * F + (size_t)hw * C + c];
  }
}
int launch_vis_w_grad(const float* dwg, int H, int C, int HW, float* dw, cudaStream_t s) {
  ::ddppo::launch_k(vis_w_grad_kernel, grid_for((size_t)H * C * HW), 256, 0, s, dwg, H, C, HW, dw);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void add_vec_kernel(const float* a, const float* b, float* out, int n) {
  DDPPO_PDL_ENTRY();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}
int launch_add_vec(const float* a, const float* b, float* out, int n, cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(add_vec_kernel, nblk(n, 256), 256, 0, s, a, b, out, n);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- init
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void init_uniform_kernel(float* p, size_t n, float lo, float hi, uint64_t seed,
                                    uint64_t stream) {
  DDPPO_PDL_ENTRY();
  const uint64_t key = mix64(mix64(seed) + 0xD1B54A32D192ED03ull * (stream + 1));
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float u = (float)(mix64(key + i) >> 40) * (1.0f / 16777216.0f);
    p[i] = lo + (hi - lo) * u;
  }
}
int launch_init_uniform(float* p, size_t n, float lo, float hi, uint64_t seed, uint64_t stream,
                        cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(init_uniform_kernel, grid_for(n), 256, 0, s, p, n, lo, hi, seed, stream);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}
__global__ void fill_kernel(float* p, size_t n, float v) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}
int launch_fill(float* p, size_t n, float v, cudaStream_t s) {
  if (!n) return DDPPO_OK;
  ::ddppo::launch_k(fill_kernel, grid_for(n), 256, 0, s, p, n, v);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
