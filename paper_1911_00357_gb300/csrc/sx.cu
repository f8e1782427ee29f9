// Kernels of the SE-ResNeXt encoder (App. "Visual Encoder": SE-ResNeXt50/101 with every
// layer's channels halved and GroupNorm; ResNeXt's grouped 3x3 convolution, Xie et al.
// 2017; squeeze-and-excitation, Hu et al. 2018).
//
// Grouped 3x3 convolution, padding 1, stride 1 or 2, on NHWC activations: channel c of
// the output reads only the cpg = C / G input channels of its group. With 32 groups the
// groups hold 2-16 channels, far narrower than a 128-row MMA tile, so these are direct
// SIMT kernels with fp32 accumulation (operands in the precision's dtype):
//   forward   one thread per output element, 9 cpg MACs;
//   dgrad     one thread per input element, the transposed taps;
//   wgrad     per (group, pixel chunk) block: the chunk's output gradients and input
//             patches staged in shared memory, each thread accumulating some of the
//             group's cpg x cpg x 9 weights; per-chunk partial sums reduced in chunk order.
// Weights are kept as [C][ky][kx][ci] (ci within the group) in the operand dtype.
//
// Squeeze-excite on the branch u (the third GroupNorm's output), per image:
//   m = mean_hw(u); a = relu(W1 m + b1); g = sigmoid(W2 a + b2); y = relu(u g + shortcut)
// and its backward. Every reduction runs in a fixed order (deterministic).
#include <algorithm>

#include "nn_kernels.cuh"

namespace ddppo {

static inline unsigned sx_blocks(size_t n, int t) {
  return (unsigned)std::min<size_t>((n + t - 1) / t, 1u << 20);
}

template <typename T> __device__ __forceinline__ float ldf(const T* p, size_t i);
template <> __device__ __forceinline__ float ldf<float>(const float* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
  return __bfloat162float(p[i]);
}

// ---------------------------------------------------------------- grouped convolution
template <typename T>
__global__ void gconv_fwd_kernel(GConv g, const T* __restrict__ x, const T* __restrict__ w,
                                 float* __restrict__ z) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)g.N * g.Ho * g.Wo * g.C;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.C);
    const size_t pix = idx / g.C;
    const int ox = (int)(pix % g.Wo), oy = (int)((pix / g.Wo) % g.Ho);
    const int n = (int)(pix / ((size_t)g.Wo * g.Ho));
    const int ci0 = (c / g.cpg) * g.cpg;
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = oy * g.s - 1 + ky;
      if (iy < 0 || iy >= g.H) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = ox * g.s - 1 + kx;
        if (ix < 0 || ix >= g.W) continue;
        const size_t xb = (((size_t)n * g.H + iy) * g.W + ix) * g.C + ci0;
        const size_t wb = (((size_t)c * 3 + ky) * 3 + kx) * g.cpg;
        for (int ci = 0; ci < g.cpg; ++ci) acc += ldf(x, xb + ci) * ldf(w, wb + ci);
      }
    }
    z[idx] = acc;
  }
}

template <typename T>
__global__ void gconv_dgrad_kernel(GConv g, const T* __restrict__ dz, const T* __restrict__ w,
                                   float* __restrict__ dx, int accumulate) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)g.N * g.H * g.W * g.C;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % g.C);
    const size_t pix = idx / g.C;
    const int ix = (int)(pix % g.W), iy = (int)((pix / g.W) % g.H);
    const int n = (int)(pix / ((size_t)g.W * g.H));
    const int gi = c / g.cpg, co0 = gi * g.cpg, ci = c - co0;
    float acc = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
      const int ty = iy + 1 - ky;  // = oy * s
      if (ty < 0 || ty % g.s) continue;
      const int oy = ty / g.s;
      if (oy >= g.Ho) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int tx = ix + 1 - kx;
        if (tx < 0 || tx % g.s) continue;
        const int ox = tx / g.s;
        if (ox >= g.Wo) continue;
        const size_t db = (((size_t)n * g.Ho + oy) * g.Wo + ox) * g.C + co0;
        for (int co = 0; co < g.cpg; ++co)
          acc += ldf(dz, db + co) * ldf(w, ((((size_t)(co0 + co)) * 3 + ky) * 3 + kx) * g.cpg + ci);
      }
    }
    dx[idx] = accumulate ? dx[idx] + acc : acc;
  }
}

constexpr int GW_PIX = 32;      // output pixels staged per tile
constexpr int GW_THREADS = 256;

// partial sums of one (group, pixel chunk): part[chunk][c_out][ci][ky][kx] (canonical
// order within the group's rows)
template <typename T>
__global__ void __launch_bounds__(GW_THREADS)
    gconv_wgrad_kernel(GConv g, const T* __restrict__ x, const T* __restrict__ dz, int pix_per_chunk,
                       float* __restrict__ part) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  const int cpg = g.cpg, gi = blockIdx.x, chunk = blockIdx.y;
  float* sdz = sh;                         // [GW_PIX][cpg]
  float* sx = sh + GW_PIX * cpg;           // [GW_PIX][9][cpg]
  const int nw = cpg * cpg * 9;            // weights of the group
  const size_t M = (size_t)g.N * g.Ho * g.Wo;
  const size_t p0 = (size_t)chunk * pix_per_chunk;
  const size_t p1 = std::min<size_t>(M, p0 + pix_per_chunk);
  constexpr int kMaxPerThread = 9;  // cpg <= 16: 2304 weights over 256 threads
  float acc[kMaxPerThread];
#pragma unroll
  for (int i = 0; i < kMaxPerThread; ++i) acc[i] = 0.f;
  for (size_t pt = p0; pt < p1; pt += GW_PIX) {
    const int np = (int)std::min<size_t>(GW_PIX, p1 - pt);
    __syncthreads();
    for (int i = threadIdx.x; i < GW_PIX * cpg; i += blockDim.x) {
      const int p = i / cpg, co = i - p * cpg;
      sdz[i] = p < np ? ldf(dz, (pt + p) * g.C + gi * cpg + co) : 0.f;
    }
    for (int i = threadIdx.x; i < GW_PIX * 9 * cpg; i += blockDim.x) {
      const int p = i / (9 * cpg), r = i - p * 9 * cpg, tap = r / cpg, ci = r - tap * cpg;
      float v = 0.f;
      if (p < np) {
        const size_t m = pt + p;
        const int ox = (int)(m % g.Wo), oy = (int)((m / g.Wo) % g.Ho);
        const int n = (int)(m / ((size_t)g.Wo * g.Ho));
        const int iy = oy * g.s - 1 + tap / 3, ix = ox * g.s - 1 + tap % 3;
        if (iy >= 0 && iy < g.H && ix >= 0 && ix < g.W)
          v = ldf(x, (((size_t)n * g.H + iy) * g.W + ix) * g.C + gi * cpg + ci);
      }
      sx[i] = v;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kMaxPerThread; ++j) {
      const int wi = threadIdx.x + j * blockDim.x;
      if (wi >= nw) break;
      // canonical order within the group: (co, ci, ky, kx)
      const int co = wi / (cpg * 9), r = wi - co * cpg * 9, ci = r / 9, tap = r - ci * 9;
      float a = acc[j];
      for (int p = 0; p < np; ++p) a += sdz[p * cpg + co] * sx[(p * 9 + tap) * cpg + ci];
      acc[j] = a;
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxPerThread; ++j) {
    const int wi = threadIdx.x + j * blockDim.x;
    if (wi >= nw) break;
    part[(size_t)chunk * g.C * cpg * 9 + (size_t)gi * nw + wi] = acc[j];
  }
}

// dw[i] (= beta dw + sum over chunks in order), i over C * cpg * 9 canonical weights
__global__ void gconv_wgrad_reduce_kernel(const float* __restrict__ part, int chunks, size_t nwt,
                                          float* __restrict__ dw, float beta) {
  DDPPO_PDL_ENTRY();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwt;
       i += (size_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int c = 0; c < chunks; ++c) v += part[(size_t)c * nwt + i];
    dw[i] = beta != 0.f ? beta * dw[i] + v : v;
  }
}

// canonical [C][cpg][3][3] fp32 -> [C][3][3][cpg] operand dtype
__global__ void gconv_w_prep_kernel(const float* __restrict__ w, int C, int cpg, void* out, int bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)C * cpg * 9;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / (cpg * 9)), r = (int)(i - (size_t)c * cpg * 9), ci = r / 9, tap = r - ci * 9;
    const size_t o = ((size_t)c * 9 + tap) * cpg + ci;
    if (bf) ((__nv_bfloat16*)out)[o] = __float2bfloat16_rn(w[i]);
    else ((float*)out)[o] = w[i];
  }
}

int gconv_wgrad_chunks(const GConv& g, int num_sms) {
  const size_t M = (size_t)g.N * g.Ho * g.Wo;
  const int G = g.C / g.cpg;
  const int want = std::max(1, (4 * num_sms + G - 1) / G);
  const int most = (int)std::max<size_t>(1, (M + GW_PIX - 1) / GW_PIX);
  return std::min(want, most);
}

int launch_gconv_fwd(const GConv& g, const void* x, const void* w, float* z, bool bf, cudaStream_t s) {
  const size_t total = (size_t)g.N * g.Ho * g.Wo * g.C;
  if (!total) return DDPPO_OK;
  if (bf)
    ::ddppo::launch_k(gconv_fwd_kernel<__nv_bfloat16>, sx_blocks(total, 256), 256, 0, s, g, (const __nv_bfloat16*)x,
                                                           (const __nv_bfloat16*)w, z);
  else
    ::ddppo::launch_k(gconv_fwd_kernel<float>, sx_blocks(total, 256), 256, 0, s, g, (const float*)x, (const float*)w, z);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_gconv_dgrad(const GConv& g, const void* dz, const void* w, float* dx, bool accumulate,
                       bool bf, cudaStream_t s) {
  const size_t total = (size_t)g.N * g.H * g.W * g.C;
  if (!total) return DDPPO_OK;
  if (bf)
    ::ddppo::launch_k(gconv_dgrad_kernel<__nv_bfloat16>, sx_blocks(total, 256), 256, 0, s,
        g, (const __nv_bfloat16*)dz, (const __nv_bfloat16*)w, dx, accumulate ? 1 : 0);
  else
    ::ddppo::launch_k(gconv_dgrad_kernel<float>, sx_blocks(total, 256), 256, 0, s, g, (const float*)dz, (const float*)w,
                                                             dx, accumulate ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_gconv_wgrad(const GConv& g, const void* x, const void* dz, float* part, size_t part_elems,
                       int num_sms, float* dw, float beta, bool bf, cudaStream_t s) {
  if (g.cpg > 16) {
    set_error("grouped convolution: at most 16 channels per group");
    return DDPPO_E_CONFIG;
  }
  const size_t M = (size_t)g.N * g.Ho * g.Wo;
  const size_t nwt = (size_t)g.C * g.cpg * 9;
  const int chunks = gconv_wgrad_chunks(g, num_sms);
  if ((size_t)chunks * nwt > part_elems) {
    set_error("grouped convolution: weight-gradient scratch too small");
    return DDPPO_E_CONFIG;
  }
  const int ppc = (int)((M + chunks - 1) / chunks);
  const dim3 grid(g.C / g.cpg, chunks);
  const size_t smem = (size_t)GW_PIX * 10 * g.cpg * sizeof(float);
  if (bf)
    ::ddppo::launch_k(gconv_wgrad_kernel<__nv_bfloat16>, grid, GW_THREADS, smem, s, g, (const __nv_bfloat16*)x,
                                                      (const __nv_bfloat16*)dz, ppc, part);
  else
    ::ddppo::launch_k(gconv_wgrad_kernel<float>, grid, GW_THREADS, smem, s, g, (const float*)x, (const float*)dz, ppc, part);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(gconv_wgrad_reduce_kernel, sx_blocks(nwt, 256), 256, 0, s, part, chunks, nwt, dw, beta);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_gconv_w_prep(const float* w, int C, int cpg, void* out, bool bf, cudaStream_t s) {
  const size_t total = (size_t)C * cpg * 9;
  ::ddppo::launch_k(gconv_w_prep_kernel, sx_blocks(total, 256), 256, 0, s, w, C, cpg, out, bf ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---------------------------------------------------------------- squeeze-excite
// m[n, c] = mean over the HW pixels of u[n, :, c]
__global__ void se_squeeze_kernel(const float* __restrict__ u, int N, int HW, int C,
                                  float* __restrict__ m) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / C;
    const int c = (int)(i - n * C);
    const float* p = u + n * HW * C + c;
    float s = 0.f;
    for (int q = 0; q < HW; ++q) s += p[(size_t)q * C];
    m[i] = s / (float)HW;
  }
}

__device__ __forceinline__ float warp_sum_sx(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// one block per image: a = relu(W1 m + b1) [Cr], g = sigmoid(W2 a + b2) [C]
__global__ void se_fc_fwd_kernel(const float* __restrict__ m, const float* __restrict__ W1,
                                 const float* __restrict__ b1, const float* __restrict__ W2,
                                 const float* __restrict__ b2, int C, int Cr, float* __restrict__ a,
                                 float* __restrict__ gate) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sm[];
  float* sm_m = sm;       // [C]
  float* sm_a = sm + C;   // [Cr]
  const int n = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < C; c += blockDim.x) sm_m[c] = m[(size_t)n * C + c];
  __syncthreads();
  for (int j = wid; j < Cr; j += nw) {
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += W1[(size_t)j * C + c] * sm_m[c];
    s = warp_sum_sx(s) + b1[j];
    if (lane == 0) {
      const float v = fmaxf(s, 0.f);
      sm_a[j] = v;
      a[(size_t)n * Cr + j] = v;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = b2[c];
    for (int j = 0; j < Cr; ++j) s += W2[(size_t)c * Cr + j] * sm_a[j];
    gate[(size_t)n * C + c] = 1.f / (1.f + expf(-s));
  }
}

// y = relu(u g[n, c] + sc) (sc = null: no shortcut), fp32 and optional bf16 copy
__global__ void se_apply_kernel(const float* __restrict__ u, const float* __restrict__ gate,
                                const float* __restrict__ sc, int N, int HW, int C,
                                float* __restrict__ y, __nv_bfloat16* __restrict__ y_bf) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * HW * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const size_t n = i / ((size_t)HW * C);
    float v = u[i] * gate[n * C + c];
    if (sc) v += sc[i];
    v = fmaxf(v, 0.f);
    y[i] = v;
    if (y_bf) y_bf[i] = __float2bfloat16_rn(v);
  }
}

// gpre = gy (y > 0) (in place allowed); dg[n, c] = sum over pixels of gpre u
__global__ void se_bwd_reduce_kernel(const float* gy, const float* __restrict__ y,
                                     const float* __restrict__ u, int N, int HW, int C, float* gpre,
                                     float* __restrict__ dg) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t n = i / C;
    const int c = (int)(i - n * C);
    float s = 0.f;
    for (int q = 0; q < HW; ++q) {
      const size_t o = (n * HW + q) * C + c;
      const float g = y[o] > 0.f ? gy[o] : 0.f;
      gpre[o] = g;
      s += g * u[o];
    }
    dg[i] = s;
  }
}

// one block per image: dq = dg g (1 - g); da = W2^T dq; dh = da (a > 0); dm = W1^T dh
__global__ void se_fc_bwd_kernel(const float* __restrict__ dg, const float* __restrict__ gate,
                                 const float* __restrict__ a, const float* __restrict__ W1,
                                 const float* __restrict__ W2, int C, int Cr, float* __restrict__ dq,
                                 float* __restrict__ dh, float* __restrict__ dm) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sm[];
  float* sm_q = sm;       // [C]
  float* sm_h = sm + C;   // [Cr]
  const int n = blockIdx.x, lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const float g = gate[(size_t)n * C + c];
    const float q = dg[(size_t)n * C + c] * g * (1.f - g);
    sm_q[c] = q;
    dq[(size_t)n * C + c] = q;
  }
  __syncthreads();
  for (int j = wid; j < Cr; j += nw) {
    float s = 0.f;
    for (int c = lane; c < C; c += 32) s += W2[(size_t)c * Cr + j] * sm_q[c];
    s = warp_sum_sx(s);
    if (lane == 0) {
      const float v = a[(size_t)n * Cr + j] > 0.f ? s : 0.f;
      sm_h[j] = v;
      dh[(size_t)n * Cr + j] = v;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.f;
    for (int j = 0; j < Cr; ++j) s += W1[(size_t)j * C + c] * sm_h[j];
    dm[(size_t)n * C + c] = s;
  }
}

// du = gpre g[n, c] + dm[n, c] / HW
__global__ void se_du_kernel(const float* __restrict__ gpre, const float* __restrict__ gate,
                             const float* __restrict__ dm, int N, int HW, int C,
                             float* __restrict__ du) {
  DDPPO_PDL_ENTRY();
  const size_t total = (size_t)N * HW * C;
  const float inv = 1.f / (float)HW;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const size_t n = i / ((size_t)HW * C);
    du[i] = gpre[i] * gate[n * C + c] + dm[n * C + c] * inv;
  }
}

// parameter gradients of the two FCs, summed over the N images in order:
//   gW1[j, c] = sum dh[n, j] m[n, c]; gb1[j] = sum dh[n, j];
//   gW2[c, j] = sum dq[n, c] a[n, j]; gb2[c] = sum dq[n, c]   (+= when accumulate)
__global__ void se_wgrad_kernel(const float* __restrict__ dq, const float* __restrict__ dh,
                                const float* __restrict__ a, const float* __restrict__ m, int N,
                                int C, int Cr, float* __restrict__ gW1, float* __restrict__ gb1,
                                float* __restrict__ gW2, float* __restrict__ gb2, int accumulate) {
  DDPPO_PDL_ENTRY();
  const size_t n1 = (size_t)Cr * C, n2 = n1 + Cr, n3 = n2 + (size_t)C * Cr, total = n3 + C;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    float* dst;
    if (i < n1) {
      const int j = (int)(i / C), c = (int)(i % C);
      for (int n = 0; n < N; ++n) s += dh[(size_t)n * Cr + j] * m[(size_t)n * C + c];
      dst = gW1 + i;
    } else if (i < n2) {
      const int j = (int)(i - n1);
      for (int n = 0; n < N; ++n) s += dh[(size_t)n * Cr + j];
      dst = gb1 + j;
    } else if (i < n3) {
      const size_t k = i - n2;
      const int c = (int)(k / Cr), j = (int)(k % Cr);
      for (int n = 0; n < N; ++n) s += dq[(size_t)n * C + c] * a[(size_t)n * Cr + j];
      dst = gW2 + k;
    } else {
      const int c = (int)(i - n3);
      for (int n = 0; n < N; ++n) s += dq[(size_t)n * C + c];
      dst = gb2 + c;
    }
    *dst = accumulate ? *dst + s : s;
  }
}

int launch_se_fwd(const SeArgs& e, cudaStream_t s) {
  const size_t NC = (size_t)e.N * e.C, tot = NC * e.HW;
  ::ddppo::launch_k(se_squeeze_kernel, sx_blocks(NC, 256), 256, 0, s, e.u, e.N, e.HW, e.C, e.m);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(se_fc_fwd_kernel, e.N, 256, (size_t)(e.C + e.Cr) * 4, s, e.m, e.W1, e.b1, e.W2, e.b2, e.C, e.Cr,
                                                             e.a, e.gate);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(se_apply_kernel, sx_blocks(tot, 256), 256, 0, s, e.u, e.gate, e.sc, e.N, e.HW, e.C, e.y, e.y_bf);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_se_bwd(const SeArgs& e, const float* gy, float* gpre, float* du, bool accumulate,
                  cudaStream_t s) {
  const size_t NC = (size_t)e.N * e.C, tot = NC * e.HW;
  ::ddppo::launch_k(se_bwd_reduce_kernel, sx_blocks(NC, 256), 256, 0, s, gy, e.y, e.u, e.N, e.HW, e.C, gpre, e.dg);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(se_fc_bwd_kernel, e.N, 256, (size_t)(e.C + e.Cr) * 4, s, e.dg, e.gate, e.a, e.W1, e.W2, e.C,
                                                             e.Cr, e.dq, e.dh, e.dm);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(se_du_kernel, sx_blocks(tot, 256), 256, 0, s, gpre, e.gate, e.dm, e.N, e.HW, e.C, du);
  DDPPO_CHECK_LAUNCH();
  const size_t np = (size_t)e.Cr * e.C * 2 + e.Cr + e.C;
  ::ddppo::launch_k(se_wgrad_kernel, sx_blocks(np, 256), 256, 0, s, e.dq, e.dh, e.a, e.m, e.N, e.C, e.Cr, e.gW1,
                                                     e.gb1, e.gW2, e.gb2, accumulate ? 1 : 0);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
