// GroupNorm with groups of two channels (C/2 groups per image), the normalisation of the
// ResNet encoder's convolutions (Sec. 4 replaces BatchNorm by GroupNorm). Activations are
// NHWC fp32 [N, HW, C].
//
// The statistics and the backward reductions split every image over S blocks (a grid of
// S x N) so that a small batch -- the 64 frames of one rollout step -- still covers every
// SM. Each thread owns V consecutive channels (V = 4, or 2 when C % 4 != 0) of one pixel
// row and loads them as one vector. Blocks write per-channel partial sums; the last block
// of an image to finish (a per-image arrival counter, re-armed by that block) combines the
// S partials in block order, so every result is deterministic. The element-wise passes
// (normalise + residual + ReLU, and the input gradient) are vectorised the same way.
#include <algorithm>

#include "nn_kernels.cuh"

namespace ddppo {

namespace {

constexpr int kThreads = 256;

template <int V>
__device__ __forceinline__ void ldv(const float* p, float (&v)[V]) {
  if constexpr (V == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
}
template <int V>
__device__ __forceinline__ void stv(float* p, const float (&v)[V]) {
  if constexpr (V == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  else *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
template <int V>
__device__ __forceinline__ void stv_bf(__nv_bfloat16* p, const float (&v)[V]) {
  if constexpr (V == 4) *reinterpret_cast<uint2*>(p) = make_uint2(pack_bf2(v[0], v[1]), pack_bf2(v[2], v[3]));
  else *reinterpret_cast<uint32_t*>(p) = pack_bf2(v[0], v[1]);
}

// E4M3 codes of v / sc (saturating), V consecutive bytes
template <int V>
__device__ __forceinline__ void stv_e4m3(uint8_t* p, const float (&v)[V], float sc) {
  uint32_t w = 0;
#pragma unroll
  for (int j = 0; j < V; ++j) w |= (uint32_t)e4m3_sat(v[j] / sc) << (8 * j);
  if (V == 4) *reinterpret_cast<uint32_t*>(p) = w;
  else *reinterpret_cast<uint16_t*>(p) = (uint16_t)w;
}

// the block's largest m folded into *amax (one atomic per block; every thread calls it)
__device__ __forceinline__ void block_amax(float m, unsigned* amax) {
  __shared__ float wm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wm[w]);
    atomicMax(amax, __float_as_uint(b));
  }
}
template <int V>
__device__ __forceinline__ void stv_op(void* p, size_t i, const float (&v)[V], bool bf) {
  if (bf) stv_bf<V>((__nv_bfloat16*)p + i, v);
  else stv<V>((float*)p + i, v);
}

// threads of the block: R = C / V per pixel row, P rows per pass
__host__ __device__ inline int rows_per_pass(int C, int V) {
  const int R = C / V;
  return R >= kThreads ? 1 : kThreads / R;
}

// sums the per-thread pair (a[v], b[v]) over the P rows of the block for every channel,
// in row order; results for channel c at out[2c], out[2c + 1]. sh holds blockDim x 2V.
template <int V>
__device__ __forceinline__ void block_pair_sums(const float (&a)[V], const float (&b)[V], float* sh,
                                                int C, float* out) {
  const int R = C / V, P = blockDim.x / R;
  for (int v = 0; v < V; ++v) {
    sh[threadIdx.x * 2 * V + v] = a[v];
    sh[threadIdx.x * 2 * V + V + v] = b[v];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    const int cv = c / V, v = c % V;
    float sa = 0.f, sb = 0.f;
    for (int r = 0; r < P; ++r) {
      const float* q = sh + (size_t)(r * R + cv) * 2 * V;
      sa += q[v];
      sb += q[V + v];
    }
    out[2 * c] = sa;
    out[2 * c + 1] = sb;
  }
}

// true in exactly one block per image: the last to arrive after writing its partials
__device__ __forceinline__ bool last_of_image(int* cnt, int S, int* flag) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *flag = atomicAdd(cnt, 1) == S - 1;
  __syncthreads();
  if (!*flag) return false;
  __threadfence();
  return true;
}

// ---- statistics: shifted sums about the image's first pixel, combined in double ----
// the block's per-channel (sum d, sum d^2), d = z - z[first pixel], over its pixel rows
// [pb, pe) of image zi, written to pp[2c], pp[2c + 1]
template <int V>
__device__ __forceinline__ void block_shifted_sums(const float* __restrict__ zi, int pb, int pe, int C,
                                                   float* sh, float* pp) {
  const int R = C / V, P = blockDim.x / R;
  const int cv = threadIdx.x % R, pr = threadIdx.x / R, c0 = cv * V;
  float K[V], s1[V], s2[V];
  ldv<V>(zi + c0, K);
#pragma unroll
  for (int v = 0; v < V; ++v) s1[v] = s2[v] = 0.f;
#pragma unroll 8
  for (int p = pb + pr; p < pe; p += P) {
    float x[V];
    ldv<V>(zi + (size_t)p * C + c0, x);
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float d = x[v] - K[v];
      s1[v] += d;
      s2[v] += d * d;
    }
  }
  block_pair_sums<V>(s1, s2, sh, C, pp);
}

// the image's group means and 1 / sqrt(var + eps) from its S x C x 2 partials, read
// through L2 into sh and combined in block order (double); results to mean[g], rstd[g]
__device__ __forceinline__ void combine_groups(const float* pim, const float* __restrict__ zi, int S,
                                               int C, int HW, float eps, float* sh, float* mean,
                                               float* rstd) {
  for (int i = threadIdx.x; i < S * C * 2; i += blockDim.x) sh[i] = __ldcg(pim + i);
  __syncthreads();
  const int G = C / 2;
  const double inv = 1.0 / HW;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    double m[2], M2[2];
    for (int j = 0; j < 2; ++j) {
      const int c = 2 * g + j;
      double a = 0.0, b = 0.0;
      for (int t = 0; t < S; ++t) {
        a += (double)sh[(t * C + c) * 2];
        b += (double)sh[(t * C + c) * 2 + 1];
      }
      m[j] = (double)zi[c] + a * inv;   // the same shift every block used
      M2[j] = b - a * a * inv;
    }
    const double dm = m[0] - m[1];
    double var = (M2[0] + M2[1] + 0.5 * HW * dm * dm) / (2.0 * HW);
    if (var < 0.0) var = 0.0;
    mean[g] = (float)(0.5 * (m[0] + m[1]));
    rstd[g] = 1.0f / sqrtf((float)var + eps);
  }
}

template <int V>
__global__ void __launch_bounds__(kThreads) gn_stats_kernel(const float* __restrict__ z, int HW, int C,
                                                            int S, float eps, float* __restrict__ part,
                                                            int* __restrict__ cnt, float* __restrict__ mean,
                                                            float* __restrict__ rstd) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  __shared__ int flag;
  const int n = blockIdx.y, sb = blockIdx.x;
  const int chunk = (HW + S - 1) / S, pb = sb * chunk, pe = min(HW, pb + chunk);
  const float* zi = z + (size_t)n * HW * C;
  block_shifted_sums<V>(zi, pb, pe, C, sh, part + ((size_t)n * S + sb) * C * 2);
  if (!last_of_image(cnt + n, S, &flag)) return;
  const int G = C / 2;
  combine_groups(part + (size_t)n * S * C * 2, zi, S, C, HW, eps, sh, mean + (size_t)n * G,
                 rstd + (size_t)n * G);
  if (threadIdx.x == 0) cnt[n] = 0;  // re-arm for the next launch on this stream
}

// ---- out = act(gn(z) + res) ----
// one vector of V channels at element offset o (channel c0) of image n; mu/rs (and mud/rsd)
// point at the group statistics of channel c0 (group c0 / 2); returns max |out| (E4M3 copy)
template <int V>
__device__ __forceinline__ float apply_vec(const GNApply& a, size_t o, int c0, const float* mu,
                                           const float* rs, const float* mud, const float* rsd,
                                           float f8s) {
  float x[V], gm[V], bt[V];
  ldv<V>(a.z + o, x);
  ldv<V>(a.gamma + c0, gm);
  ldv<V>(a.beta + c0, bt);
#pragma unroll
  for (int v = 0; v < V; ++v) x[v] = (x[v] - mu[v / 2]) * rs[v / 2] * gm[v] + bt[v];
  if (a.resid) {
    float r[V];
    ldv<V>(a.resid + o, r);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] += r[v];
  }
  if (a.zd) {
    float d[V], gd[V], bd[V];
    ldv<V>(a.zd + o, d);
    ldv<V>(a.gamma_d + c0, gd);
    ldv<V>(a.beta_d + c0, bd);
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] += (d[v] - mud[v / 2]) * rsd[v / 2] * gd[v] + bd[v];
  }
  if (a.relu) {
#pragma unroll
    for (int v = 0; v < V; ++v) x[v] = fmaxf(x[v], 0.f);
  }
  if (a.out) stv<V>(a.out + o, x);
  if (a.out_bf) stv_bf<V>(a.out_bf + o, x);
  float f8m = 0.f;
  if (a.out_f8) {
    stv_e4m3<V>(a.out_f8 + o, x, f8s);
#pragma unroll
    for (int v = 0; v < V; ++v) f8m = fmaxf(f8m, fabsf(x[v]));
  }
  return f8m;
}

template <int V>
__global__ void __launch_bounds__(kThreads) gn_apply_kernel(GNApply a, int HW, int C) {
  DDPPO_PDL_ENTRY();
  const int R = C / V, G = C / 2;
  const int n = blockIdx.y;
  const int per = HW * R;
  const size_t ib = (size_t)n * HW * C;
  const float f8s = a.out_f8 ? *a.f8_scale : 1.f;
  float f8m = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
    const int c0 = (i % R) * V;
    const size_t gq = (size_t)n * G + c0 / 2;
    const float* mud = a.zd ? a.mean_d + gq : nullptr;
    const float* rsd = a.zd ? a.rstd_d + gq : nullptr;
    f8m = fmaxf(f8m, apply_vec<V>(a, ib + (size_t)i * V, c0, a.mean + gq, a.rstd + gq, mud, rsd, f8s));
  }
  if (a.out_f8) block_amax(f8m, a.f8_amax);
}

// ---- statistics and normalisation in one launch ----
// Every block of the (S, N) grid is resident (cooperative launch). Each block sums its
// pixel rows as the statistics kernel does (z, and zd when present); the S blocks of an
// image then meet at a per-image barrier: an arrival counter, and a departure counter
// whose last increment re-arms both for the next launch. The wait is bounded: on a
// run-out the sticky timeout flag is set and the block returns without writing. After
// the barrier each block combines the image's partials in block order exactly as the
// statistics kernel's last block does (so the statistics are bit-identical for the same
// S), block 0 of the image stores them for the backward, and every block normalises the
// rows it just summed (still in L2): z is read from HBM once, and one launch replaces two.
constexpr unsigned GN_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ bool image_barrier(int* arrive, int* depart, int S, int32_t* err,
                                              int* s_ok) {
  __threadfence();  // this thread's partial sums are visible device-wide before the arrival
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(arrive, 1);
    int ok = 0;
    for (unsigned i = 0; i < GN_SPIN_LIMIT; ++i) {
      if (*(volatile int*)arrive >= S) { ok = 1; break; }
      if (err && (*(volatile int32_t*)err & ERRF_TIMEOUT)) break;
      __nanosleep(64);
    }
    if (!ok && err) atomicOr(err, ERRF_TIMEOUT);
    __threadfence();
    // every block has stopped reading `arrive` once the departures reach S
    if (atomicAdd(depart, 1) == S - 1) {
      atomicExch(arrive, 0);
      atomicExch(depart, 0);
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

template <int V>
__global__ void __launch_bounds__(kThreads) gn_fused_kernel(GNApply a, int HW, int C, int S, float eps,
                                                            float* __restrict__ part,
                                                            float* __restrict__ part_d, int* arrive,
                                                            int* depart, int32_t* err) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  __shared__ int s_ok;
  const int n = blockIdx.y, sb = blockIdx.x, G = C / 2;
  const int chunk = (HW + S - 1) / S, pb = sb * chunk, pe = min(HW, pb + chunk);
  const size_t ib = (size_t)n * HW * C;
  float* st = sh + max((int)blockDim.x * 2 * V, S * C * 2);  // [4][G]: mean, rstd, mean_d, rstd_d
  block_shifted_sums<V>(a.z + ib, pb, pe, C, sh, part + ((size_t)n * S + sb) * C * 2);
  if (a.zd) {
    __syncthreads();
    block_shifted_sums<V>(a.zd + ib, pb, pe, C, sh, part_d + ((size_t)n * S + sb) * C * 2);
  }
  if (!image_barrier(arrive + n, depart + n, S, err, &s_ok)) return;
  combine_groups(part + (size_t)n * S * C * 2, a.z + ib, S, C, HW, eps, sh, st, st + G);
  if (a.zd) {
    __syncthreads();
    combine_groups(part_d + (size_t)n * S * C * 2, a.zd + ib, S, C, HW, eps, sh, st + 2 * G,
                   st + 3 * G);
  }
  __syncthreads();
  if (sb == 0) {
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      const_cast<float*>(a.mean)[(size_t)n * G + g] = st[g];
      const_cast<float*>(a.rstd)[(size_t)n * G + g] = st[G + g];
      if (a.zd) {
        const_cast<float*>(a.mean_d)[(size_t)n * G + g] = st[2 * G + g];
        const_cast<float*>(a.rstd_d)[(size_t)n * G + g] = st[3 * G + g];
      }
    }
  }
  const int R = C / V, P = blockDim.x / R;
  const int cv = threadIdx.x % R, pr = threadIdx.x / R, c0 = cv * V;
  const float f8s = a.out_f8 ? *a.f8_scale : 1.f;
  float f8m = 0.f;
  for (int p = pb + pr; p < pe; p += P)
    f8m = fmaxf(f8m, apply_vec<V>(a, ib + (size_t)p * C + c0, c0, st + c0 / 2, st + G + c0 / 2,
                                  st + 2 * G + c0 / 2, st + 3 * G + c0 / 2, f8s));
  if (a.out_f8) block_amax(f8m, a.f8_amax);
}

// ---- one block per image: statistics and normalisation without any grid barrier ----
// The block sums the whole image (the statistics kernel's S = 1 arithmetic), combines in
// shared memory, and normalises the image it just read (an L2 hit). An ordinary launch:
// nothing waits on another block, so it needs no co-residency.
__device__ __forceinline__ void combine_groups_one(const float* p, const float* __restrict__ zi,
                                                   int C, int HW, float eps, float* mean,
                                                   float* rstd) {
  const int G = C / 2;
  const double inv = 1.0 / HW;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    double m[2], M2[2];
    for (int j = 0; j < 2; ++j) {
      const int c = 2 * g + j;
      const double a = 0.0 + (double)p[c * 2], b = 0.0 + (double)p[c * 2 + 1];
      m[j] = (double)zi[c] + a * inv;
      M2[j] = b - a * a * inv;
    }
    const double dm = m[0] - m[1];
    double var = (M2[0] + M2[1] + 0.5 * HW * dm * dm) / (2.0 * HW);
    if (var < 0.0) var = 0.0;
    mean[g] = (float)(0.5 * (m[0] + m[1]));
    rstd[g] = 1.0f / sqrtf((float)var + eps);
  }
}

template <int V>
__global__ void __launch_bounds__(kThreads) gn_image_kernel(GNApply a, int HW, int C, float eps) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  const int n = blockIdx.x, G = C / 2;
  const size_t ib = (size_t)n * HW * C;
  float* pz = sh + (int)blockDim.x * 2 * V;  // [C][2] partial sums of z, then of zd
  float* pd = pz + 2 * C;
  float* st = pd + 2 * C;                    // [4][G]: mean, rstd, mean_d, rstd_d
  block_shifted_sums<V>(a.z + ib, 0, HW, C, sh, pz);
  if (a.zd) {
    __syncthreads();
    block_shifted_sums<V>(a.zd + ib, 0, HW, C, sh, pd);
  }
  __syncthreads();
  combine_groups_one(pz, a.z + ib, C, HW, eps, st, st + G);
  if (a.zd) combine_groups_one(pd, a.zd + ib, C, HW, eps, st + 2 * G, st + 3 * G);
  __syncthreads();
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const_cast<float*>(a.mean)[(size_t)n * G + g] = st[g];
    const_cast<float*>(a.rstd)[(size_t)n * G + g] = st[G + g];
    if (a.zd) {
      const_cast<float*>(a.mean_d)[(size_t)n * G + g] = st[2 * G + g];
      const_cast<float*>(a.rstd_d)[(size_t)n * G + g] = st[3 * G + g];
    }
  }
  const int R = C / V, P = blockDim.x / R;
  const int cv = threadIdx.x % R, pr = threadIdx.x / R, c0 = cv * V;
  const float f8s = a.out_f8 ? *a.f8_scale : 1.f;
  float f8m = 0.f;
#pragma unroll 4
  for (int p = pr; p < HW; p += P)
    f8m = fmaxf(f8m, apply_vec<V>(a, ib + (size_t)p * C + c0, c0, st + c0 / 2, st + G + c0 / 2,
                                  st + 2 * G + c0 / 2, st + 3 * G + c0 / 2, f8s));
  if (a.out_f8) block_amax(f8m, a.f8_amax);
}

// ---- backward reductions: g = dy (masked by relu_y > 0), xhat = (z - mu) rstd;
//      per image and channel sum(g) and sum(g xhat); group means of gamma-weighted sums ----
template <int V>
__global__ void __launch_bounds__(kThreads) gn_bwd_reduce_kernel(GNBack b, int HW, int C, int S,
                                                                 float* __restrict__ part,
                                                                 int* __restrict__ cnt) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  __shared__ int flag;
  const int R = C / V, P = blockDim.x / R, G = C / 2;
  const int n = blockIdx.y, sb = blockIdx.x;
  const int cv = threadIdx.x % R, pr = threadIdx.x / R, c0 = cv * V;
  const int chunk = (HW + S - 1) / S, pb = sb * chunk, pe = min(HW, pb + chunk);
  const size_t ib = (size_t)n * HW * C;
  float mu[V], rs[V], sg[V], sgx[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    mu[v] = b.mean[(size_t)n * G + (c0 + v) / 2];
    rs[v] = b.rstd[(size_t)n * G + (c0 + v) / 2];
    sg[v] = sgx[v] = 0.f;
  }
#pragma unroll 8
  for (int p = pb + pr; p < pe; p += P) {
    const size_t o = ib + (size_t)p * C + c0;
    float d[V], x[V];
    ldv<V>(b.z + o, x);
    ldv<V>(b.dy + o, d);
    if (b.relu_from_z) {
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (!((x[v] - mu[v]) * rs[v] * b.gamma[c0 + v] + b.beta[c0 + v] > 0.f)) d[v] = 0.f;
    }
    if (b.relu_y) {
      float y[V];
      ldv<V>(b.relu_y + o, y);
#pragma unroll
      for (int v = 0; v < V; ++v) d[v] = y[v] > 0.f ? d[v] : 0.f;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sg[v] += d[v];
      sgx[v] += d[v] * ((x[v] - mu[v]) * rs[v]);
    }
  }
  float* pp = part + ((size_t)n * S + sb) * C * 2;
  block_pair_sums<V>(sg, sgx, sh, C, pp);
  if (!last_of_image(cnt + n, S, &flag)) return;
  // per-channel totals (block order), then the group means of gamma-weighted sums
  const float* pim = part + (size_t)n * S * C * 2;
  for (int i = threadIdx.x; i < S * C * 2; i += blockDim.x) sh[i] = __ldcg(pim + i);
  __syncthreads();
  float* tot = sh + S * C * 2;  // [C][2]
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float a = 0.f, e = 0.f;
    for (int t = 0; t < S; ++t) {
      a += sh[(t * C + c) * 2];
      e += sh[(t * C + c) * 2 + 1];
    }
    tot[2 * c] = a;
    tot[2 * c + 1] = e;
    b.dbeta_part[(size_t)n * C + c] = a;
    b.dgamma_part[(size_t)n * C + c] = e;
  }
  __syncthreads();
  const float inv = 1.0f / (float)(2 * HW);
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const float g0 = b.gamma[2 * g], g1 = b.gamma[2 * g + 1];
    b.m1[(size_t)n * G + g] = (tot[4 * g] * g0 + tot[4 * g + 2] * g1) * inv;
    b.m2[(size_t)n * G + g] = (tot[4 * g + 1] * g0 + tot[4 * g + 3] * g1) * inv;
  }
  if (threadIdx.x == 0) cnt[n] = 0;
}

// ---- dz = rstd (g gamma - m1 - xhat m2); optionally g itself (the masked gradient) ----
template <int V>
__global__ void __launch_bounds__(kThreads) gn_bwd_apply_kernel(GNBack b, int HW, int C) {
  DDPPO_PDL_ENTRY();
  const int R = C / V, G = C / 2;
  const int n = blockIdx.y;
  const int per = HW * R;
  const size_t ib = (size_t)n * HW * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
    const int c0 = (i % R) * V;
    const size_t o = ib + (size_t)i * V;
    float d[V], x[V], gm[V], r[V];
    ldv<V>(b.z + o, x);
    ldv<V>(b.gamma + c0, gm);
    ldv<V>(b.dy + o, d);
    if (b.relu_from_z) {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const size_t gq = (size_t)n * G + (c0 + v) / 2;
        if (!((x[v] - b.mean[gq]) * b.rstd[gq] * gm[v] + b.beta[c0 + v] > 0.f)) d[v] = 0.f;
      }
    }
    if (b.relu_y) {
      float y[V];
      ldv<V>(b.relu_y + o, y);
#pragma unroll
      for (int v = 0; v < V; ++v) d[v] = y[v] > 0.f ? d[v] : 0.f;
      if (b.g_out) stv<V>(b.g_out + o, d);
    }
    const size_t gi = (size_t)n * G + c0 / 2;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const float mu = b.mean[gi + v / 2], rs = b.rstd[gi + v / 2];
      const float xh = (x[v] - mu) * rs;
      r[v] = rs * (d[v] * gm[v] - b.m1[gi + v / 2] - xh * b.m2[gi + v / 2]);
    }
    if (b.dz32) stv<V>(b.dz32 + o, r);
    if (b.dzop) stv_op<V>(b.dzop, o, r, b.op_bf16);
  }
}

// ---- backward, one block per image: the reduction (the reduce kernel's S = 1 arithmetic),
//      the group means in shared memory, then the input gradient of the image just read ----
template <int V>
__global__ void __launch_bounds__(kThreads) gn_bwd_image_kernel(GNBack b, int HW, int C) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  const int R = C / V, P = blockDim.x / R, G = C / 2;
  const int n = blockIdx.x;
  const int cv = threadIdx.x % R, pr = threadIdx.x / R, c0 = cv * V;
  const size_t ib = (size_t)n * HW * C;
  float* part = sh + blockDim.x * 2 * V;  // [C][2]: sum g, sum g xhat
  float* m12 = part + 2 * C;              // [2][G]: m1, m2
  float mu[V], rs[V], sg[V], sgx[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    mu[v] = b.mean[(size_t)n * G + (c0 + v) / 2];
    rs[v] = b.rstd[(size_t)n * G + (c0 + v) / 2];
    sg[v] = sgx[v] = 0.f;
  }
#pragma unroll 8
  for (int p = pr; p < HW; p += P) {
    const size_t o = ib + (size_t)p * C + c0;
    float d[V], x[V];
    ldv<V>(b.z + o, x);
    ldv<V>(b.dy + o, d);
    if (b.relu_from_z) {
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (!((x[v] - mu[v]) * rs[v] * b.gamma[c0 + v] + b.beta[c0 + v] > 0.f)) d[v] = 0.f;
    }
    if (b.relu_y) {
      float y[V];
      ldv<V>(b.relu_y + o, y);
#pragma unroll
      for (int v = 0; v < V; ++v) d[v] = y[v] > 0.f ? d[v] : 0.f;
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      sg[v] += d[v];
      sgx[v] += d[v] * ((x[v] - mu[v]) * rs[v]);
    }
  }
  block_pair_sums<V>(sg, sgx, sh, C, part);
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    b.dbeta_part[(size_t)n * C + c] = 0.f + part[2 * c];
    b.dgamma_part[(size_t)n * C + c] = 0.f + part[2 * c + 1];
  }
  const float inv = 1.0f / (float)(2 * HW);
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    const float g0 = b.gamma[2 * g], g1 = b.gamma[2 * g + 1];
    const float t0 = 0.f + part[4 * g], t1 = 0.f + part[4 * g + 1];
    const float t2 = 0.f + part[4 * g + 2], t3 = 0.f + part[4 * g + 3];
    m12[g] = (t0 * g0 + t2 * g1) * inv;
    m12[G + g] = (t1 * g0 + t3 * g1) * inv;
  }
  __syncthreads();
  float gm[V];
  ldv<V>(b.gamma + c0, gm);
#pragma unroll 4
  for (int p = pr; p < HW; p += P) {
    const size_t o = ib + (size_t)p * C + c0;
    float d[V], x[V], r[V];
    ldv<V>(b.z + o, x);
    ldv<V>(b.dy + o, d);
    if (b.relu_from_z) {
#pragma unroll
      for (int v = 0; v < V; ++v)
        if (!((x[v] - mu[v]) * rs[v] * gm[v] + b.beta[c0 + v] > 0.f)) d[v] = 0.f;
    }
    if (b.relu_y) {
      float y[V];
      ldv<V>(b.relu_y + o, y);
#pragma unroll
      for (int v = 0; v < V; ++v) d[v] = y[v] > 0.f ? d[v] : 0.f;
      if (b.g_out) stv<V>(b.g_out + o, d);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int g = (c0 + v) / 2;
      const float xh = (x[v] - mu[v]) * rs[v];
      r[v] = rs[v] * (d[v] * gm[v] - m12[g] - xh * m12[G + g]);
    }
    if (b.dz32) stv<V>(b.dz32 + o, r);
    if (b.dzop) stv_op<V>(b.dzop, o, r, b.op_bf16);
  }
}

int num_sms_cached() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      sms = 1;
  }
  return sms;
}

bool gn_shape_ok(int C) { return C >= 2 && C % 2 == 0 && C / (C % 4 == 0 ? 4 : 2) <= kThreads; }

// blocks per image: enough for ~8 blocks per SM overall, at least one pixel pass each
int gn_split(int N, int HW, int C, const GnScratch& w) {
  // images of at most 32K elements (128 KB): one block each -- a block sums such an image
  // faster than S blocks combine their partials (measured: the 64-image act batch); and any
  // image size once there are at least 4 images per SM (one block each already fills the GPU)
  if ((long)HW * C <= 32768 || N >= 4 * num_sms_cached()) return 1;
  const int V = C % 4 == 0 ? 4 : 2;
  const int P = rows_per_pass(C, V);
  const int want = (8 * num_sms_cached() + N - 1) / N;
  int S = std::min(want, (HW + P - 1) / P);
  S = std::min(S, 64);
  S = std::min(S, std::max(1, 4096 / C));  // the combine stages S x C x 2 floats in shared memory
  S = std::max(S, 1);
  while (S > 1 && (size_t)N * S * C * 2 > w.part_elems) --S;
  return S;
}

unsigned apply_blocks(int N, int HW, int C, int V) {
  const long per = (long)HW * (C / V);
  const int want = (8 * num_sms_cached() + N - 1) / N;
  long bx = (per + kThreads - 1) / kThreads;
  bx = std::min<long>(bx, std::max(want, 1));
  return (unsigned)std::max<long>(bx, 1);
}

int threads_for(int C, int V) {
  const int R = C / V;
  return R * rows_per_pass(C, V);
}

}  // namespace

size_t gn_part_elems(int max_images, int max_C) {
  return (size_t)(max_images + 8 * num_sms_cached() + 64) * max_C * 2;
}

// dynamic shared memory of the one-launch kernel for S blocks per image
static size_t fused_smem(int S, int C, int V) {
  const int th = threads_for(C, V);
  return ((size_t)std::max(th * 2 * V, S * C * 2) + 2 * (size_t)C) * sizeof(float);
}

// blocks per image of the one-launch form: gn_split's choice, lowered until all S x N
// blocks are resident at once; 0 when even S = 1 is not (the two-launch form then keeps
// gn_split's choice). The statistics launch of the two-launch form uses the same S, so
// the two forms give bit-identical statistics.
static int gn_split_one_launch(int N, int HW, int C, const GnScratch& w) {
  if (!w.cnt2) return 0;
  const int V = C % 4 == 0 ? 4 : 2;
  void (*kern)(GNApply, int, int, int, float, float*, float*, int*, int*, int32_t*) =
      V == 4 ? gn_fused_kernel<4> : gn_fused_kernel<2>;
  const int th = threads_for(C, V);
  const int sms = num_sms_cached();
  for (int S = gn_split(N, HW, C, w); S >= 1; --S) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, th, fused_smem(S, C, V)) != cudaSuccess)
      return 0;
    if ((long)S * N <= (long)occ * sms) return S;
  }
  return 0;
}

int launch_gn_stats(const float* z, int N, int HW, int C, float eps, float* mean, float* rstd,
                    const GnScratch& w, cudaStream_t s) {
  if (!N || !HW) return DDPPO_OK;
  if (!gn_shape_ok(C) || N > w.max_images || N > 65535) {
    set_error("gn: unsupported channel count or too many images for the scratch");
    return DDPPO_E_CONFIG;
  }
  const int V = C % 4 == 0 ? 4 : 2;
  const int S1 = gn_split_one_launch(N, HW, C, w);
  const int S = S1 ? S1 : gn_split(N, HW, C, w);
  const int th = threads_for(C, V);
  const size_t smem = std::max((size_t)th * 2 * V, (size_t)S * C * 2) * sizeof(float);
  const dim3 grid(S, N);
  if (V == 4) ::ddppo::launch_k(gn_stats_kernel<4>, grid, th, smem, s, z, HW, C, S, eps, w.part, w.cnt, mean, rstd);
  else ::ddppo::launch_k(gn_stats_kernel<2>, grid, th, smem, s, z, HW, C, S, eps, w.part, w.cnt, mean, rstd);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_gn_fused(const GNApply& a, int N, int HW, int C, float eps, const GnScratch& w,
                    int32_t* err, cudaStream_t s, bool* launched) {
  *launched = false;
  if (!N || !HW) { *launched = true; return DDPPO_OK; }
  if (!w.cnt2 || !gn_shape_ok(C) || N > w.max_images || N > 65535) return DDPPO_OK;
  const int V = C % 4 == 0 ? 4 : 2;
  const int th = threads_for(C, V);
  void (*kern)(GNApply, int, int, int, float, float*, float*, int*, int*, int32_t*) =
      V == 4 ? gn_fused_kernel<4> : gn_fused_kernel<2>;
  const int nt = a.zd ? 2 : 1;
  if (gn_split(N, HW, C, w) == 1) {
    // one block per image. With many images (at least 4 per SM: the update's minibatches)
    // one launch, whose blocks normalise the image they just summed (re-read from L2);
    // with few (the 64-image act batch) the statistics launch then a normalise launch that
    // spreads each image over many blocks, which measured faster there
    if (N < 4 * num_sms_cached()) return DDPPO_OK;
    const size_t smem = ((size_t)th * 2 * V + 6 * (size_t)C) * sizeof(float);
    if (V == 4) ::ddppo::launch_k(gn_image_kernel<4>, N, th, smem, s, a, HW, C, eps);
    else ::ddppo::launch_k(gn_image_kernel<2>, N, th, smem, s, a, HW, C, eps);
    DDPPO_CHECK_LAUNCH();
    *launched = true;
    return DDPPO_OK;
  }
  // every block resident at once, and the partials of z (and zd) in the scratch;
  // otherwise two launches
  const int S = gn_split_one_launch(N, HW, C, w);
  if (S < 1 || (size_t)nt * N * S * C * 2 > w.part_elems) return DDPPO_OK;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(S, N);
  cfg.blockDim = dim3(th);
  cfg.dynamicSmemBytes = fused_smem(S, C, V);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  float* part_d = w.part + (size_t)N * S * C * 2;
  DDPPO_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, a, HW, C, S, eps, w.part, part_d, w.cnt, w.cnt2, err));
  *launched = true;
  return DDPPO_OK;
}

int launch_gn_apply(const GNApply& a, int N, int HW, int C, cudaStream_t s) {
  if (!N || !HW) return DDPPO_OK;
  if (!gn_shape_ok(C) || N > 65535) { set_error("gn: unsupported shape"); return DDPPO_E_CONFIG; }
  const int V = C % 4 == 0 ? 4 : 2;
  const dim3 grid(apply_blocks(N, HW, C, V), N);
  if (V == 4) ::ddppo::launch_k(gn_apply_kernel<4>, grid, kThreads, 0, s, a, HW, C);
  else ::ddppo::launch_k(gn_apply_kernel<2>, grid, kThreads, 0, s, a, HW, C);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_gn_bwd(const GNBack& b, int N, int HW, int C, const GnScratch& w, cudaStream_t s) {
  if (!N || !HW) return DDPPO_OK;
  if (!gn_shape_ok(C) || N > w.max_images || N > 65535) {
    set_error("gn: unsupported channel count or too many images for the scratch");
    return DDPPO_E_CONFIG;
  }
  const int V = C % 4 == 0 ? 4 : 2;
  const int S = gn_split(N, HW, C, w);
  const int th = threads_for(C, V);
  if (S == 1 && N >= 4 * num_sms_cached()) {
    // many small images: one block per image, reduction and input gradient in one launch
    const size_t smem1 = ((size_t)th * 2 * V + 3 * (size_t)C) * sizeof(float);
    if (V == 4) ::ddppo::launch_k(gn_bwd_image_kernel<4>, N, th, smem1, s, b, HW, C);
    else ::ddppo::launch_k(gn_bwd_image_kernel<2>, N, th, smem1, s, b, HW, C);
    DDPPO_CHECK_LAUNCH();
    return DDPPO_OK;
  }
  const size_t smem = std::max((size_t)th * 2 * V, (size_t)(S + 1) * C * 2) * sizeof(float);
  const dim3 grid(S, N);
  if (V == 4) ::ddppo::launch_k(gn_bwd_reduce_kernel<4>, grid, th, smem, s, b, HW, C, S, w.part, w.cnt);
  else ::ddppo::launch_k(gn_bwd_reduce_kernel<2>, grid, th, smem, s, b, HW, C, S, w.part, w.cnt);
  DDPPO_CHECK_LAUNCH();
  const dim3 ga(apply_blocks(N, HW, C, V), N);
  if (V == 4) ::ddppo::launch_k(gn_bwd_apply_kernel<4>, ga, kThreads, 0, s, b, HW, C);
  else ::ddppo::launch_k(gn_bwd_apply_kernel<2>, ga, kThreads, 0, s, b, HW, C);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- GroupNorm apply + ReLU + 3x3 / stride-2 / pad-1 max pool (4 channels per thread) ----
__global__ void __launch_bounds__(kThreads) gn_relu_maxpool_kernel(GNApply a, int H, int W, int C,
                                                                   float* __restrict__ pool,
                                                                   __nv_bfloat16* __restrict__ pool_bf,
                                                                   uint8_t* __restrict__ arg) {
  DDPPO_PDL_ENTRY();
  const int Hq = (H - 1) / 2 + 1, Wq = (W - 1) / 2 + 1, C4 = C / 4, G = C / 2;
  const int n = blockIdx.y, per = Hq * Wq * C4;
  const float* zi = a.z + (size_t)n * H * W * C;
  const float f8s = a.out_f8 ? *a.f8_scale : 1.f;
  float f8m = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
    const int c4 = i % C4, pix = i / C4, c0 = c4 * 4;
    const int ox = pix % Wq, oy = pix / Wq;
    float gm[4], bt[4], mu[4], rs[4];
    ldv<4>(a.gamma + c0, gm);
    ldv<4>(a.beta + c0, bt);
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      mu[v] = a.mean[(size_t)n * G + (c0 + v) / 2];
      rs[v] = a.rstd[(size_t)n * G + (c0 + v) / 2];
    }
    float best[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
    int bi[4] = {0, 0, 0, 0};
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = oy * 2 - 1 + ky;
      if (iy < 0 || iy >= H) continue;
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = ox * 2 - 1 + kx;
        if (ix < 0 || ix >= W) continue;
        float x[4];
        ldv<4>(zi + ((size_t)iy * W + ix) * C + c0, x);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float y = fmaxf((x[v] - mu[v]) * rs[v] * gm[v] + bt[v], 0.f);
          if (y > best[v]) { best[v] = y; bi[v] = ky * 3 + kx; }
        }
      }
    }
    const size_t o = (size_t)n * per * 4 + (size_t)i * 4;
    stv<4>(pool + o, best);
    if (pool_bf) stv_bf<4>(pool_bf + o, best);
    if (a.out_f8) {
      stv_e4m3<4>(a.out_f8 + o, best, f8s);
#pragma unroll
      for (int v = 0; v < 4; ++v) f8m = fmaxf(f8m, best[v]);
    }
    *reinterpret_cast<uchar4*>(arg + o) = make_uchar4(bi[0], bi[1], bi[2], bi[3]);
  }
  if (a.out_f8) block_amax(f8m, a.f8_amax);
}

int launch_gn_relu_maxpool(const GNApply& a, int N, int H, int W, int C, float* pool,
                           __nv_bfloat16* pool_bf, uint8_t* arg, cudaStream_t s) {
  if (!N) return DDPPO_OK;
  const int Hq = (H - 1) / 2 + 1, Wq = (W - 1) / 2 + 1;
  if (C % 4 || N > 65535 || (int64_t)Hq * Wq * C >= (1ll << 31)) {
    set_error("gn_relu_maxpool: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  const long per = (long)Hq * Wq * (C / 4);
  const dim3 gb((unsigned)std::max<long>(1, std::min<long>((per + kThreads - 1) / kThreads,
                                                           (8l * num_sms_cached() + N - 1) / N)),
                N);
  ::ddppo::launch_k(gn_relu_maxpool_kernel, gb, kThreads, 0, s, a, H, W, C, pool, pool_bf, arg);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
