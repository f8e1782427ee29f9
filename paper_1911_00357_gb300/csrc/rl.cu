// Learning-step kernels: the PPO clipped-surrogate loss (Eq. 2) with value and entropy
// terms fused with its exact gradient, the global gradient norm, Adam (Kingma & Ba 2015),
// the per-epoch env permutation for minibatches, and the optional advantage
// normalisation. Every reduction is block partials followed by one fixed-order pass.
#include "rl.cuh"

namespace ddppo {

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block reduction of NV values per thread into part[blockIdx.x * NV + k] (256 threads)
template <int NV>
__device__ void block_partials(float (&v)[NV], float* part) {
  __shared__ float sh[NV][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const float s = wsum(v[k]);
    if (lane == 0) sh[k][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    float s = 0.f;
    for (int q = 0; q < 8; ++q) s += sh[threadIdx.x][q];
    part[blockIdx.x * NV + threadIdx.x] = s;
  }
}

// per sample i:
//   logp = log_softmax(logits)[a], rho = exp(logp - logp_old)
//   pol_i = -min(rho A, clip(rho) A); v_i = 0.5 (R - V)^2; H_i = -sum p log p
//   d logp = -rho A when the unclipped term is the active minimum (ties split evenly
//   between the two branches, which sum to the same when rho is inside the clip range)
//   dlogits_j = [dlogp (1[j=a] - p_j) + c_e p_j (log p_j + H_i)] / n ; dV = c_v (V - R) / n
__global__ void __launch_bounds__(256) ppo_loss_kernel(int n, const float* __restrict__ logits,
                                                       const float* __restrict__ values,
                                                       const int32_t* __restrict__ actions,
                                                       const float* __restrict__ logp_old,
                                                       const float* __restrict__ adv,
                                                       const float* __restrict__ ret, float clip,
                                                       float cv, float ce, float* dlogits,
                                                       float* dvalues, float* part) {
  DDPPO_PDL_ENTRY();
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float lg[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) lg[q] = logits[(size_t)i * 4 + q];
    const float mx = fmaxf(fmaxf(lg[0], lg[1]), fmaxf(lg[2], lg[3]));
    float z = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) z += expf(lg[q] - mx);
    const float lse = mx + logf(z);
    float lp[4], p[4], H = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lp[q] = lg[q] - lse;
      p[q] = expf(lp[q]);
      H -= p[q] * lp[q];
    }
    int a = actions[i];
    a = a < 0 ? 0 : (a > 3 ? 3 : a);
    const float A = adv[i];
    const float rho = expf(lp[a] - logp_old[i]);
    const float s1 = rho * A;
    const float rc = fminf(fmaxf(rho, 1.f - clip), 1.f + clip);
    const float s2 = rc * A;
    const bool inside = rho >= 1.f - clip && rho <= 1.f + clip;
    const float dlp = (inside || s1 < s2) ? -rho * A : 0.f;
    const float V = values[i], R = ret[i];
    const float inv = 1.0f / (float)n;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      dlogits[(size_t)i * 4 + q] = inv * (dlp * ((q == a ? 1.f : 0.f) - p[q]) + ce * p[q] * (lp[q] + H));
    dvalues[i] = inv * cv * (V - R);
    acc[0] += -fminf(s1, s2);
    acc[1] += 0.5f * (R - V) * (R - V);
    acc[2] += H;
    acc[3] += fabsf(rho - 1.f) > clip ? 1.f : 0.f;
    acc[4] += logp_old[i] - lp[a];
  }
  block_partials<5>(acc, part);
}

// the sum over nb blocks of NV partials each (part[b * NV + k]) by one block of kFinal
// threads, in a fixed order: thread i adds partials i, i + kFinal, ... in turn, then a fixed
// halving tree over the threads. Every thread reads its partials before the first barrier.
constexpr int kFinal = 256;
template <int NV>
__device__ void final_sums(const float* part, int nb, float (&out)[NV]) {
  __shared__ float sh[NV][kFinal];
  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.f;
  for (int b = threadIdx.x; b < nb; b += kFinal)
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += part[b * NV + k];
#pragma unroll
  for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kFinal / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
#pragma unroll
      for (int k = 0; k < NV; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < NV; ++k) out[k] = sh[k][0];
}

__global__ void __launch_bounds__(kFinal) ppo_loss_final(int nb, int n, const float* part, float cv,
                                                        float ce, float* stats) {
  DDPPO_PDL_ENTRY();
  float s[5];
  final_sums<5>(part, nb, s);  // part may alias stats: all reads precede the writes below
  if (threadIdx.x != 0) return;
  const float inv = 1.0f / (float)n;
  const float pol = s[0] * inv, vl = s[1] * inv, ent = s[2] * inv;
  stats[0] = pol + cv * vl - ce * ent;
  stats[1] = pol;
  stats[2] = vl;
  stats[3] = ent;
  stats[4] = s[3] * inv;
  stats[5] = s[4] * inv;
  stats[6] = 0.f;
  stats[7] = 0.f;
}

int launch_ppo_loss(int n, const float* logits, const float* values, const int32_t* actions,
                    const float* logp_old, const float* adv, const float* ret, float clip, float cv,
                    float ce, float* stats, float* dlogits, float* dvalues, float* part,
                    size_t part_elems, cudaStream_t s) {
  if (n <= 0) return DDPPO_OK;
  // without scratch one block covers all samples and reduces into stats itself
  int nb = part ? (n + 255) / 256 : 1;
  if (nb > 1024) nb = 1024;
  if (!part) part = stats;
  else if ((size_t)nb * 5 > part_elems) { set_error("ppo_loss: scratch too small"); return DDPPO_E_CONFIG; }
  ::ddppo::launch_k(ppo_loss_kernel, nb, 256, 0, s, n, logits, values, actions, logp_old, adv, ret, clip, cv, ce,
                                     dlogits, dvalues, part);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(ppo_loss_final, 1, kFinal, 0, s, nb, n, part, cv, ce, stats);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

int launch_ppo_loss_blocks(int n, const float* logits, const float* values, const int32_t* actions,
                           const float* logp_old, const float* adv, const float* ret, float clip,
                           float cv, float ce, float* stats, float* dlogits, float* dvalues,
                           float* part, int nb, cudaStream_t s) {
  if (n <= 0) return DDPPO_OK;
  ::ddppo::launch_k(ppo_loss_kernel, nb, 256, 0, s, n, logits, values, actions, logp_old, adv, ret, clip, cv, ce,
                                     dlogits, dvalues, part);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(ppo_loss_final, 1, kFinal, 0, s, nb, n, part, cv, ce, stats);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- sum of squares / sums, two-stage ----
__global__ void __launch_bounds__(256) sumsq_partial(const float* __restrict__ x, size_t n,
                                                     float* part, int square, const float* shift) {
  DDPPO_PDL_ENTRY();
  float v[1] = {0.f};
  const float mu = shift ? shift[0] : 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = x[i] - mu;
    v[0] += square ? d * d : d;
  }
  block_partials<1>(v, part);
}
__global__ void __launch_bounds__(kFinal) sum_final(int nb, const float* __restrict__ part, float* out,
                                                   int mode, float scale) {
  DDPPO_PDL_ENTRY();
  float t[1];
  final_sums<1>(part, nb, t);
  if (threadIdx.x != 0) return;
  const float s = t[0];
  if (mode == 0) out[0] = sqrtf(s);          // L2 norm
  else if (mode == 1) out[0] = s * scale;    // mean
  else out[0] = sqrtf(s * scale);            // population std
}

static int reduce_blocks(size_t n) {
  size_t b = (n + 255) / 256;
  if (b > 1024) b = 1024;
  if (b < 1) b = 1;
  return (int)b;
}

int launch_grad_norm(const float* g, size_t n, float* norm_out, float* part, size_t part_elems,
                     cudaStream_t s) {
  const int nb = reduce_blocks(n);
  if ((size_t)nb > part_elems) { set_error("grad_norm: scratch too small"); return DDPPO_E_CONFIG; }
  ::ddppo::launch_k(sumsq_partial, nb, 256, 0, s, g, n, part, 1, nullptr);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(sum_final, 1, kFinal, 0, s, nb, part, norm_out, 0, 1.f);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// Adam step t = *t_dev + t_off (bias corrections 1 - beta^t computed once per block)
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, const float* __restrict__ norm,
                            float max_norm, float lr, float b1, float b2, float eps,
                            const int64_t* __restrict__ t_dev, int t_off) {
  DDPPO_PDL_ENTRY();
  __shared__ float s_bc[2];
  if (threadIdx.x == 0) {
    const double t = (double)(*t_dev + t_off);
    s_bc[0] = (float)(1.0 - pow((double)b1, t));
    s_bc[1] = (float)(1.0 - pow((double)b2, t));
  }
  __syncthreads();
  const float bc1 = s_bc[0], bc2 = s_bc[1];
  float coef = 1.f;
  if (norm && max_norm > 0.f) coef = fminf(1.f, max_norm / (norm[0] + 1e-6f));
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * coef;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

int launch_adam(float* p, const float* g, float* m, float* v, size_t n, const float* norm,
                float max_norm, float lr, float b1, float b2, float eps, const int64_t* t_dev,
                int t_off, cudaStream_t s) {
  size_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  ::ddppo::launch_k(adam_kernel, (unsigned)b, 256, 0, s, p, g, m, v, n, norm, max_norm, lr, b1, b2, eps, t_dev,
                                          t_off);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- env permutation: Fisher-Yates over the counter hash (seed, env 0, update, stream 7) ----
__device__ __forceinline__ uint64_t sm64r(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void perm_kernel(uint64_t seed, const int64_t* __restrict__ update_dev, int64_t epoch,
                            int E, int32_t* perm) {
  DDPPO_PDL_ENTRY();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t update = *update_dev;
  for (int i = 0; i < E; ++i) perm[i] = i;
  uint64_t k = sm64r(seed);
  k = sm64r(k + 0);
  k = sm64r(k + (uint64_t)update);
  for (int i = E - 1; i >= 1; --i) {
    const uint64_t idx = ((uint64_t)epoch * E + i) & 0xFFFFFFFFFFull;
    const uint64_t h = sm64r(k + ((7ull << 40) | idx));
    const int j = (int)(((h >> 32) * (uint64_t)(i + 1)) >> 32);
    const int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
}
int launch_permutation(uint64_t seed, const int64_t* update_dev, int64_t epoch, int E,
                       int32_t* perm, cudaStream_t s) {
  ::ddppo::launch_k(perm_kernel, 1, 32, 0, s, seed, update_dev, epoch, E, perm);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

// ---- advantage normalisation: (A - mean) / (std + 1e-5), population std ----
__global__ void normalize_kernel(const float* __restrict__ x, float* __restrict__ y, size_t n,
                                 const float* __restrict__ mean, const float* __restrict__ sd) {
  DDPPO_PDL_ENTRY();
  const float mu = mean[0], inv = 1.0f / (sd[0] + 1e-5f);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = (x[i] - mu) * inv;
}
int launch_normalize_adv(const float* adv, float* out, size_t n, float* scal2, float* part,
                         size_t part_elems, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  if ((size_t)nb > part_elems) { set_error("normalize: scratch too small"); return DDPPO_E_CONFIG; }
  ::ddppo::launch_k(sumsq_partial, nb, 256, 0, s, adv, n, part, 0, nullptr);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(sum_final, 1, kFinal, 0, s, nb, part, scal2, 1, 1.0f / (float)n);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(sumsq_partial, nb, 256, 0, s, adv, n, part, 1, scal2);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(sum_final, 1, kFinal, 0, s, nb, part, scal2 + 1, 2, 1.0f / (float)n);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(normalize_kernel, reduce_blocks(n), 256, 0, s, adv, out, n, scal2, scal2 + 1);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

__global__ void put_scalar_kernel(float* dst, const float* src) {
  DDPPO_PDL_ENTRY(); dst[0] = src[0]; }
int launch_copy_scalar(float* dst, const float* src, cudaStream_t s) {
  ::ddppo::launch_k(put_scalar_kernel, 1, 1, 0, s, dst, src);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
