// Generalised advantage estimation (Sec. 4 "Training": gamma 0.99, GAE tau 0.95) as a
// warp-level reverse scan of affine maps.
//
// A_t = delta_t + c_t A_{t+1} with delta_t = r_t + gamma (1-d_t) V_{t+1} - V_t and
// c_t = gamma lam (1-d_t) is an affine recurrence. A CTA stages a [T, 32-env] tile of
// (delta, c) into shared memory with coalesced loads; warp w scans env w: lane l composes
// the maps of its T/32 steps into (P_l, Q_l), a shuffle scan composes lanes l..31, and each
// lane then replays its chunk from the value entering it. The tile goes back out coalesced.
#include "common.cuh"

namespace ddppo {

__global__ void __launch_bounds__(1024) gae_kernel(const float* __restrict__ r,
                                                   const uint8_t* __restrict__ d,
                                                   const float* __restrict__ v, int T, int E,
                                                   float gamma, float lam, float* __restrict__ adv,
                                                   float* __restrict__ ret) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  float* sdelta = sh;           // [T][32]
  float* sc = sh + T * 32;      // [T][32]
  const int e0 = blockIdx.x * 32;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < T * 32; idx += nt) {
    const int t = idx >> 5, j = idx & 31, e = e0 + j;
    float de = 0.f, c = 0.f;
    if (e < E) {
      const float nd = d[(size_t)t * E + e] ? 0.f : 1.f;
      de = r[(size_t)t * E + e] + gamma * nd * v[(size_t)(t + 1) * E + e] - v[(size_t)t * E + e];
      c = gamma * lam * nd;
    }
    sdelta[idx] = de;
    sc[idx] = c;
  }
  __syncthreads();
  const int lane = tid & 31, w = tid >> 5, nw = nt >> 5;
  const int L = (T + 31) / 32;
  const int t0 = min(T, lane * L), t1 = min(T, t0 + L);
  for (int j = w; j < 32; j += nw) {
    float P = 0.f, Q = 1.f;
    for (int t = t1 - 1; t >= t0; --t) {
      const float c = sc[t * 32 + j];
      P = sdelta[t * 32 + j] + c * P;
      Q = c * Q;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float Pn = __shfl_down_sync(0xffffffffu, P, o);
      const float Qn = __shfl_down_sync(0xffffffffu, Q, o);
      if (lane + o < 32) {
        P = P + Q * Pn;
        Q = Q * Qn;
      }
    }
    float A = __shfl_down_sync(0xffffffffu, P, 1);
    if (lane == 31) A = 0.f;
    for (int t = t1 - 1; t >= t0; --t) {
      A = sdelta[t * 32 + j] + sc[t * 32 + j] * A;
      sdelta[t * 32 + j] = A;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < T * 32; idx += nt) {
    const int t = idx >> 5, j = idx & 31, e = e0 + j;
    if (e < E) {
      const float A = sdelta[idx];
      adv[(size_t)t * E + e] = A;
      ret[(size_t)t * E + e] = A + v[(size_t)t * E + e];
    }
  }
}

int launch_gae(const float* r, const uint8_t* d, const float* v, int T, int E, float gamma,
               float lam, float* adv, float* ret, cudaStream_t s) {
  const size_t smem = (size_t)T * 32 * 2 * sizeof(float);
  if (smem > 227 * 1024) {
    set_error("gae: T too large for one shared-memory tile");
    return DDPPO_E_CONFIG;
  }
  if (smem > 48 * 1024)
    DDPPO_CHECK_CUDA(cudaFuncSetAttribute(gae_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
  if (E == 0 || T == 0) return DDPPO_OK;
  ::ddppo::launch_k(gae_kernel, (E + 31) / 32, 1024, smem, s, r, d, v, T, E, gamma, lam, adv, ret);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
