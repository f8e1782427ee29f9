// The LSTM recurrence over a whole segment in one cooperative launch per layer and pass
// (App. "Agent Design": the agent's LSTM; Sec. 4 "Training": back-propagation through time
// over the rollout).
//
// Per step the recurrence is a small contraction -- [E envs] x [4H gate rows] x [H] --
// followed by the cell update, and the next step needs every unit's new state. Launched
// step by step that is two launches of a few microseconds of work each, T times per layer
// and pass. Here one grid of G CTAs (U = H / G units each, one CTA per SM) runs all T
// steps: each CTA keeps the recurrent weights of its units in registers (its 4U gate rows
// of W_hh for the forward, its U columns for the backward), the operand rows staged in
// shared memory, the contraction split over K with a fixed-order reduction, and one
// grid-wide barrier per step (a monotone arrival counter, the waits bounded: on a run-out
// the kernel sets the sticky timeout flag and returns). The launch is cooperative, so all
// CTAs are resident.
//
// Forward, step t:  z = gx_t + R(h_{t-1} m_t) W_hh^T   (R: the operand dtype)
//                   c_t = f (c_{t-1} m_t) + i g,  h_t = o tanh(c_t)
// Backward, step t: dh = dh_above_t + m_{t+1} dh_rec;  dc = dh o (1 - tanh^2 c_t) + m_{t+1} dc_carry
//                   dz = (dc g i(1-i), dc c_{t-1} m_t f(1-f), dc i (1-g^2), dh tanh(c_t) o(1-o))
//                   dc_carry <- dc f;  dh_rec <- R(dz_t) W_hh  (for step t-1)
// The arithmetic is that of the step-by-step kernels; only the contraction's fp32
// summation order differs.
#include <algorithm>

#include "nn_kernels.cuh"

namespace ddppo {

namespace {

constexpr int LS_THREADS = 256;
constexpr int LS_KPER = 32;     // recurrent weights per thread (registers)
constexpr int LS_ET_FWD = 32;   // envs per staged tile (forward)
constexpr int LS_ET_BWD = 16;   // envs per staged tile (backward: rows of 4H)
constexpr int LS_MAX_E = 64;
constexpr unsigned LS_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ float ld_op_cg(const void* p, size_t i, int bf) {
  if (bf) {
    const unsigned short v = __ldcg((const unsigned short*)p + i);
    return __uint_as_float((unsigned)v << 16);
  }
  return __ldcg((const float*)p + i);
}
__device__ __forceinline__ float round_op(float v, int bf) {
  return bf ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}
__device__ __forceinline__ void st_opv(void* p, size_t i, float v, int bf) {
  if (bf) ((__nv_bfloat16*)p)[i] = __float2bfloat16_rn(v);
  else ((float*)p)[i] = v;
}
__device__ __forceinline__ float sigm(float x) { return 1.f / (1.f + expf(-x)); }

// dst[0, n) (fp32, shared) <- src[off, off + n) (operand dtype, global, read through L2);
// n and off multiples of 8. 16-byte loads, eight in flight per thread: the staging is one
// or two L2 round trips rather than one per element.
__device__ __forceinline__ void stage_flat(float* dst, const void* src, size_t off, int n, int bf) {
  constexpr int UNR = 8;
  if (bf) {
    const uint4* sv = reinterpret_cast<const uint4*>((const __nv_bfloat16*)src + off);
    const int nv = n >> 3;
    for (int i0 = threadIdx.x; i0 < nv; i0 += blockDim.x * UNR) {
      uint4 v[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int j = i0 + u * blockDim.x;
        if (j < nv) v[u] = __ldcg(sv + j);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int j = i0 + u * blockDim.x;
        if (j >= nv) break;
        const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
        float4* d = reinterpret_cast<float4*>(dst + (size_t)j * 8);
        d[0] = make_float4(__uint_as_float(w[0] << 16), __uint_as_float(w[0] & 0xffff0000u),
                           __uint_as_float(w[1] << 16), __uint_as_float(w[1] & 0xffff0000u));
        d[1] = make_float4(__uint_as_float(w[2] << 16), __uint_as_float(w[2] & 0xffff0000u),
                           __uint_as_float(w[3] << 16), __uint_as_float(w[3] & 0xffff0000u));
      }
    }
  } else {
    const float4* sv = reinterpret_cast<const float4*>((const float*)src + off);
    const int nv = n >> 2;
    for (int i0 = threadIdx.x; i0 < nv; i0 += blockDim.x * UNR) {
      float4 v[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int j = i0 + u * blockDim.x;
        if (j < nv) v[u] = __ldcg(sv + j);
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int j = i0 + u * blockDim.x;
        if (j >= nv) break;
        reinterpret_cast<float4*>(dst)[j] = v[u];
      }
    }
  }
}

// grid-wide barrier number `round` (0, 1, ...): every CTA adds one arrival and waits for
// (round + 1) * gridDim.x; false when the wait ran out (timeout flag set)
__device__ bool grid_barrier(unsigned* bar, unsigned round, int32_t* err, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const unsigned target = (round + 1) * gridDim.x;
    int ok = 0;
    for (unsigned i = 0; i < LS_SPIN_LIMIT; ++i) {
      if (*(volatile unsigned*)bar >= target) { ok = 1; break; }
      if (err && (*(volatile int32_t*)err & ERRF_TIMEOUT)) break;  // another CTA gave up
      __nanosleep(32);
    }
    if (!ok && err) atomicOr(err, ERRF_TIMEOUT);
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

}  // namespace

// rows of a CTA: r = q * U + uu (gate q, unit u0 + uu) -> W_hh row q * H + u0 + uu
__global__ void __launch_bounds__(LS_THREADS, 1) lstm_seq_fwd_kernel(LstmSeq a) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  __shared__ int s_ok;
  const int H = a.H, U = H / gridDim.x, R4 = 4 * U, u0 = blockIdx.x * U;
  const int KC = LS_THREADS / R4, kper = H / KC;
  const int ET = min(a.E, LS_ET_FWD);
  float* hs = sh;                          // [ET][H]
  float* zp = hs + (size_t)ET * H;         // [R4][ET][KC]
  float* zs = zp + (size_t)R4 * ET * KC;   // [ET][R4]
  const int tid = threadIdx.x, r = tid / KC, kc = tid - r * KC;
  const int bf = a.op_bf16;
  // this thread's slice of its row: k = kk * KC + kc
  float w[LS_KPER];
  {
    const int q = r / U, uu = r - q * U;
    const size_t row = (size_t)q * H + u0 + uu;
#pragma unroll
    for (int kk = 0; kk < LS_KPER; ++kk)
      w[kk] = kk < kper ? ld_op_cg(a.Whh, row * H + (size_t)kk * KC + kc, bf) : 0.f;
  }
  const int E = a.E;
  for (int t = 0; t < a.T; ++t) {
    for (int e0 = 0; e0 < E; e0 += ET) {
      const int ne = min(ET, E - e0);
      // stage the masked previous state of the tile (operand dtype values)
      if (t == 0) {
        for (int i = tid; i < ne * H; i += LS_THREADS) {
          const int e = i / H, k = i - e * H;
          hs[i] = a.m[e0 + e] ? round_op(a.h0[(size_t)(e0 + e) * H + k], bf) : 0.f;
        }
      } else {
        stage_flat(hs, a.hm, ((size_t)t * E + e0) * H, ne * H, bf);
      }
      __syncthreads();
      for (int e = 0; e < ne; ++e) {
        const float* he = hs + (size_t)e * H + kc;
        float acc = 0.f;
#pragma unroll
        for (int kk = 0; kk < LS_KPER; ++kk)
          if (kk < kper) acc += he[kk * KC] * w[kk];
        zp[((size_t)r * ET + e) * KC + kc] = acc;
      }
      __syncthreads();
      for (int i = tid; i < ne * R4; i += LS_THREADS) {
        const int e = i / R4, rr = i - e * R4;
        const int q = rr / U, uu = rr - q * U;
        float z = a.gx[((size_t)t * E + e0 + e) * 4 * H + (size_t)q * H + u0 + uu];
        const float* p = zp + ((size_t)rr * ET + e) * KC;
        for (int c = 0; c < KC; ++c) z += p[c];
        zs[e * R4 + rr] = z;
      }
      __syncthreads();
      for (int i = tid; i < ne * U; i += LS_THREADS) {
        const int e = i / U, uu = i - e * U, ge = e0 + e, u = u0 + uu;
        const float zi = zs[e * R4 + uu], zf = zs[e * R4 + U + uu];
        const float zg = zs[e * R4 + 2 * U + uu], zo = zs[e * R4 + 3 * U + uu];
        const float ig = sigm(zi), fg = sigm(zf), gg = tanhf(zg), og = sigm(zo);
        const size_t idx = (size_t)ge * H + u;
        const float cprev = t == 0 ? a.c0[idx] : a.c[(size_t)(t - 1) * E * H + idx];
        const float cp = a.m[(size_t)t * E + ge] ? cprev : 0.f;
        const float c = fg * cp + ig * gg;
        const float h = og * tanhf(c);
        const size_t gb = ((size_t)t * E + ge) * 4 * H;
        a.gates[gb + u] = ig;
        a.gates[gb + H + u] = fg;
        a.gates[gb + 2 * H + u] = gg;
        a.gates[gb + 3 * H + u] = og;
        const size_t o = (size_t)t * E * H + idx;
        a.c[o] = c;
        a.h[o] = h;
        if (a.y_op) st_opv(a.y_op, o, h, bf);
        if (t == 0) st_opv(a.hm, idx, a.m[ge] ? a.h0[idx] : 0.f, bf);  // hm_0 for the backward
        if (t + 1 < a.T) st_opv(a.hm, o + (size_t)E * H, a.m[(size_t)(t + 1) * E + ge] ? h : 0.f, bf);
      }
      __syncthreads();
    }
    if (t + 1 < a.T && !grid_barrier(a.bar, (unsigned)t, a.err, &s_ok)) return;
  }
}

// columns of a CTA: its units u0 .. u0 + U - 1 of W_hh [4H, H]; thread (uu, jc) holds
// W_hh[j][u0 + uu] for j = jj * JC + jc
__global__ void __launch_bounds__(LS_THREADS, 1) lstm_seq_bwd_kernel(LstmSeq a) {
  DDPPO_PDL_ENTRY();
  extern __shared__ float sh[];
  __shared__ int s_ok;
  const int H = a.H, U = H / gridDim.x, u0 = blockIdx.x * U, G4 = 4 * H;
  const int JC = LS_THREADS / U, jper = G4 / JC;
  const int E = a.E, ET = min(E, LS_ET_BWD);
  float* dgs = sh;                         // [ET][4H]
  float* zp = dgs + (size_t)ET * G4;       // [U][ET][JC]
  float* dh_rec = zp + (size_t)U * ET * JC;  // [E][U]
  float* dc_carry = dh_rec + (size_t)E * U;  // [E][U]
  const int tid = threadIdx.x, uu_b = tid / JC, jc = tid - uu_b * JC;
  const int bf = a.op_bf16;
  float w[LS_KPER];
#pragma unroll
  for (int jj = 0; jj < LS_KPER; ++jj)
    w[jj] = jj < jper ? ld_op_cg(a.Whh, ((size_t)jj * JC + jc) * H + u0 + uu_b, bf) : 0.f;
  for (int t = a.T - 1; t >= 0; --t) {
    // phase A: the gate gradients of this CTA's units
    for (int i = tid; i < E * U; i += LS_THREADS) {
      const int e = i / U, uu = i - e * U, u = u0 + uu;
      const size_t idx = (size_t)e * H + u, o = (size_t)t * E * H + idx;
      const size_t gb = ((size_t)t * E + e) * G4;
      const float ig = a.gates[gb + u], fg = a.gates[gb + H + u];
      const float gg = a.gates[gb + 2 * H + u], og = a.gates[gb + 3 * H + u];
      const float c = a.c[o];
      const float cprev = t == 0 ? a.c0[idx] : a.c[o - (size_t)E * H];
      const float cp = a.m[(size_t)t * E + e] ? cprev : 0.f;
      const bool carry = t + 1 < a.T && a.m[(size_t)(t + 1) * E + e];
      float dh = a.dh_above[o];
      if (carry) dh += dh_rec[i];
      const float tc = tanhf(c);
      float dc = dh * og * (1.f - tc * tc);
      if (carry) dc += dc_carry[i];
      const float dzi = dc * gg * ig * (1.f - ig);
      const float dzf = dc * cp * fg * (1.f - fg);
      const float dzg = dc * ig * (1.f - gg * gg);
      const float dzo = dh * tc * og * (1.f - og);
      dc_carry[i] = dc * fg;
      a.dg32[gb + u] = dzi;
      a.dg32[gb + H + u] = dzf;
      a.dg32[gb + 2 * H + u] = dzg;
      a.dg32[gb + 3 * H + u] = dzo;
      st_opv(a.dg_op, gb + u, dzi, bf);
      st_opv(a.dg_op, gb + H + u, dzf, bf);
      st_opv(a.dg_op, gb + 2 * H + u, dzg, bf);
      st_opv(a.dg_op, gb + 3 * H + u, dzo, bf);
    }
    if (t == 0) break;
    if (!grid_barrier(a.bar, (unsigned)(a.T - 1 - t), a.err, &s_ok)) return;
    // phase B: dh_rec[e][u] = sum_j R(dz_t)[e][j] W_hh[j][u] for this CTA's units
    for (int e0 = 0; e0 < E; e0 += ET) {
      const int ne = min(ET, E - e0);
      stage_flat(dgs, a.dg_op, ((size_t)t * E + e0) * G4, ne * G4, bf);
      __syncthreads();
      for (int e = 0; e < ne; ++e) {
        const float* de = dgs + (size_t)e * G4 + jc;
        float acc = 0.f;
#pragma unroll
        for (int jj = 0; jj < LS_KPER; ++jj)
          if (jj < jper) acc += de[jj * JC] * w[jj];
        zp[((size_t)uu_b * ET + e) * JC + jc] = acc;
      }
      __syncthreads();
      for (int i = tid; i < ne * U; i += LS_THREADS) {
        const int e = i / U, uu = i - e * U;
        const float* p = zp + ((size_t)uu * ET + e) * JC;
        float s = 0.f;
        for (int c = 0; c < JC; ++c) s += p[c];
        dh_rec[(e0 + e) * U + uu] = s;
      }
      __syncthreads();
    }
  }
}

// CTAs for hidden size H: the most CTAs (a divisor of H, at most the SM count) whose units'
// recurrent weights fit LS_KPER registers per thread; 0 when no grid qualifies
int lstm_seq_grid(int H, int num_sms) {
  for (int G = std::min(H, num_sms); G >= 1; --G) {
    if (H % G) continue;
    const int U = H / G;
    if (4 * U > LS_THREADS || LS_THREADS % (4 * U) || LS_THREADS % U) continue;
    const int KC = LS_THREADS / (4 * U), JC = LS_THREADS / U;
    if (H % KC || (4 * H) % JC) continue;
    if (H / KC > LS_KPER || 4 * H / JC > LS_KPER) continue;
    return G;
  }
  return 0;
}

static size_t fwd_smem(int H, int G, int E) {
  const int U = H / G, R4 = 4 * U, KC = LS_THREADS / R4, ET = std::min(E, LS_ET_FWD);
  return ((size_t)ET * H + (size_t)R4 * ET * KC + (size_t)ET * R4) * sizeof(float);
}
static size_t bwd_smem(int H, int G, int E) {
  const int U = H / G, JC = LS_THREADS / U, ET = std::min(E, LS_ET_BWD);
  return ((size_t)ET * 4 * H + (size_t)U * ET * JC + 2 * (size_t)E * U) * sizeof(float);
}

bool lstm_seq_supported(int H, int E, int num_sms) {
  if (E < 1 || E > LS_MAX_E) return false;
  const int G = lstm_seq_grid(H, num_sms);
  if (!G) return false;
  return fwd_smem(H, G, E) <= 200 * 1024 && bwd_smem(H, G, E) <= 200 * 1024;
}

// a single step has no barrier: a plain launch (it need not wait for the whole grid to be
// resident beside kernels of other streams); longer segments launch cooperatively
static int launch_seq(void (*kern)(LstmSeq), const LstmSeq& a, size_t smem, int G, cudaStream_t s) {
  const bool coop = a.T > 1;
  if (coop) DDPPO_CHECK_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s));
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(G);
  cfg.blockDim = dim3(LS_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = coop ? 1 : 0;
  DDPPO_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
  return DDPPO_OK;
}

int launch_lstm_seq_fwd(const LstmSeq& a, int num_sms, cudaStream_t s) {
  const int G = lstm_seq_grid(a.H, num_sms);
  if (!G || a.E > LS_MAX_E) {
    set_error("lstm_seq: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  return launch_seq(lstm_seq_fwd_kernel, a, fwd_smem(a.H, G, a.E), G, s);
}

int launch_lstm_seq_bwd(const LstmSeq& a, int num_sms, cudaStream_t s) {
  const int G = lstm_seq_grid(a.H, num_sms);
  if (!G || a.E > LS_MAX_E) {
    set_error("lstm_seq: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  return launch_seq(lstm_seq_bwd_kernel, a, bwd_smem(a.H, G, a.E), G, s);
}

}  // namespace ddppo
