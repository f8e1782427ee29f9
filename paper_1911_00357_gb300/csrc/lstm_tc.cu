// The LSTM forward recurrence on the 5th-generation tensor cores: one launch per layer
// runs all T steps of a segment (App. "Agent Design": the agent's LSTM; Sec. 4
// "Training": the forward pass recomputed over the rollout before back-propagation).
//
// Per step the recurrence is z = gx_t + R(h_{t-1} m_t) W_hh^T followed by the cell
// update, and the next step needs every unit's new state. Here the contraction is
// computed transposed (gate rows x envs) by tcgen05: CTA j owns the 32 units
// [32 j, 32 j + 32), i.e. 128 gate rows, which form the M = 128 side of the MMA. Its
// rows of W_hh (128 x H bf16, 128-byte-swizzled K-major) are staged into shared memory
// once and stay resident for the whole segment. Every step:
//   1. the masked state entering the step, R(h_{t-1} m_t) (E x H bf16, written by all
//      CTAs in the previous step), is staged into shared memory in the same swizzled
//      layout, env rows padded with zeros to N = 32, 64 or 128;
//   2. one thread issues the H / 16 MMAs (M = 128, N, K = 16) into an fp32 TMEM
//      accumulator and commits them to an mbarrier;
//   3. 16 warps read the accumulator: warp w takes TMEM lanes (rows) 32 (w % 4) .. + 31 and
//      columns 8 (w / 4) .. + 7 of every 32-column chunk. Row r holds gate r % 4 of unit
//      r / 4, so a warp holds all four gates of 8 units; a per-warp shared-memory transpose
//      hands each lane 2 (unit, env) cells per chunk, whose cell state c stays in registers
//      across the steps;
//   4. the lane adds gx, applies the gate nonlinearities and the cell update (the same
//      arithmetic as the step-by-step cell kernel), and writes the gates, c, h, the
//      layer output and the masked state entering the next step;
//   5. a grid-wide barrier (monotone arrival counter) ends the step.
// Every wait is bounded: a wait that runs out sets the sticky timeout flag; the CTA then
// waits (again bounded) for its own MMAs still in flight before it frees its tensor memory.
// Only the contraction's fp32 summation order differs from the step-by-step path.
#include <algorithm>

#include "nn_kernels.cuh"
#include "tc_common.cuh"

namespace ddppo {

namespace {

constexpr int LT_THREADS = 512;  // 16 warps: 4 per 32 TMEM lanes, each 8 columns of a chunk
constexpr int LT_UNITS = 32;     // hidden units per CTA (128 gate rows)
constexpr int LT_PITCH = 9;      // floats per row of the per-warp transpose tile (8 columns)

__device__ __forceinline__ float lt_sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// grid-wide barrier number `round`: every CTA adds one arrival and waits (bounded) for
// (round + 1) * gridDim.x; false when the wait ran out (timeout flag set)
__device__ bool lt_grid_barrier(unsigned* bar, unsigned round, int32_t* err, int* s_ok) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(bar, 1u);
    const unsigned target = (round + 1) * gridDim.x;
    int ok = 0;
    for (unsigned i = 0; i < TC_SPIN_LIMIT; ++i) {
      if (*(volatile unsigned*)bar >= target) { ok = 1; break; }
      if (err && (*(volatile int32_t*)err & ERRF_TIMEOUT)) break;
      __nanosleep(32);
    }
    if (!ok && err) atomicOr(err, ERRF_TIMEOUT);
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// 16-byte chunk `c` (0..7) of row `r` of a 128-byte-swizzled K-major atom
__device__ __forceinline__ uint32_t sw128_off(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

}  // namespace

// NCH: 32-env column chunks of the accumulator (N = 32 NCH)
template <int NCH>
__global__ void __launch_bounds__(LT_THREADS, 1) lstm_tc_fwd_kernel(LstmTc a) {
  constexpr int NP = 32 * NCH;
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ uint64_t mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_ok;
  __shared__ int abort_flag;
  const int H = a.H, E = a.E, G4 = 4 * H, KA = H / 64;  // K atoms of 64 elements
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int u0 = blockIdx.x * LT_UNITS;
  uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                                 // KA atoms of 128 rows x 128 B
  uint8_t* sB = sA + (size_t)KA * 128 * 128;          // KA atoms of NP rows x 128 B
  float* zt = (float*)(sB + (size_t)KA * NP * 128);   // [16 warps][32][LT_PITCH]
  float* ztw = zt + warp * 32 * LT_PITCH;
  const int qd = warp & 3, cg = warp >> 2;  // TMEM lane quadrant, 8-column group
  volatile int* abort = &abort_flag;

  if (threadIdx.x == 0) {
    mbar_init(&mma_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"((uint32_t)NP));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();    // the allocation is done before any thread of the block triggers
  DDPPO_PDL_ENTRY();
  // resident A: row r = 4 uu + q  <-  W_hh row q H + u0 + uu (eight 16-byte loads in flight
  // per thread)
  for (int i0 = threadIdx.x; i0 < 128 * (H / 8); i0 += LT_THREADS * 8) {
    uint4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * LT_THREADS;
      const int r = i / (H / 8), kc = i - r * (H / 8);
      const int q = r & 3, uu = r >> 2;
      if (i < 128 * (H / 8))
        v[j] = __ldg(reinterpret_cast<const uint4*>(a.Whh + ((size_t)q * H + u0 + uu) * H) + kc);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int i = i0 + j * LT_THREADS;
      if (i >= 128 * (H / 8)) break;
      const int r = i / (H / 8), kc = i - r * (H / 8);
      *reinterpret_cast<uint4*>(sA + (size_t)(kc >> 3) * 128 * 128 + sw128_off(r, kc & 7)) = v[j];
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = f16_idesc(128, NP, 0, 0);

  // this lane's cells: unit k of the warp's 8, envs 8 cg + eo + 4 i (i = 0, 1) of every
  // 32-env chunk
  const int k = lane & 7, eo = lane >> 3;
  const int u = u0 + 8 * qd + k;
  float cst[NCH][2];
  // the input projection of the next step does not depend on the recurrence: it is loaded
  // into registers before the step's barrier, off the critical path
  float zg[NCH][2][4];
  auto load_gx = [&](int t) {
    const float* gx_t = a.gx + (size_t)t * E * G4;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int e = ch * 32 + 8 * cg + eo + 4 * i;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          zg[ch][i][q] = e < E ? gx_t[(size_t)e * G4 + (size_t)q * H + u] : 0.f;
      }
  };
  load_gx(0);
  bool failed = false;
  uint32_t issued = 0;  // MMA batches committed (for the drain after a run-out)
  for (int t = 0; t < a.T && !failed; ++t) {
    // 1. stage R(h_{t-1} m_t): rows e < E from hm[t], zero rows up to NP
    const __nv_bfloat16* hm_t = a.hm + (size_t)t * E * H;
    for (int i0 = threadIdx.x; i0 < NP * (H / 8); i0 += LT_THREADS * 8) {
      uint4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = i0 + j * LT_THREADS;
        const int e = i / (H / 8), kc = i - e * (H / 8);
        v[j] = make_uint4(0u, 0u, 0u, 0u);
        if (i < NP * (H / 8) && e < E)
          v[j] = __ldcg(reinterpret_cast<const uint4*>(hm_t + (size_t)e * H) + kc);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int i = i0 + j * LT_THREADS;
        if (i >= NP * (H / 8)) break;
        const int e = i / (H / 8), kc = i - e * (H / 8);
        *reinterpret_cast<uint4*>(sB + (size_t)(kc >> 3) * NP * 128 + sw128_off(e, kc & 7)) = v[j];
      }
    }
    // the staged operand is read by the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 2. the contraction
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
      for (int kk = 0; kk < H / 16; ++kk) {
        const int j = kk >> 2, k4 = kk & 3;
        const uint64_t da = sw128_desc(a0 + (uint32_t)j * 128 * 128 + k4 * 32);
        const uint64_t db = sw128_desc(b0 + (uint32_t)j * NP * 128 + k4 * 32);
        tc_mma(tmem, da, db, idesc, kk > 0 ? 1u : 0u, 0);
      }
      tc_commit(&mma_bar);
    }
    ++issued;
    // 3. wait for it; each warp reads its 32 rows, chunk by chunk
    // (uniform: a thread whose wait ran out makes the whole CTA stop)
    const bool ok = __syncthreads_and(mbar_wait(&mma_bar, (uint32_t)(t & 1), abort, a.err) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint8_t* m_t = a.m + (size_t)t * E;
    const uint8_t* m_n = t + 1 < a.T ? a.m + (size_t)(t + 1) * E : nullptr;
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      if (!ok) break;
      uint32_t r[8];
      const uint32_t taddr = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(ch * 32 + cg * 8);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 8; ++j) ztw[lane * LT_PITCH + j] = __uint_as_float(r[j]);
      __syncwarp();
      // 4. the cells (unit u, env e = 32 ch + 8 cg + eo + 4 i)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int el = eo + 4 * i, e = ch * 32 + 8 * cg + el;
        if (e >= E) continue;
        const float zi = zg[ch][i][0] + ztw[(4 * k + 0) * LT_PITCH + el];
        const float zf = zg[ch][i][1] + ztw[(4 * k + 1) * LT_PITCH + el];
        const float zq = zg[ch][i][2] + ztw[(4 * k + 2) * LT_PITCH + el];
        const float zo = zg[ch][i][3] + ztw[(4 * k + 3) * LT_PITCH + el];
        const float ig = lt_sigm(zi), fg = lt_sigm(zf), gg = tanhf(zq), og = lt_sigm(zo);
        const size_t idx = (size_t)e * H + u;
        const float cprev = t == 0 ? a.c0[idx] : cst[ch][i];
        const float cp = m_t[e] ? cprev : 0.f;
        const float c = fg * cp + ig * gg;
        const float h = og * tanhf(c);
        cst[ch][i] = c;
        const size_t gb = ((size_t)t * E + e) * G4;
        a.gates[gb + u] = ig;
        a.gates[gb + H + u] = fg;
        a.gates[gb + 2 * H + u] = gg;
        a.gates[gb + 3 * H + u] = og;
        const size_t o = (size_t)t * E * H + idx;
        a.c[o] = c;
        a.h[o] = h;
        if (a.y_op) a.y_op[o] = __float2bfloat16_rn(h);
        if (m_n) a.hm[o + (size_t)E * H] = __float2bfloat16_rn(m_n[e] ? h : 0.f);
      }
      __syncwarp();  // the next chunk rewrites the transpose tile
    }
    // the accumulator is rewritten by the next step's MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (!ok) { failed = true; break; }
    if (t + 1 < a.T) load_gx(t + 1);
    // 5. every CTA's state for step t + 1 is written before anyone stages it
    if (t + 1 < a.T && !lt_grid_barrier(a.bar, (unsigned)t, a.err, &s_ok)) failed = true;
  }
  __syncthreads();
  if (*abort && threadIdx.x == 0 && issued > 0) {
    // a wait ran out: the last committed batch may still be running; wait (bounded) for it
    // before the tensor memory is freed
    mbar_drain_wait(&mma_bar, (uint32_t)((issued - 1) & 1u));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NP));
  }
}

static int lt_nch(int E) { return E <= 32 ? 1 : E <= 64 ? 2 : E <= 128 ? 4 : 0; }

static size_t lt_smem(int H, int E) {
  const int np = 32 * lt_nch(E);
  return 1024 + (size_t)(128 + np) * H * 2 + (size_t)(LT_THREADS / 32) * 32 * LT_PITCH * sizeof(float);
}

bool lstm_tc_supported(int H, int E, int num_sms) {
  if (E < 1 || !lt_nch(E) || H < 64 || H % 64 || H / LT_UNITS > num_sms) return false;
  return lt_smem(H, E) <= 225 * 1024;
}

int launch_lstm_tc_fwd(const LstmTc& a, int num_sms, cudaStream_t s) {
  if (!lstm_tc_supported(a.H, a.E, num_sms)) {
    set_error("lstm_tc: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  if (a.T < 1) return DDPPO_OK;
  const int nch = lt_nch(a.E);
  void (*kern)(LstmTc) = nch == 1 ? lstm_tc_fwd_kernel<1>
                       : nch == 2 ? lstm_tc_fwd_kernel<2> : lstm_tc_fwd_kernel<4>;
  const size_t smem = lt_smem(a.H, a.E);
  DDPPO_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // a single step has no barrier: a plain launch; longer segments launch cooperatively so
  // that every CTA of the grid is resident
  const bool coop = a.T > 1;
  if (coop) DDPPO_CHECK_CUDA(cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.H / LT_UNITS);
  cfg.blockDim = dim3(LT_THREADS);
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

}  // namespace ddppo
