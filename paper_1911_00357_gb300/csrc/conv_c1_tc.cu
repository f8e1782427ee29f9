// Single-channel convolution on tcgen05 -- the encoder's stem (App. "Visual Encoder": a
// 7x7 / stride-2 convolution of the 1-channel depth image) -- without an im2col matrix.
//
// A tile is 128 consecutive output pixels (NHWC order). Its patches (k x k taps of the one
// input channel, zero outside the image and past k^2, 64 taps per row) are gathered by the
// CTA's threads straight into shared memory in the 128-byte-swizzled K-major layout the
// MMA reads; the Cout x 64 weights stay resident for the whole kernel. One thread issues
// the 4 MMAs (M = 128, N = Cout, K = 16) of a tile into fp32 TMEM and commits them to an
// mbarrier; the 4 warps then read their 32 rows, transpose through shared memory and
// store whole output rows (y = acc, or y = beta y + acc). With the patch matrix never
// written, the convolution moves the input once and the fp32 output once instead of
// writing and re-reading k^2-wide patch rows. The MMAs are those of the im2col + GEMM
// path (K padded to 64 with zeros, the same four K = 16 steps), so the results are the
// same. Persistent CTAs (several per SM) walk the tiles; every wait is bounded, and after
// a run-out the CTA waits (bounded) for its last committed MMAs before freeing TMEM.
#include <algorithm>

#include "nn_kernels.cuh"
#include "tc_common.cuh"

namespace ddppo {

namespace {

constexpr int CC_THREADS = 128;
constexpr int CC_PITCH = 17;  // floats per staged row of a 16-column chunk

__device__ __forceinline__ uint32_t cc_sw128(int r, int c) {
  return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ uint32_t cc_pack(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

}  // namespace

// NC16: output channels / 16 (Cout = 16, 32 or 64)
template <int NC16>
__global__ void __launch_bounds__(CC_THREADS, 5) conv_c1_tc_kernel(ConvC1 a) {
  constexpr int COUT = 16 * NC16;
  constexpr uint32_t TCOLS = COUT < 32 ? 32 : COUT;
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;                  // 128 rows x 128 B
  uint8_t* sB = base + 128 * 128;      // COUT rows x 128 B
  float* stage = (float*)(sB + COUT * 128);  // [4 warps][32][CC_PITCH]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* st = stage + warp * 32 * CC_PITCH;
  volatile int* abort = &abort_flag;
  const int KK = a.k * a.k;
  const int M = a.N * a.Ho * a.Wo;  // < 2^31 (checked by the launcher)
  const int HoWo = a.Ho * a.Wo;
  const int ntiles = (M + 127) / 128;

  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  __syncthreads();    // the allocation is done before any thread of the block triggers
  DDPPO_PDL_ENTRY();
  // resident weights: row co = w[co, 0 .. k^2), zero up to 64 taps
  for (int i = threadIdx.x; i < COUT * 8; i += CC_THREADS) {
    const int co = i >> 3, c = i & 7;
    uint32_t v[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int t0 = c * 8 + 2 * h, t1 = t0 + 1;
      const __nv_bfloat16 lo = t0 < KK ? a.w[(size_t)co * a.ldw + t0] : __float2bfloat16_rn(0.f);
      const __nv_bfloat16 hi = t1 < KK ? a.w[(size_t)co * a.ldw + t1] : __float2bfloat16_rn(0.f);
      v[h] = cc_pack(lo, hi);
    }
    *reinterpret_cast<uint4*>(sB + cc_sw128(co, c)) = make_uint4(v[0], v[1], v[2], v[3]);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = f16_idesc(128, COUT, 0, 0);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);

  // this thread's chunk of taps (fixed over the tiles): offsets of taps 8 cc .. 8 cc + 7
  const int cc = threadIdx.x & 7, rr = threadIdx.x >> 3;
  int tdy[8], tdx[8];
  uint32_t tval = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int t = cc * 8 + q;
    tdy[q] = t / a.k - a.p;
    tdx[q] = t % a.k - a.p;
    if (t < KK) tval |= 1u << q;
  }
  uint32_t it = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int m0 = tile * 128;
    // 1. the tile's patches: 128 rows x 8 chunks of 8 taps. Thread i fills chunk i % 8 of
    // rows i / 8 + 16 j (j = 0..7): its 8 taps are fixed, and all 64 loads are in flight
    // before they are packed and stored
    {
      __nv_bfloat16 tv[8][8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int m = m0 + rr + 16 * j;
        const bool in_m = m < M;
        const int n = in_m ? m / HoWo : 0;
        const int rem = in_m ? m - n * HoWo : 0;
        const int oy = rem / a.Wo, ox = rem - oy * a.Wo;
        const int y0 = oy * a.s, x0 = ox * a.s;
        const __nv_bfloat16* xi = a.x + (size_t)n * a.H * a.W;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int iy = y0 + tdy[q], ix = x0 + tdx[q];
          const bool ok = in_m && ((tval >> q) & 1) && iy >= 0 && iy < a.H && ix >= 0 && ix < a.W;
          tv[j][q] = ok ? xi[iy * a.W + ix] : zero;
        }
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<uint4*>(sA + cc_sw128(rr + 16 * j, cc)) =
            make_uint4(cc_pack(tv[j][0], tv[j][1]), cc_pack(tv[j][2], tv[j][3]),
                       cc_pack(tv[j][4], tv[j][5]), cc_pack(tv[j][6], tv[j][7]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 2. the tile's 4 MMAs
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_addr(sA), b0 = smem_addr(sB);
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
        tc_mma(tmem, sw128_desc(a0 + k4 * 32), sw128_desc(b0 + k4 * 32), idesc, k4 > 0 ? 1u : 0u, 0);
      tc_commit(&bar);
    }
    const bool ok = __syncthreads_and(mbar_wait(&bar, it & 1u, abort, a.err) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) break;
    // 3. epilogue: warp w owns rows 32 w .. 32 w + 31, 16 columns at a time
    const int row0 = m0 + warp * 32;
#pragma unroll
    for (int c16 = 0; c16 < NC16; ++c16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c16 * 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) st[lane * CC_PITCH + j] = __uint_as_float(r[j]);
      __syncwarp();
      // two rows per instruction: lanes 0-15 row i, lanes 16-31 row i + 1 (64 B each)
      const int col = lane & 15, hr = lane >> 4;
#pragma unroll 4
      for (int i = 0; i < 32; i += 2) {
        const int m = row0 + i + hr;
        float v = st[(i + hr) * CC_PITCH + col];
        if (m < M) {
          float* yp = a.y + (size_t)m * COUT + c16 * 16 + col;
          if (a.beta != 0.f) v += a.beta * *yp;
          *yp = v;
        }
      }
      __syncwarp();
    }
    // the accumulator and the patch tile are rewritten by the next tile
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  __syncthreads();
  if (*abort && threadIdx.x == 0) mbar_drain_wait(&bar, it & 1u);  // the last committed batch
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TCOLS));
  }
}

bool conv_c1_tc_supported(int k, int Cout) {
  return k >= 1 && k * k <= 64 && (Cout == 16 || Cout == 32 || Cout == 64);
}

static size_t cc_smem(int cout) {
  return 1024 + 128 * 128 + (size_t)cout * 128 + (size_t)4 * 32 * CC_PITCH * sizeof(float);
}

int launch_conv_c1_tc(const ConvC1& a, int num_sms, cudaStream_t s) {
  if (!conv_c1_tc_supported(a.k, a.Cout) || a.ldw < a.k * a.k) {
    set_error("conv_c1_tc: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  const long long M = (long long)a.N * a.Ho * a.Wo;
  if (M <= 0) return DDPPO_OK;
  if (M > (1LL << 30)) {
    set_error("conv_c1_tc: too many output pixels");
    return DDPPO_E_CONFIG;
  }
  const long long ntiles = (M + 127) / 128;
  void (*kern)(ConvC1) = a.Cout == 16 ? conv_c1_tc_kernel<1>
                       : a.Cout == 32 ? conv_c1_tc_kernel<2> : conv_c1_tc_kernel<4>;
  const size_t smem = cc_smem(a.Cout);
  // CTAs per SM from the kernel's own limits: shared memory (227 KiB per SM, 1 KiB reserved
  // per CTA), tensor memory (512 columns per SM), registers, and at most 8
  const int tcols = a.Cout < 32 ? 32 : a.Cout;
  cudaFuncAttributes fa{};
  DDPPO_CHECK_CUDA(cudaFuncGetAttributes(&fa, kern));
  const int regs = std::max(1, ((fa.numRegs + 7) / 8) * 8) * CC_THREADS;  // per CTA
  const int occ = std::max(1, std::min({8, (int)(232448 / (smem + 1024)), 512 / tcols, 65536 / regs}));
  const long long grid = std::min<long long>(ntiles, (long long)num_sms * occ);
  ::ddppo::launch_k(kern, (unsigned)grid, CC_THREADS, smem, s, a);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
