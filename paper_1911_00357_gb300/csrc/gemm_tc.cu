// BF16 (and E4M3) GEMM on the 5th-generation tensor cores (sm_103a):
// C[M,N] (+)= A[M,K] B[N,K]^T.
//
//   * TMA (cp.async.bulk.tensor.2d) stages 128x64 A tiles and BNx64 B tiles into shared
//     memory in the 128-byte swizzled K-major layout; out-of-range rows/columns are
//     zero-filled by the copy engine, so ragged M, N and K need no special path.
//   * A 4-stage ring of mbarriers: "full" (TMA -> MMA, transaction bytes) and "empty"
//     (MMA -> TMA, signalled by tcgen05.commit when the MMAs reading a stage retire).
//   * One thread issues tcgen05.mma.cta_group::1.kind::f16 (M=128, N=BN, K=16 per
//     instruction) accumulating in fp32 in tensor memory (BN columns of TMEM); E4M3
//     operands use kind::f8f6f4 (K=32) on the same byte layouts, with the two per-tensor
//     scales applied in the epilogue.
//   * Convolutions gather their operand tiles themselves: a 4-D TMA box per filter tap,
//     or one halo box per tile read through row-shifted descriptors (for 3x3 filters on
//     images at most 32 wide: whole image rows per tile, the three column taps as one
//     N = 3 x 32 MMA per filter row, combined in the epilogue by lane shuffles).
//   * Epilogue: 4 warps each read their 32 TMEM lanes (rows) with tcgen05.ld.32x32b and
//     apply beta/bias/ReLU, storing fp32 or bf16 -- or fp32 split-K partials that a
//     fixed-order reduction combines. Where the tile's rows are whole output rows, each
//     warp stages its 32 x 32 block in the swizzle a tensor copy reads and issues one
//     cp.async.bulk.tensor store (C for beta != 0 comes in by a tensor load); otherwise
//     it transposes through shared memory and stores row by row.
//   * Small-M problems (the per-step LSTM recurrences) are computed transposed (swap AB)
//     so the 128-row MMA dimension covers the large side.
// Every wait is bounded; a wait that runs out sets the sticky timeout flag and the CTA
// stops: its epilogue stores nothing, and before the tensor memory is freed the CTA waits
// (again with a limit) for its own asynchronous work still in flight -- the TMA loads it
// issued into stages the MMA thread never consumed, and the MMAs it issued (one final
// tcgen05.commit covers all of them) -- so no copy or MMA lands in freed memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "gemm.cuh"
#include "tc_common.cuh"

namespace ddppo {

constexpr int TC_BM = 128, TC_BK = 64, TC_STAGES = 16;  // TC_STAGES: deepest ring
// epilogue staging: 32 x 32 floats per epilogue warp, 1024-byte aligned. The transpose
// path stores element (row i, column j) at i * 32 + (j ^ i) (conflict-free both ways); the
// tensor-store path writes 128-byte rows whose 16-byte chunks sit at chunk ^ (row & 7) --
// the layout a SWIZZLE_128B tensor copy reads (SWIZZLE_64B for bf16 rows of 64 bytes).
constexpr int TC_EPI_FLOATS = 32 * 32;
// dynamic part; the static part (barriers, 16 KiB epilogue staging: 17 KiB in all) makes up
// the rest of the 227 KiB opt-in limit
constexpr size_t TC_SMEM_MAX = 205 * 1024;
constexpr size_t TC_SMEM_TWO_PER_SM = 94 * 1024;  // dynamic bytes that still fit two CTAs per SM

struct TcSmem {
  // stage buffers are carved from dynamic shared memory (1024-byte aligned)
  uint64_t full[TC_STAGES];
  uint64_t empty[TC_STAGES];
  uint64_t done;
  uint64_t drain;      // final commit of the MMA thread after an abort
  uint32_t issued;     // ring stages whose TMA loads the producer issued
  uint32_t consumed;   // ring stages the MMA thread waited for
  uint32_t tmem_base;
  int abort;
};

// After an abort (uniform once every role has left its loop): thread 0 waits for the
// TMA loads of the stages issued but never consumed, stage it % stages completing phase
// (it / stages) & 1 -- at most `stages` of them, since the producer waits for a stage's
// release before refilling it -- and, in the halo mode, for the resident weights.
__device__ __forceinline__ void drain_unconsumed(uint64_t* full, uint32_t consumed, uint32_t issued,
                                                 int stages, uint64_t* weights) {
  for (uint32_t it = consumed; it < issued; ++it)
    mbar_drain_wait(&full[it % stages], (it / stages) & 1u);
  if (weights) mbar_drain_wait(weights, 0u);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1, int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4, %5, %6}], [%2];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
}

// K-major tile with 64-byte rows (32 bf16 K-elements), 64-byte swizzle: 8-row groups
// 512 B apart; used by the implicit convolution when C = 32
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;              // SWIZZLE_64B
  return d;
}

// implicit-im2col parameters of a convolution A operand (passed by value to the kernel).
// on = 1: forward / input-gradient convolution, A = [output pixels, (tap, channel)] K-major,
//         one box of cbw channels x 128 pixels per K block;
// on = 2: weight gradient, A = [(tap, channel), output pixels] MN-major: per 64-pixel K
//         block, 128 / cbw boxes of 64 pixels x cbw channels (one per tap / channel block).
// on = 3: halo (stride-1 'same' convolution): per channel block ONE box of the input (the
//         tile's output rows plus the filter's halo, rows of pitch Wp = W + 2p) is staged,
//         and every filter tap reads it as a row-shifted view. Tile rows are "anchors" on
//         the Wp-pitch grid; anchors outside the image are computed and discarded.
// on = 4: row halo (3x3 stride-1 'same' convolution of 32 channels, W in {8, 16, 32}, at
//         most 32 output channels): a tile is R = 128 / W whole image rows; its box holds
//         those rows and the rows above and below (W columns from x = 0, pitch W, so each
//         filter row ky is the box shifted by ky W rows -- a whole number of 512-byte
//         swizzle atoms). One MMA per (ky, 16-channel step) multiplies by the three column
//         taps at once (N = 96: B rows (kx, co)), giving D_kx at every pixel; the epilogue
//         forms out(x) = D_1(x) + D_0(x - 1) + D_2(x + 1) with the neighbours' values taken
//         by lane shuffles (a row never crosses a warp) and zero at the image's edges.
struct ConvA {
  int on = 0;
  int C = 0, cbw = 64;       // input channels, channels per K-block (64 or 32)
  int k = 1, s = 1, p = 0;
  int Ho = 1, Wo = 1;
  int hi = 1;                // output rows per pixel block (or Ho when a block spans images)
  // halo mode
  int N = 1, H = 1, W = 1;   // images and their (input = output) size
  int Wp = 1, Hh = 1;        // anchor row pitch W + 2p, anchor rows per image H + 2p
  int ni = 0;                // images per tile (small images), or 0: tiles within one image
  int tpi = 1;               // tiles per image when ni == 0
  int rows_box = 1;          // rows of the halo box (per image)
  int R = 0;                 // row halo: image rows per tile
  int tiles_m = 1;
  uint32_t halo_bytes = 0;   // stride of the two halo stages in shared memory
  uint32_t box_bytes = 0;    // bytes one halo box delivers
};

// output row of anchor r of halo-mode tile tm, or -1 when the anchor is not an output pixel
__device__ __forceinline__ long long halo_out_row(const ConvA& ca, int tm, int r) {
  int img, y, x;
  if (ca.on == 4) {
    img = tm / ca.tpi;
    const int rr = r / ca.W;
    x = r - rr * ca.W;
    y = (tm - img * ca.tpi) * ca.R + rr;
  } else if (ca.ni) {
    const int per = ca.Hh * ca.Wp;
    const int i = r / per, rem = r - i * per;
    if (i >= ca.ni) return -1;
    img = tm * ca.ni + i;
    y = rem / ca.Wp;
    x = rem - y * ca.Wp;
  } else {
    img = tm / ca.tpi;
    const int a = (tm - img * ca.tpi) * 128 + r;
    y = a / ca.Wp;
    x = a - y * ca.Wp;
  }
  if (img >= ca.N || y >= ca.H || x >= ca.W) return -1;
  return ((long long)img * ca.H + y) * ca.W + x;
}

// MN-major tile with 64-byte rows (32 MN-elements), 64-byte swizzle: blocks of 32 MN
// columns 64 rows (4 KiB) apart (LBO), 8-row K groups 512 B apart (SBO)
__device__ __forceinline__ uint64_t sw64_mn_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(4096 >> 4) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// MN-major tile: rows of 64 MN-elements (128 B), one row per K index; blocks of 64 MN
// columns are 64 rows (8 KiB) apart (LBO); 8-row K groups 1024 B apart (SBO).
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(8192 >> 4) << 16;    // leading byte offset: next 64-wide MN block
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset: next 8-row K group
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// 32 accumulator columns of this warp's 32 TMEM lanes -> registers (waits for the load)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// tensor store of one 32 x 32 block of the output from shared memory (bulk async group of
// the issuing thread); rows and columns outside the tensor are not written
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   (uint64_t)map),
               "r"(smem_addr(src)), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y,
                                             int z) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                   (uint64_t)map),
               "r"(smem_addr(src)), "r"(x), "r"(y), "r"(z)
               : "memory");
}
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// Persistent, warp-specialised kernel. Warp 0 streams (tile, k-block) stages through the
// shared-memory ring with TMA; warp 1 issues the MMAs of a tile into one of two TMEM
// accumulators; warps 2..5 drain the other accumulator (tcgen05.ld -> a tensor store from
// swizzled shared memory, or a shared-memory transpose and coalesced row stores), so one
// tile's epilogue overlaps the next tile's loads and MMAs.
// Tiles are (m, n, split) triples walked with stride gridDim.x.
constexpr int TC_PTHREADS = 192;

template <int BN>
__global__ void __launch_bounds__(TC_PTHREADS, 2)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   int M, int N, int K, int kchunk, float* __restrict__ C, int ldc, int c_bf16,
                   float beta, const float* __restrict__ bias, int relu, int trans_out,
                   float* __restrict__ partial, int32_t* err, int a_mn, int b_mn, int stages,
                   int tiles_m, int tiles_n, int splits, ConvA ca, int fp8,
                   const float* __restrict__ scale_a, const float* __restrict__ scale_b,
                   const __grid_constant__ CUtensorMap mapC, int tma_out_req) {
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ TcSmem ctl;
  __shared__ uint64_t acc_full[2], acc_empty[2];
  __shared__ uint64_t epi_bar[4];  // tensor loads of C blocks (beta != 0), one per epilogue warp
  // epilogue staging, one 32 x 32 block per epilogue warp (static: known to be shared memory)
  __shared__ __align__(1024) float epi_stage[4][TC_EPI_FLOATS];
  // stage sizes follow the K extent of one ring slot (32 channels for narrow convolutions);
  // the halo mode has a ring of `stages` halo boxes (A) and all the weights resident (B)
  const bool halo = ca.on >= 3;
  const bool rowh = BN == 32 && ca.on == 4;  // the row halo has one 32-column N tile
  // accumulator columns: BN per buffer, or 96 (three column taps x 32) in the row halo,
  // spaced 128 apart
  const uint32_t acc_stride = rowh ? 128u : (uint32_t)BN, tcols = 2u * acc_stride;
  const int kslot = (ca.on == 1 || halo) ? ca.cbw : TC_BK;
  const uint32_t A_BYTES = halo ? ca.halo_bytes : TC_BM * kslot * 2, B_BYTES = BN * kslot * 2;
  uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = base;
  uint8_t* sB = base + stages * A_BYTES;  // halo mode: the resident weights
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = tiles_m * tiles_n * splits;
  volatile int* abort = &ctl.abort;

  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&ctl.full[s], 1);
      mbar_init(&ctl.empty[s], 1);
    }
    mbar_init(&ctl.done, 1);  // halo mode: resident weights landed
    mbar_init(&ctl.drain, 1);
    ctl.issued = 0;
    ctl.consumed = 0;
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
    }
    for (int b = 0; b < 4; ++b) mbar_init(&epi_bar[b], 1);
    ctl.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&ctl.tmem_base)),
                 "r"(tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  DDPPO_PDL_ENTRY();  // after the barrier set-up and the tensor-memory allocation
  const uint32_t tmem = ctl.tmem_base;

  if (warp == 0 && halo) {
    if (lane == 0) {
      // halo producer: the weights of every (tap, channel block) once, resident for the
      // whole kernel; then per (tile, channel block) one input box through the ring
      const int nkk = ca.k * ca.k, ncb = ca.C / ca.cbw;
      const uint32_t wbox = (uint32_t)BN * ca.cbw * 2;
      mbar_expect_tx(&ctl.done, wbox * nkk * ncb);
      for (int tap = 0; tap < nkk; ++tap)
        for (int cb = 0; cb < ncb; ++cb)
          tma_load_2d(sB + (tap * ncb + cb) * wbox, &mapB, &ctl.done, tap * ca.C + cb * ca.cbw, 0);
      uint32_t hit = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        const int tm = t % tiles_m, z = t / (tiles_m * tiles_n);
        int img, ybase, xbase = -ca.p;
        if (rowh) {
          img = tm / ca.tpi;
          ybase = (tm - img * ca.tpi) * ca.R - 1;
          xbase = 0;
        } else if (ca.ni) {
          img = tm * ca.ni;
          ybase = -ca.p;
        } else {
          img = tm / ca.tpi;
          ybase = ((tm - img * ca.tpi) * TC_BM) / ca.Wp - ca.p;
        }
        const int cb_end = min(ca.C, z * kchunk + kchunk);
        for (int c0 = z * kchunk; c0 < cb_end; c0 += ca.cbw, ++hit) {
          const int hs = hit % stages;
          if (!mbar_wait(&ctl.empty[hs], ((hit / stages) & 1u) ^ 1u, abort, err)) break;
          mbar_expect_tx(&ctl.full[hs], ca.box_bytes);
          tma_load_4d(sA + hs * A_BYTES, &mapA, &ctl.full[hs], c0, xbase, ybase, img);
        }
      }
      ctl.issued = hit;
    }
  } else if (warp == 1 && halo) {
    if (lane == 0) {
      // halo MMA issuer: tap (ky, kx) reads the staged box from row off + ky Wp + kx on
      const int NM = rowh ? 96 : BN;  // MMA N: the row halo's three column taps x 32
      const uint32_t idesc = fp8 ? f8_idesc(TC_BM, NM) : f16_idesc(TC_BM, NM, 0, 0);
      const int nkk = ca.k * ca.k, ncb = ca.C / ca.cbw, rb = ca.cbw * 2;
      const uint32_t wbox = (uint32_t)BN * ca.cbw * 2;
      const bool wok = mbar_wait(&ctl.done, 0u, abort, err);
      uint32_t hit = 0, ti = 0;
      for (int t = blockIdx.x; t < ntiles && wok && !*abort; t += gridDim.x, ++ti) {
        const int tm = t % tiles_m, z = t / (tiles_m * tiles_n);
        const int off = ca.ni ? 0 : ((tm % ca.tpi) * TC_BM) % ca.Wp;
        const uint32_t buf = ti & 1u, bph = (ti >> 1) & 1u;
        if (!mbar_wait(&acc_empty[buf], bph ^ 1u, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + buf * acc_stride;
        uint32_t acc = 0;
        const int cb_end = min(ca.C, z * kchunk + kchunk);
        for (int c0 = z * kchunk; c0 < cb_end; c0 += ca.cbw, ++hit) {
          const int hs = hit % stages;
          if (!mbar_wait(&ctl.full[hs], (hit / stages) & 1u, abort, err)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t h0 = smem_addr(sA + hs * A_BYTES);
          const int cb = c0 / ca.cbw;
          if (rowh) {
            // filter row ky: the box from row ky W on; B = the weights of taps (ky, 0..2),
            // resident one after another (96 rows of 64 bytes)
            for (int ky = 0; ky < 3; ++ky) {
              const uint32_t arow = h0 + (uint32_t)(ky * ca.W) * (uint32_t)rb;
              const uint32_t b0 = smem_addr(sB + (ky * 3 * ncb + cb) * wbox);
              for (int kq = 0; kq < ca.cbw / 16; ++kq) {
                tc_mma(dacc, sw64_desc(arow + kq * 32), sw64_desc(b0 + kq * 32), idesc, acc, fp8);
                acc = 1u;
              }
            }
          }
          for (int tap = 0; tap < (rowh ? 0 : nkk); ++tap) {
            const int ky = tap / ca.k, kx = tap - ky * ca.k;
            const uint32_t arow = h0 + (uint32_t)(off + ky * ca.Wp + kx) * rb;
            const uint32_t b0 = smem_addr(sB + (tap * ncb + cb) * wbox);
            for (int kq = 0; kq < ca.cbw / 16; ++kq) {
              const uint64_t da = ca.cbw == 32 ? sw64_desc(arow + kq * 32) : sw128_desc(arow + kq * 32);
              const uint64_t db = ca.cbw == 32 ? sw64_desc(b0 + kq * 32) : sw128_desc(b0 + kq * 32);
              tc_mma(dacc, da, db, idesc, acc, fp8);
              acc = 1u;
            }
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_addr(&ctl.empty[hs]))
              : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&acc_full[buf]))
            : "memory");
      }
      ctl.consumed = hit;
      if (*abort) {
        tc_commit(&ctl.drain);  // arrives once every MMA this thread issued has completed
        mbar_drain_wait(&ctl.drain, 0u);
      }
    }
  } else if (warp == 0) {
    if (lane == 0) {
      // TMA producer over every (tile, k-block) of this CTA
      const int kstep = ca.on == 1 ? ca.cbw : TC_BK;
      uint32_t tx = (uint32_t)(TC_BM + BN) * kstep * 2;
      uint32_t it = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        const int tm = t % tiles_m, tn = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
        const int m0 = tm * TC_BM, n0 = tn * BN;
        const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
        const int nkb = (kend - kbeg + kstep - 1) / kstep;
        // weight gradient: boxes of this tile's (tap, channel) rows that exist (rows >= M
        // are left unloaded; their accumulator rows are never stored)
        int nbox = 0;
        if (ca.on == 2) {
          nbox = min(TC_BM / ca.cbw, (M - m0 + ca.cbw - 1) / ca.cbw);
          tx = (uint32_t)BN * TC_BK * 2 + (uint32_t)nbox * 64 * ca.cbw * 2;
        }
        int img = 0, oy0 = 0;
        if (ca.on == 1) {
          const int pix = ca.Ho * ca.Wo;
          img = m0 / pix;
          oy0 = (m0 - img * pix) / ca.Wo;
        }
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % stages;
          const uint32_t ph = (it / stages) & 1u;
          if (!mbar_wait(&ctl.empty[s], ph ^ 1u, abort, err)) break;
          mbar_expect_tx(&ctl.full[s], tx);
          const int k = kbeg + kb * kstep;
          if (ca.on == 2) {
            const int pix = ca.Ho * ca.Wo;
            const int im = k / pix, oy = (k - im * pix) / ca.Wo;
            for (int j = 0; j < nbox; ++j) {
              const int kk = m0 + j * ca.cbw;
              const int tap = kk / ca.C, c0 = kk - tap * ca.C;
              const int ky = tap / ca.k, kx = tap - ky * ca.k;
              tma_load_4d(sA + s * A_BYTES + j * (64 * ca.cbw * 2), &mapA, &ctl.full[s], c0,
                          kx - ca.p, oy * ca.s - ca.p + ky, im);
            }
#pragma unroll
            for (int j = 0; j < BN / 64; ++j)
              tma_load_2d(sB + s * B_BYTES + j * 8192, &mapB, &ctl.full[s], n0 + 64 * j, k);
            continue;
          }
          if (ca.on) {
            // A: the input box of this filter tap and channel block (zero outside the image)
            const int tap = k / ca.C, c0 = k - tap * ca.C;
            const int ky = tap / ca.k, kx = tap - ky * ca.k;
            tma_load_4d(sA + s * A_BYTES, &mapA, &ctl.full[s], c0, kx - ca.p, oy0 * ca.s - ca.p + ky,
                        img);
            tma_load_2d(sB + s * B_BYTES, &mapB, &ctl.full[s], k, n0);
            continue;
          }
          if (a_mn) {
            tma_load_2d(sA + s * A_BYTES, &mapA, &ctl.full[s], m0, k);
            tma_load_2d(sA + s * A_BYTES + 8192, &mapA, &ctl.full[s], m0 + 64, k);
          } else {
            tma_load_2d(sA + s * A_BYTES, &mapA, &ctl.full[s], k, m0);
          }
          if (b_mn) {
#pragma unroll
            for (int j = 0; j < BN / 64; ++j)
              tma_load_2d(sB + s * B_BYTES + j * 8192, &mapB, &ctl.full[s], n0 + 64 * j, k);
          } else {
            tma_load_2d(sB + s * B_BYTES, &mapB, &ctl.full[s], k, n0);
          }
        }
      }
      ctl.issued = it;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      const uint32_t idesc = fp8 ? f8_idesc(TC_BM, BN) : f16_idesc(TC_BM, BN, a_mn, b_mn);
      const int kstep = ca.on == 1 ? ca.cbw : TC_BK;
      const bool sw64 = ca.on == 1 && ca.cbw == 32;
      const bool a_sw64_mn = ca.on == 2 && ca.cbw == 32;
      uint32_t it = 0, ti = 0;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++ti) {
        const int z = t / (tiles_m * tiles_n);
        const int kbeg = z * kchunk, kend = min(K, kbeg + kchunk);
        const int nkb = (kend - kbeg + kstep - 1) / kstep;
        const uint32_t buf = ti & 1u, bph = (ti >> 1) & 1u;
        if (!mbar_wait(&acc_empty[buf], bph ^ 1u, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t dacc = tmem + buf * BN;
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % stages;
          const uint32_t ph = (it / stages) & 1u;
          if (!mbar_wait(&ctl.full[s], ph, abort, err)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_addr(sA + s * A_BYTES), b0 = smem_addr(sB + s * B_BYTES);
          for (int k = 0; k < kstep / 16; ++k) {
            uint64_t da, db;
            if (sw64) {
              da = sw64_desc(a0 + k * 32);
              db = sw64_desc(b0 + k * 32);
            } else if (a_sw64_mn) {
              da = sw64_mn_desc(a0 + k * 1024);
              db = sw128_mn_desc(b0 + k * 2048);
            } else {
              da = a_mn ? sw128_mn_desc(a0 + k * 2048) : sw128_desc(a0 + k * 32);
              db = b_mn ? sw128_mn_desc(b0 + k * 2048) : sw128_desc(b0 + k * 32);
            }
            const uint32_t acc = (kb | k) ? 1u : 0u;
            tc_mma(dacc, da, db, idesc, acc, fp8);
          }
          asm volatile(
              "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                  smem_addr(&ctl.empty[s]))
              : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_addr(&acc_full[buf]))
            : "memory");
      }
      ctl.consumed = it;
      if (*abort) {
        tc_commit(&ctl.drain);  // arrives once every MMA this thread issued has completed
        mbar_drain_wait(&ctl.drain, 0u);
      }
    }
  } else {
    // epilogue warps 2..5: warp w reads TMEM lanes 32 (w % 4) .. +31
    const int q = warp & 3;
    float* stage_out = epi_stage[q];
    // the tensor store reads the staging block through the swizzle of its 1024-byte atom
    const int tma_out = (smem_addr(&epi_stage[0][0]) & 1023u) ? 0 : tma_out_req;
    uint32_t epi_ph = 0;     // phase of this warp's C-load barrier
    bool c_pending = false;  // a C load whose wait ran out (drained at the end)
    const int Mo = trans_out ? N : M, No = trans_out ? M : N;
    // per-tensor scales of E4M3 operands (exactly 1 otherwise)
    const float alpha = (scale_a ? *scale_a : 1.f) * (scale_b ? *scale_b : 1.f);
    uint32_t ti = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++ti) {
      const int tm = t % tiles_m, tn = (t / tiles_m) % tiles_n, z = t / (tiles_m * tiles_n);
      const int m0 = tm * TC_BM, n0 = tn * BN;
      const uint32_t buf = ti & 1u, bph = (ti >> 1) & 1u;
      const bool ok = mbar_wait(&acc_full[buf], bph, abort, err);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row = m0 + q * 32 + lane;
      // halo mode: output row of this lane's tile row, computed once per tile and handed to
      // the row loop by shuffles
      const long long my_orow = halo ? halo_out_row(ca, tm, q * 32 + lane) : 0;
      const int px = rowh ? (q * 32 + lane) % ca.W : 0;  // row halo: this lane's image column
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;  // columns past N: nothing to read or store
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + buf * acc_stride + (uint32_t)c0;
        if (rowh) {
          // out(x) = D_1(x) + D_0(x - 1) + D_2(x + 1), in that order; the neighbours' values
          // come from lanes -1 / +1 of the same image row, zero past the row's ends
          float o[32];
          tmem_ld32(taddr + 32u, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) o[j] = __uint_as_float(r[j]);
          tmem_ld32(taddr, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float v = __shfl_up_sync(0xffffffffu, __uint_as_float(r[j]), 1);
            if (px > 0) o[j] += v;
          }
          tmem_ld32(taddr + 64u, r);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float v = __shfl_down_sync(0xffffffffu, __uint_as_float(r[j]), 1);
            if (px < ca.W - 1) o[j] += v;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(o[j]);
        } else {
          tmem_ld32(taddr, r);
        }
        if (!ok) continue;
        if (tma_out) {
          // tensor-store path (rows of the tile are consecutive output rows, no transposed
          // output): this lane's row of 32 values, formed exactly as the transpose path
          // below forms them -- scale; then for C: + beta C (one fused multiply-add, C read
          // by a tensor load of the same block), + bias, ReLU, output type; split-K
          // partials stay raw -- written to the staging block in the swizzled layout and
          // stored by one tensor copy
          if (c_pending) continue;  // a C load ran out of time: this CTA stores nothing more
          char* sb = reinterpret_cast<char*>(stage_out);
          const bool part = tma_out == 3;
          const int img = rowh ? tm / ca.tpi : 0;
          const int ty = rowh ? (tm - img * ca.tpi) * ca.R * ca.W + q * 32 : m0 + q * 32;
          // the previous tensor store from this block has finished reading it
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
          float cv[32];
          if (beta != 0.f && !part) {
            if (lane == 0) {
              mbar_expect_tx(&epi_bar[q], 4096u);  // fp32 output (the host's condition)
              if (rowh) tma_load_3d(sb, &mapC, &epi_bar[q], n0 + c0, ty, img);
              else tma_load_2d(sb, &mapC, &epi_bar[q], n0 + c0, ty);
            }
            const bool got = __all_sync(0xffffffffu, mbar_wait(&epi_bar[q], epi_ph, abort, err));
            epi_ph ^= 1u;
            if (!got) {
              c_pending = true;  // drained before the kernel ends
              continue;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              const float4 t = *reinterpret_cast<const float4*>(sb + lane * 128 + ((c ^ (lane & 7)) << 4));
              cv[4 * c] = t.x; cv[4 * c + 1] = t.y; cv[4 * c + 2] = t.z; cv[4 * c + 3] = t.w;
            }
            __syncwarp();  // every lane has read its row before the block is rewritten
          }
          const float bl = (bias && !part) ? bias[min(n0 + c0 + lane, N - 1)] : 0.f;
          float x[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            float v = __uint_as_float(r[j]);
            if (fp8) v *= alpha;
            if (!part) {
              if (beta != 0.f) v = __fmaf_rn(beta, cv[j], v);
              v += __shfl_sync(0xffffffffu, bl, j);
              if (relu) v = fmaxf(v, 0.f);
            }
            x[j] = v;
          }
          if (tma_out != 2) {
            // fp32: 128-byte rows, 16-byte chunk c of row l at chunk c ^ (l & 7)
#pragma unroll
            for (int c = 0; c < 8; ++c)
              *reinterpret_cast<float4*>(sb + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                  make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
          } else {
            // bf16: 64-byte rows, 16-byte chunk c of row l at chunk c ^ ((l >> 1) & 3)
#pragma unroll
            for (int c = 0; c < 4; ++c)
              *reinterpret_cast<uint4*>(sb + lane * 64 + ((c ^ ((lane >> 1) & 3)) << 4)) =
                  make_uint4(bf16x2_bits(x[8 * c], x[8 * c + 1]), bf16x2_bits(x[8 * c + 2], x[8 * c + 3]),
                             bf16x2_bits(x[8 * c + 4], x[8 * c + 5]), bf16x2_bits(x[8 * c + 6], x[8 * c + 7]));
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) {
            // row halo: [images, H W, N], the warp's 32 rows are pixels of one image from
            // y0 W + 32 q on (pixels past the image's last one are not written); split-K
            // partials: [splits, M, N]; otherwise [M, N]
            if (rowh) tma_store_3d(&mapC, sb, n0 + c0, ty, img);
            else if (part) tma_store_3d(&mapC, sb, n0 + c0, ty, z);
            else tma_store_2d(&mapC, sb, n0 + c0, ty);
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
          }
          continue;
        }
        if (trans_out) {
          if (row >= M) continue;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = n0 + c0 + j;
            if (col >= N) break;
            float v = __uint_as_float(r[j]) * alpha;
            if (partial) {
              partial[((size_t)z * Mo + col) * No + row] = v;
              continue;
            }
            const size_t o = (size_t)col * ldc + row;
            if (beta != 0.f) v = __fmaf_rn(beta, C[o], v);
            if (bias) v += bias[row];
            if (relu) v = fmaxf(v, 0.f);
            if (c_bf16) ((__nv_bfloat16*)C)[o] = __float2bfloat16_rn(v);
            else C[o] = v;
          }
          continue;
        }
        // transpose through shared memory: lane l then owns column c0 + l of the 32 rows,
        // so every store instruction writes 32 consecutive values of one row
#pragma unroll
        for (int j = 0; j < 32; ++j) stage_out[lane * 32 + (j ^ lane)] = __uint_as_float(r[j]);
        if (fp8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) stage_out[lane * 32 + (j ^ lane)] *= alpha;
        }
        __syncwarp();
        const int col = n0 + c0 + lane;
        const bool cin = col < N;
        const float bv = (bias && cin) ? bias[col] : 0.f;
        if (halo) {
#pragma unroll 1
          for (int i0 = 0; i0 < 32; i0 += 8) {
            float v[8];
            long long orows[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              v[k] = stage_out[(i0 + k) * 32 + (lane ^ (i0 + k))];
              orows[k] = __shfl_sync(0xffffffffu, my_orow, i0 + k);
            }
            if (!cin) continue;
            // accumulated output: the group's eight loads are issued before its stores
            float cv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (beta != 0.f && !partial) {
#pragma unroll
              for (int k = 0; k < 8; ++k)
                if (orows[k] >= 0) cv[k] = C[(size_t)orows[k] * ldc + col];
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const long long orow = orows[k];
              if (orow < 0) continue;
              float x = v[k];
              if (partial) {
                partial[((size_t)z * Mo + orow) * No + col] = x;
                continue;
              }
              const size_t o = (size_t)orow * ldc + col;
              if (beta != 0.f) x = __fmaf_rn(beta, cv[k], x);
              x += bv;
              if (relu) x = fmaxf(x, 0.f);
              if (c_bf16) ((__nv_bfloat16*)C)[o] = __float2bfloat16_rn(x);
              else C[o] = x;
            }
          }
          __syncwarp();
          continue;
        }
        const int nrows = min(32, M - (m0 + q * 32));
        // eight rows at a time: the shared-memory loads of a group are all in flight before
        // its global stores
#pragma unroll 1
        for (int i0 = 0; i0 < 32; i0 += 8) {
          float v[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = stage_out[(i0 + k) * 32 + (lane ^ (i0 + k))];
          if (!cin || i0 >= nrows) continue;
          if (partial) {
            float* pz = partial + ((size_t)z * Mo + m0 + q * 32 + i0) * No + col;
#pragma unroll
            for (int k = 0; k < 8; ++k)
              if (i0 + k < nrows) pz[(size_t)k * No] = v[k];
            continue;
          }
          const size_t o0 = (size_t)(m0 + q * 32 + i0) * ldc + col;
          if (beta != 0.f) {
            float cv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) cv[k] = i0 + k < nrows ? C[o0 + (size_t)k * ldc] : 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __fmaf_rn(beta, cv[k], v[k]);
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            float x = v[k] + bv;
            if (relu) x = fmaxf(x, 0.f);
            if (i0 + k < nrows) {
              if (c_bf16) ((__nv_bfloat16*)C)[o0 + (size_t)k * ldc] = __float2bfloat16_rn(x);
              else C[o0 + (size_t)k * ldc] = x;
            }
          }
        }
        __syncwarp();  // the next chunk rewrites stage_out
      }
      // the accumulator may be overwritten by the next tile
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acc_empty[buf]))
                     : "memory");
      }
      if (!ok) break;
    }
    // every tensor store of this warp has completed before the kernel ends, and a C load
    // whose wait ran out has landed before the shared memory is released
    if (tma_out && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (c_pending) mbar_drain_wait(&epi_bar[q], epi_ph ^ 1u);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (ctl.abort) {  // every role has left its loop: the flag no longer changes
    if (threadIdx.x == 0)
      drain_unconsumed(ctl.full, ctl.consumed, ctl.issued, stages, halo ? &ctl.done : nullptr);
    __syncthreads();
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols));
  }
}

// ---------------------------------------------------------------- host side
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 2-D bf16 tensor [rows, cols] with row stride ld elements, box [box_rows, 64 columns]
static bool make_map(CUtensorMap* m, const void* ptr, int rows, int cols, int ld, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// bf16 [rows, cols] with row stride ld, box [box_rows, box_cols], given swizzle
static bool make_map_sw(CUtensorMap* m, const void* ptr, int rows, int cols, int ld, int box_rows,
                        int box_cols, CUtensorMapSwizzle sw) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The output C as a tensor-store target: fp32 rows (SWIZZLE_128B) or bf16 rows
// (SWIZZLE_64B), boxes of 32 rows x 32 columns. hw > 0: as a 3-D tensor [rows / hw, hw,
// cols] (the row halo stores per image, so a ragged last tile stops at the image's last
// pixel). False when the layout does not allow it (the transpose path stores instead).
static bool make_out_map(CUtensorMap* m, void* C, int rows, int cols, int ldc, int bf16, int hw) {
  auto fn = encode_fn();
  if (!fn) return false;
  const size_t es = bf16 ? 2 : 4;
  if (((uintptr_t)C & 15) || ((size_t)ldc * es) % 16 || cols < 32 || rows < 32) return false;
  const CUtensorMapDataType dt = bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const CUtensorMapSwizzle sw = bf16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  cuuint32_t estr[3] = {1, 1, 1};
  if (hw > 0) {
    if (hw < 32 || rows % hw) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)hw, (cuuint64_t)(rows / hw)};
    cuuint64_t strides[2] = {(cuuint64_t)ldc * es, (cuuint64_t)hw * ldc * es};
    cuuint32_t box[3] = {32u, 32u, 1u};
    return fn(m, dt, 3, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ldc * es};
  cuuint32_t box[2] = {32u, 32u};
  return fn(m, dt, 2, C, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// NHWC bf16 input as a 4-D tensor [C, W, H, N]; one box = the cbw channels of the
// (hi or Ho) x Wo output pixels of a tile, sampled with the convolution stride
static bool make_conv_map(CUtensorMap* m, const void* x, const ConvShape& c, const ConvA& ca) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int ni = (c.Ho * c.Wo >= TC_BM) ? 1 : TC_BM / (c.Ho * c.Wo);
  cuuint64_t dims[4] = {(cuuint64_t)c.C, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
  cuuint64_t strides[3] = {(cuuint64_t)c.C * 2, (cuuint64_t)c.W * c.C * 2,
                           (cuuint64_t)c.H * c.W * c.C * 2};
  cuuint32_t box[4] = {(cuuint32_t)ca.cbw, (cuuint32_t)(c.Wo * c.s), (cuuint32_t)(ca.hi * c.s),
                       (cuuint32_t)ni};
  cuuint32_t estr[4] = {1, (cuuint32_t)c.s, (cuuint32_t)c.s, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            ca.cbw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Halo-mode geometry of a stride-1 'same' convolution (odd k, p = k / 2, C = 32 or a
// multiple of 64). Fills ca when non-null; false when the shape is not covered.
static int halo_bn(int cout) { return cout <= 32 ? 32 : cout <= 64 ? 64 : cout <= 128 ? 128 : 0; }
constexpr size_t TC_HALO_WEIGHTS_MAX = 96 * 1024;  // resident weights of one halo convolution

// Taken for 32-channel inputs, where the 4-D gather moves 64-byte rows once per filter tap;
// with 64 or more channels the resident weights leave room for one CTA per SM and the
// gather path is faster.
static bool halo_geom(const ConvShape& c, ConvA* ca) {
  if (c.s != 1 || c.k % 2 == 0 || c.p != c.k / 2 || c.C != 32) return false;
  if (c.Ho != c.H || c.Wo != c.W) return false;
  const int bn = halo_bn(c.Cout);
  if (!bn) return false;
  const size_t wbytes = (size_t)bn * c.k * c.k * c.C * 2;
  if (wbytes > TC_HALO_WEIGHTS_MAX) return false;
  if (c.k == 3 && bn == 32 && (c.W == 8 || c.W == 16 || c.W == 32) && c.H >= TC_BM / c.W) {
    // row halo: R whole rows per tile, the box R + 2 rows of W pixels (64 bytes each)
    const int R = TC_BM / c.W;
    const uint32_t box = (uint32_t)((R + 2) * c.W * 64);
    if (ca) {
      ca->on = 4;
      ca->C = 32; ca->cbw = 32; ca->k = 3; ca->s = 1; ca->p = 1;
      ca->Ho = c.Ho; ca->Wo = c.Wo;
      ca->N = c.N; ca->H = c.H; ca->W = c.W; ca->Wp = c.W; ca->Hh = c.H;
      ca->ni = 0; ca->tpi = (c.H + R - 1) / R; ca->rows_box = R + 2; ca->R = R;
      ca->tiles_m = c.N * ca->tpi;
      ca->halo_bytes = (box + 1023) / 1024 * 1024;
      ca->box_bytes = box;
    }
    return true;
  }
  const int Wp = c.W + 2 * c.p, Hh = c.H + 2 * c.p, per = Hh * Wp;
  const int cbw = c.C == 32 ? 32 : 64, rb = cbw * 2;
  int ni, tpi, rows_box, rows_need;
  if (per <= TC_BM) {
    ni = TC_BM / per;
    tpi = 1;
    rows_box = Hh;
    rows_need = TC_BM + (c.k - 1) * (Wp + 1);
  } else {
    ni = 0;
    tpi = (c.H * Wp + TC_BM - 1) / TC_BM;
    // rows of the box: enough for the farthest row read from the largest in-row offset
    rows_box = (Wp - 1 + TC_BM - 1 + (c.k - 1) * (Wp + 1)) / Wp + 1;
    rows_need = Wp - 1 + TC_BM + (c.k - 1) * (Wp + 1);
  }
  if (Wp > 256 || rows_box > 256) return false;
  const int box_rows = rows_box * Wp * (ni ? ni : 1);
  const int rows_alloc = std::max(box_rows, rows_need);
  const uint32_t halo_bytes = (uint32_t)(((size_t)rows_alloc * rb + 1023) / 1024 * 1024);
  if (2 * (size_t)halo_bytes + wbytes + 1024 > TC_SMEM_MAX) return false;
  if (ca) {
    ca->on = 3;
    ca->C = c.C; ca->cbw = cbw; ca->k = c.k; ca->s = 1; ca->p = c.p;
    ca->Ho = c.Ho; ca->Wo = c.Wo;
    ca->N = c.N; ca->H = c.H; ca->W = c.W; ca->Wp = Wp; ca->Hh = Hh;
    ca->ni = ni; ca->tpi = tpi; ca->rows_box = rows_box;
    ca->tiles_m = ni ? (c.N + ni - 1) / ni : c.N * tpi;
    ca->halo_bytes = halo_bytes;
    ca->box_bytes = (uint32_t)box_rows * rb;
  }
  return true;
}

// shared memory of a halo-mode launch: the box ring and the resident weights
static size_t halo_smem(const ConvA& ca, int bn, int stages) {
  return (size_t)stages * ca.halo_bytes + (size_t)bn * ca.k * ca.k * ca.C * 2 + 1024;
}

// NHWC bf16 input as [C, W, H, N]; one box = the halo of a tile: cbw channels x Wp columns
// (from x = -p; the row halo: W columns from x = 0) x rows_box rows x (ni or 1) images,
// zero outside the image
static bool make_halo_map(CUtensorMap* m, const void* x, const ConvShape& c, const ConvA& ca) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[4] = {(cuuint64_t)c.C, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
  cuuint64_t strides[3] = {(cuuint64_t)c.C * 2, (cuuint64_t)c.W * c.C * 2,
                           (cuuint64_t)c.H * c.W * c.C * 2};
  cuuint32_t box[4] = {(cuuint32_t)ca.cbw, (cuuint32_t)ca.Wp, (cuuint32_t)ca.rows_box,
                       (cuuint32_t)(ca.ni ? ca.ni : 1)};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            ca.cbw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// weight-gradient gather: 64-pixel K blocks of whole output rows (or whole images)
static bool convw_geom(const ConvShape& c, int* hi, int* ni) {
  if (c.Wo < 1 || c.Ho < 1 || 64 % c.Wo) return false;
  const int pix = c.Ho * c.Wo;
  if (pix >= 64) {
    *hi = 64 / c.Wo;
    *ni = 1;
    if (c.Ho % *hi) return false;
  } else {
    if (64 % pix) return false;
    *hi = c.Ho;
    *ni = 64 / pix;
  }
  return *hi * c.s <= 256 && c.Wo * c.s <= 256;
}

static bool make_convw_map(CUtensorMap* m, const void* x, const ConvShape& c, int cbw) {
  auto fn = encode_fn();
  int hi = 0, ni = 0;
  if (!fn || !convw_geom(c, &hi, &ni)) return false;
  cuuint64_t dims[4] = {(cuuint64_t)c.C, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
  cuuint64_t strides[3] = {(cuuint64_t)c.C * 2, (cuuint64_t)c.W * c.C * 2,
                           (cuuint64_t)c.H * c.W * c.C * 2};
  cuuint32_t box[4] = {(cuuint32_t)cbw, (cuuint32_t)(c.Wo * c.s), (cuuint32_t)(hi * c.s),
                       (cuuint32_t)ni};
  cuuint32_t estr[4] = {1, (cuuint32_t)c.s, (cuuint32_t)c.s, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE,
            cbw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gemm_convw_supported(const ConvShape& c, const void* input, const void* dz) {
  if (!encode_fn()) return false;
  if (!(c.C == 32 || (c.C > 0 && c.C % 64 == 0))) return false;
  if (((uintptr_t)input & 15) || ((uintptr_t)dz & 15)) return false;
  if (c.k < 1 || c.s < 1 || c.s > 8 || c.N < 1) return false;
  int hi = 0, ni = 0;
  return convw_geom(c, &hi, &ni);
}

// the 4-D gather path: whole output rows per 128-pixel tile (or whole images per tile)
static bool gather_ok(const ConvShape& c) {
  if (c.C % 32 || c.C <= 0) return false;
  if (TC_BM % c.Wo || c.Wo * c.s > 256) return false;
  const int pix = c.Ho * c.Wo;
  if (pix >= TC_BM) {
    const int hi = TC_BM / c.Wo;
    if (c.Ho % hi || hi * c.s > 256) return false;
  } else {
    if (TC_BM % pix || c.Ho * c.s > 256) return false;
  }
  return c.k >= 1 && c.s >= 1 && c.s <= 8;
}

bool gemm_conv_supported(const ConvShape& c, const void* input) {
  if (!encode_fn() || ((uintptr_t)input & 15)) return false;
  return halo_geom(c, nullptr) || gather_ok(c);
}

template <int BN>
static size_t tc_smem(int stages, int kslot) {
  return (size_t)stages * (TC_BM + BN) * kslot * 2 + 1024;
}
static size_t tc_smem_bn(int bn, int stages, int kslot) {
  return bn == 128 ? tc_smem<128>(stages, kslot) : tc_smem<64>(stages, kslot);
}
// deepest ring within a budget (two CTAs per SM for BN = 64, one for BN = 128)
static int ring_for(int bn, int kslot) {
  const size_t budget = bn == 64 ? TC_SMEM_TWO_PER_SM : TC_SMEM_MAX;
  int st = TC_STAGES;
  while (st > 2 && tc_smem_bn(bn, st, kslot) > budget) --st;
  return st;
}

bool gemm_tc_supported(const GemmDesc& d) {
  if (!encode_fn()) return false;
  if (d.K < 16 || d.M < 1 || d.N < 1) return false;
  if ((d.lda % 8) || (d.ldb % 8)) return false;  // 16-byte row strides for TMA
  if (((uintptr_t)d.A & 15) || ((uintptr_t)d.B & 15)) return false;
  if ((int64_t)d.M > (1ll << 31) - 1 || (int64_t)d.N > (1ll << 31) - 1) return false;
  return true;
}

struct TcCfg {
  int bn = 64;       // N tile: 32 (halo convolutions), 64 or 128
  int stages = 3;    // shared-memory ring depth: 2..TC_STAGES
  int split = 0;     // 0: split K when the grid would be short of SMs; 1: never split
  int halo = 0;      // convolution through the halo path (1) or the 4-D gather (0)
};

struct TcTuner {
  bool on = true;
  std::map<std::tuple<int, int, int, int, int, int, int>, TcCfg> table;
  void* scratch = nullptr;  // trial output
  size_t scratch_bytes = 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
};

TcTuner* tc_tuner_create(size_t scratch_bytes) {
  TcTuner* t = new TcTuner();
  if (cudaMalloc(&t->scratch, scratch_bytes) != cudaSuccess) {
    t->scratch = nullptr;
    scratch_bytes = 0;
  }
  t->scratch_bytes = scratch_bytes;
  cudaEventCreate(&t->e0);
  cudaEventCreate(&t->e1);
  return t;
}
void tc_tuner_destroy(TcTuner* t) {
  if (!t) return;
  if (t->scratch) cudaFree(t->scratch);
  if (t->e0) cudaEventDestroy(t->e0);
  if (t->e1) cudaEventDestroy(t->e1);
  delete t;
}
void tc_tuner_enable(TcTuner* t, bool on) { if (t) t->on = on; }
int64_t tc_tuner_shapes(const TcTuner* t) { return t ? (int64_t)t->table.size() : 0; }

// table image: int32 words {magic, version, count} then count records of 7 key words and
// 4 configuration words (N tile, ring depth, split policy, halo path)
static const int32_t kTuneMagic = 0x54544444, kTuneVersion = 6, kTuneRec = 11;

size_t tc_tuner_export(const TcTuner* t, void* buf, size_t cap) {
  const size_t cnt = t ? t->table.size() : 0;
  const size_t need = (3 + cnt * kTuneRec) * sizeof(int32_t);
  if (!buf || cap < need) return need;
  int32_t* w = (int32_t*)buf;
  w[0] = kTuneMagic; w[1] = kTuneVersion; w[2] = (int32_t)cnt;
  int32_t* r = w + 3;
  if (t)
    for (const auto& kv : t->table) {
      const auto& k = kv.first;
      r[0] = std::get<0>(k); r[1] = std::get<1>(k); r[2] = std::get<2>(k); r[3] = std::get<3>(k);
      r[4] = std::get<4>(k); r[5] = std::get<5>(k); r[6] = std::get<6>(k);
      r[7] = kv.second.bn; r[8] = kv.second.stages; r[9] = kv.second.split;
      r[10] = kv.second.halo;
      r += kTuneRec;
    }
  return need;
}

int tc_tuner_import(TcTuner* t, const void* buf, size_t size) {
  if (!t) { set_error("autotune import: no tuner (precision 0)"); return DDPPO_E_CONFIG; }
  const int32_t* w = (const int32_t*)buf;
  if (!buf || size < 3 * sizeof(int32_t) || w[0] != kTuneMagic || w[1] != kTuneVersion || w[2] < 0 ||
      size != (3 + (size_t)w[2] * kTuneRec) * sizeof(int32_t)) {
    set_error("autotune import: not a tuning table image of this version");
    return DDPPO_E_CONFIG;
  }
  const int32_t* r = w + 3;
  for (int32_t i = 0; i < w[2]; ++i, r += kTuneRec) {
    TcCfg c;
    c.bn = r[7]; c.stages = r[8]; c.split = r[9]; c.halo = r[10];
    if ((c.bn != 32 && c.bn != 64 && c.bn != 128) || c.stages < 2 || c.stages > TC_STAGES - 2 ||
        (c.split != 0 && c.split != 1) || (c.halo != 0 && c.halo != 1)) {
      set_error("autotune import: bad configuration record");
      return DDPPO_E_CONFIG;
    }
    t->table[std::make_tuple(r[0], r[1], r[2], r[3], r[4], r[5], r[6])] = c;
  }
  return DDPPO_OK;
}

static int kslot_of(const GemmDesc& d) {
  if (d.conv) return d.conv->C % 64 == 0 ? 64 : 32;
  return TC_BK;
}

static TcCfg default_cfg(int N, int kslot) {
  TcCfg c;
  c.bn = N > 64 ? 128 : 64;
  c.stages = std::min(ring_for(c.bn, kslot), c.bn == 64 ? 3 : 4);
  c.split = 0;
  return c;
}

template <int BN>
static int launch_tc(const CUtensorMap& ma, const CUtensorMap& mb, int M, int N, int K,
                     const GemmDesc& d, int trans, int a_mn, int b_mn, const GemmWorkspace& ws,
                     const TcCfg& cfg, const ConvA& ca, cudaStream_t s) {
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    DDPPO_CHECK_CUDA(cudaFuncSetAttribute(gemm_tc_kernel<BN>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)TC_SMEM_MAX));
    attr_done[dev] = true;
  }
  const bool halo = ca.on >= 3;
  const int gm = halo ? ca.tiles_m : (M + TC_BM - 1) / TC_BM, gn = (N + BN - 1) / BN;
  const int tiles = gm * gn;
  // split-K: over K elements, or over channel blocks in the halo mode (every block runs all
  // filter taps)
  const int kstep = (ca.on == 1 || halo) ? ca.cbw : TC_BK;
  const int Ksplit = halo ? ca.C : K;
  const size_t smem = halo ? halo_smem(ca, BN, cfg.stages) : tc_smem<BN>(cfg.stages, kstep);
  if (smem > TC_SMEM_MAX || cfg.stages < 2 || cfg.stages > TC_STAGES - 2) {
    set_error("gemm_tc: ring depth exceeds shared memory");
    return DDPPO_E_CONFIG;
  }
  const int per_sm = smem <= TC_SMEM_TWO_PER_SM ? 2 : 1;
  // split K until every resident CTA slot has a tile
  int splits = 1;
  const int target = ws.num_sms * per_sm;
  if (cfg.split == 0 && tiles < target && (halo ? Ksplit >= 2 * kstep : K >= 8 * TC_BK)) {
    splits = min((target + tiles - 1) / tiles, halo ? Ksplit / kstep : K / (4 * TC_BK));
    const size_t per = (size_t)d.M * d.N;
    splits = (int)min((size_t)splits, ws.partial_elems / max(per, (size_t)1));
    if (splits < 2) splits = 1;
  }
  int kchunk = (Ksplit + splits - 1) / splits;
  kchunk = (kchunk + kstep - 1) / kstep * kstep;
  splits = (Ksplit + kchunk - 1) / kchunk;
  float* partial = splits > 1 ? ws.partial : nullptr;
  // persistent grid: one CTA per SM (two where shared memory allows), each walking tiles
  // with stride gridDim.x; the ring streams across tile boundaries
  const int stages = cfg.stages;
  const int ntiles = gm * gn * splits;
  const int grid = min(ntiles, ws.num_sms * per_sm);
  // tensor-store epilogue: whole output rows per tile row (plain, 4-D gather and row-halo
  // tiles), into C (beta C read by a tensor load of each block) or into split-K partials
  CUtensorMap mc;
  memset(&mc, 0, sizeof(mc));
  int tma_out = 0;
  if (tma_epilogue_enabled() && !trans && (ca.on == 0 || ca.on == 1 || ca.on == 4)) {
    if (partial) {
      if (ca.on != 4 && make_out_map(&mc, partial, splits * M, N, N, 0, M)) tma_out = 3;
    } else if ((d.beta == 0.f || !d.c_bf16) &&  // C is read back (beta != 0) in fp32 only
               make_out_map(&mc, d.C, M, N, d.ldc, d.c_bf16, ca.on == 4 ? ca.H * ca.W : 0)) {
      tma_out = d.c_bf16 ? 2 : 1;
    }
  }
  ::ddppo::launch_k(gemm_tc_kernel<BN>, grid, TC_PTHREADS, smem, s,
      ma, mb, M, N, K, kchunk, (float*)d.C, d.ldc, d.c_bf16, d.beta, d.bias, d.relu, trans,
      partial, ws.err, a_mn, b_mn, stages, gm, gn, splits, ca, d.fp8, d.scale_a, d.scale_b, mc,
      tma_out);
  DDPPO_CHECK_LAUNCH();
  if (partial)
    DDPPO_TRY(launch_splitk_reduce(d.M, d.N, splits, partial, (float*)d.C, d.ldc, d.c_bf16, d.beta,
                                   d.bias, d.relu, s));
  return DDPPO_OK;
}

static int run_cfg(const GemmDesc& d, const GemmWorkspace& ws, const TcCfg& cfg, cudaStream_t s) {
  if (d.convw) {
    // computed transposed: M' = (tap, channel) rows gathered from the input (MN-major),
    // N' = output channels from dz [pixels][cout] (MN-major); stored as dW[co][kk]
    const ConvShape& c = *d.convw;
    ConvA ca;
    ca.on = 2;
    ca.C = c.C;
    ca.cbw = c.C == 32 ? 32 : 64;
    ca.k = c.k; ca.s = c.s; ca.p = c.p; ca.Ho = c.Ho; ca.Wo = c.Wo;
    CUtensorMap ma, mb;
    if (!make_convw_map(&ma, d.B, c, ca.cbw) || !make_map(&mb, d.A, d.K, d.M, d.lda, TC_BK)) {
      set_error("gemm_tc: weight-gradient tensor map encoding failed");
      return DDPPO_E_CUDA;
    }
    if (cfg.bn == 128) return launch_tc<128>(ma, mb, d.N, d.M, d.K, d, 1, 1, 1, ws, cfg, ca, s);
    return launch_tc<64>(ma, mb, d.N, d.M, d.K, d, 1, 1, 1, ws, cfg, ca, s);
  }
  if (d.conv && (cfg.halo || !gather_ok(*d.conv)) && halo_geom(*d.conv, nullptr)) {
    const ConvShape& c = *d.conv;
    ConvA ca;
    halo_geom(c, &ca);
    const CUtensorMapSwizzle sw = ca.cbw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    const int bn = halo_bn(c.Cout);  // one N tile: the weights stay resident
    if (c.Cout != d.N) {
      set_error("gemm_tc: convolution output channels disagree with N");
      return DDPPO_E_CONFIG;
    }
    CUtensorMap ma, mb;
    if (!make_halo_map(&ma, d.A, c, ca) || !make_map_sw(&mb, d.B, d.N, d.K, d.ldb, bn, ca.cbw, sw)) {
      set_error("gemm_tc: halo convolution tensor map encoding failed");
      return DDPPO_E_CUDA;
    }
    if (bn == 32) return launch_tc<32>(ma, mb, d.M, d.N, d.K, d, 0, 0, 0, ws, cfg, ca, s);
    if (bn == 128) return launch_tc<128>(ma, mb, d.M, d.N, d.K, d, 0, 0, 0, ws, cfg, ca, s);
    return launch_tc<64>(ma, mb, d.M, d.N, d.K, d, 0, 0, 0, ws, cfg, ca, s);
  }
  if (d.conv) {
    const ConvShape& c = *d.conv;
    ConvA ca;
    ca.on = 1;
    ca.C = c.C;
    ca.cbw = c.C % 64 == 0 ? 64 : 32;
    ca.k = c.k; ca.s = c.s; ca.p = c.p; ca.Ho = c.Ho; ca.Wo = c.Wo;
    ca.hi = c.Ho * c.Wo >= TC_BM ? TC_BM / c.Wo : c.Ho;
    const CUtensorMapSwizzle sw = ca.cbw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap ma, mb;
    if (!make_conv_map(&ma, d.A, c, ca) ||
        !make_map_sw(&mb, d.B, d.N, d.K, d.ldb, cfg.bn, ca.cbw, sw)) {
      set_error("gemm_tc: convolution tensor map encoding failed");
      return DDPPO_E_CUDA;
    }
    if (cfg.bn == 128) return launch_tc<128>(ma, mb, d.M, d.N, d.K, d, 0, 0, 0, ws, cfg, ca, s);
    return launch_tc<64>(ma, mb, d.M, d.N, d.K, d, 0, 0, 0, ws, cfg, ca, s);
  }
  // swap A and B when M is small: the MMA's 128-row side then covers N
  const bool swap = d.M < TC_BM && d.N > d.M;
  const void* A = swap ? d.B : d.A;
  const void* Bm = swap ? d.A : d.B;
  const int lda = swap ? d.ldb : d.lda, ldb = swap ? d.lda : d.ldb;
  const int a_mn = swap ? d.b_t : d.a_t, b_mn = swap ? d.a_t : d.b_t;
  const int M = swap ? d.N : d.M, N = swap ? d.M : d.N;
  const int BN = cfg.bn;
  CUtensorMap ma, mb;
  // K-major operand: [rows = M|N, cols = K] boxes of 128|BN rows x 64 K;
  // MN-major operand: [rows = K, cols = M|N] boxes of 64 K rows x 64 columns
  const bool okA = a_mn ? make_map(&ma, A, d.K, M, lda, TC_BK) : make_map(&ma, A, M, d.K, lda, TC_BM);
  const bool okB = b_mn ? make_map(&mb, Bm, d.K, N, ldb, TC_BK) : make_map(&mb, Bm, N, d.K, ldb, BN);
  if (!okA || !okB) {
    set_error("gemm_tc: tensor map encoding failed");
    return DDPPO_E_CUDA;
  }
  const ConvA none;
  if (BN == 128) return launch_tc<128>(ma, mb, M, N, d.K, d, swap ? 1 : 0, a_mn, b_mn, ws, cfg, none, s);
  return launch_tc<64>(ma, mb, M, N, d.K, d, swap ? 1 : 0, a_mn, b_mn, ws, cfg, none, s);
}

// time every candidate on a scratch output (beta = 0, same operands); keep the fastest
static TcCfg tune(const GemmDesc& d, const GemmWorkspace& ws, TcTuner& t, cudaStream_t s) {
  const bool swap = d.convw || (!d.conv && d.M < TC_BM && d.N > d.M);
  const int Nk = swap ? d.M : d.N;
  const int kslot = kslot_of(d);
  const bool hal = d.conv && halo_geom(*d.conv, nullptr);
  const bool gat = !d.conv || gather_ok(*d.conv);
  std::vector<TcCfg> cands;
  if (gat)
    for (int bn : {64, 128}) {
      if (bn == 128 && Nk <= 64) continue;
      for (int st : {2, 3, 4}) {
        if (tc_smem_bn(bn, st, kslot) > TC_SMEM_MAX) continue;
        for (int sp = 0; sp <= 1; ++sp) {
          TcCfg c;
          c.bn = bn; c.stages = st; c.split = sp;
          cands.push_back(c);
        }
      }
    }
  if (hal)
    for (int st : {2, 3, 4})
      for (int sp = 0; sp <= 1; ++sp) {
        TcCfg c;
        c.bn = halo_bn(d.conv->Cout); c.stages = st; c.split = sp; c.halo = 1;
        cands.push_back(c);
      }
  GemmDesc trial = d;
  trial.C = t.scratch;
  trial.ldc = d.N;
  trial.beta = 0.f;
  TcCfg best = default_cfg(Nk, kslot);
  if (hal && !gat) {
    best.bn = halo_bn(d.conv->Cout);
    best.stages = 2;
    best.halo = 1;
  }
  float best_ms = 1e30f;
  for (const TcCfg& c : cands) {
    if (run_cfg(trial, ws, c, s) != DDPPO_OK) continue;  // warm-up
    cudaEventRecord(t.e0, s);
    for (int r = 0; r < 3; ++r) run_cfg(trial, ws, c, s);
    cudaEventRecord(t.e1, s);
    if (cudaEventSynchronize(t.e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.e0, t.e1);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  return best;
}

int gemm_tc(const GemmDesc& d, const GemmWorkspace& ws, cudaStream_t s) {
  const bool swap = d.convw || (!d.conv && d.M < TC_BM && d.N > d.M);
  TcCfg cfg = default_cfg(swap ? d.M : d.N, kslot_of(d));
  ConvA hca;
  if (d.conv && halo_geom(*d.conv, &hca) && (hca.on == 4 || !gather_ok(*d.conv))) {
    const ConvA& ca = hca;
    cfg.halo = 1;
    cfg.bn = halo_bn(d.conv->Cout);
    cfg.stages = 2;  // halo boxes in flight: as many as fit two CTAs per SM, else 2
    for (int st = 4; st > 2; --st)
      if (halo_smem(ca, cfg.bn, st) <= TC_SMEM_TWO_PER_SM) { cfg.stages = st; break; }
  }
  TcTuner* t = ws.tuner;
  if (t && t->on) {
    const ConvShape* cv = d.conv ? d.conv : d.convw;
    const int mode = d.a_t * 2 + d.b_t + (d.conv ? 4 : 0) + (d.convw ? 128 : 0) +
                     (cv ? 8 * cv->s + 256 * cv->Wo + 65536 * cv->k : 0);
    const auto key = std::make_tuple(d.M, d.N, d.K, mode, d.c_bf16 + 2 * d.fp8,
                                     d.beta != 0.f ? 1 : 0, d.lda * 8 + d.ldb);
    auto it = t->table.find(key);
    if (it != t->table.end()) {
      cfg = it->second;
    } else {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(s, &cs);
      const size_t need = (size_t)d.M * d.N * (d.c_bf16 ? 2 : 4);
      if (cs == cudaStreamCaptureStatusNone && t->scratch && need <= t->scratch_bytes) {
        cfg = tune(d, ws, *t, s);
        t->table[key] = cfg;
      }
    }
  }
  return run_cfg(d, ws, cfg, s);
}

// ---------------------------------------------------------------- halo weight gradient
// Weight gradient of a 3x3 / stride-1 / pad-1 convolution of a 32-channel input into 32
// output channels (the first ResNet stage):
//   dW[co, (ky, kx, c)] = sum over output pixels a of dz[a, co] x[a + (ky - 1, kx - 1), c].
// Work unit: RB whole rows of one image, as Wp = W + 2 "anchors" per row (anchors x >= W
// carry dz = 0: the dz box reads past the row end, where TMA fills zeros). Per unit one box
// of dz (RB rows x Wp) and one box of the input with its halo (RB + 3 rows x Wp, from
// x = -1, y = y0 - 1, plus one row) are staged, both 64-byte swizzled, rows = anchors. Per 16-anchor
// K step and filter row ky one MMA (M = 128, N = 32) computes the three kx taps at once:
// the A operand is MN-major (channels contiguous) and its four 32-channel atoms sit one
// 64-byte row apart (leading byte offset 64), so atom j reads the input shifted by j
// anchors -- tap kx = j (the fourth is discarded). Three TMEM accumulators (ky) of 32
// columns collect every unit a CTA takes; each CTA writes its partial sums once and a
// fixed-order reduction adds the CTAs.
constexpr int WH_THREADS = 128;
constexpr int WH_STAGES = 3;

__device__ __forceinline__ uint64_t sw64_mn_desc_lbo(uint32_t saddr, uint32_t lbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

__global__ void __launch_bounds__(WH_THREADS, 1)
    wgrad_halo_kernel(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapDZ,
                      int Wp, int RB, int nrb, int nunits, uint32_t x_bytes, uint32_t dz_bytes,
                      uint32_t x_stride, uint32_t dz_stride, int stages, float* __restrict__ part,
                      int32_t* err) {
  extern __shared__ __align__(1024) uint8_t dyn[];
  __shared__ uint64_t full[WH_STAGES], empty[WH_STAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ uint32_t n_issued, n_consumed;  // ring stages loaded / waited for (drain)
  uint8_t* base = (uint8_t*)(((uintptr_t)dyn + 1023) & ~(uintptr_t)1023);
  uint8_t* sX = base;
  uint8_t* sD = base + stages * x_stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  volatile int* abort = &abort_flag;
  if (threadIdx.x == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    n_issued = 0;
    n_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_base)),
                 "r"(128));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  DDPPO_PDL_ENTRY();  // after the barrier set-up and the tensor-memory allocation
  const uint32_t tmem = tmem_base;
  const int kq = RB * Wp / 16;
  const bool has_work = (int)blockIdx.x < nunits;

  if (warp == 0 && lane == 0) {
    uint32_t it = 0;
    for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x, ++it) {
      const int s = it % stages;
      if (!mbar_wait(&empty[s], ((it / stages) & 1u) ^ 1u, abort, err)) break;
      const int img = u / nrb, y0 = (u - img * nrb) * RB;
      mbar_expect_tx(&full[s], x_bytes + dz_bytes);
      tma_load_4d(sX + s * x_stride, &mapX, &full[s], 0, -1, y0 - 1, img);
      tma_load_4d(sD + s * dz_stride, &mapDZ, &full[s], 0, 0, y0, img);
    }
    n_issued = it;
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = f16_idesc(TC_BM, 32, 1, 1);
    uint32_t it = 0;
    for (int u = blockIdx.x; u < nunits && !*abort; u += gridDim.x, ++it) {
      const int s = it % stages;
      if (!mbar_wait(&full[s], (it / stages) & 1u, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t x0 = smem_addr(sX + s * x_stride), d0 = smem_addr(sD + s * dz_stride);
      for (int k = 0; k < kq; ++k) {
        const uint64_t db = sw64_mn_desc_lbo(d0 + (uint32_t)k * 16 * 64, 4096);
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const uint64_t da = sw64_mn_desc_lbo(x0 + (uint32_t)(ky * Wp + k * 16) * 64, 64);
          const uint32_t acc = (it | k) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + ky * 32),
              "l"(da), "l"(db), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&empty[s]))
          : "memory");
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&done))
        : "memory");
    n_consumed = it;
    // after an abort the epilogue no longer waits for `done`; this thread does, so that
    // every MMA it issued has completed before the accumulators are freed
    if (*abort) mbar_drain_wait(&done, 0u);
  }
  __syncwarp();
  // epilogue: warp w holds TMEM rows 32 w .. 32 w + 31 = tap kx = w, channel c = lane
  const bool ok = has_work ? mbar_wait(&done, 0u, abort, err) : true;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp < 3) {
#pragma unroll 1
    for (int ky = 0; ky < 3; ++ky) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ky * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
          "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
            "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
            "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
            "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float* dst = part + ((((size_t)blockIdx.x * 3 + ky) * 3 + warp) * 32 + lane) * 32;
#pragma unroll
      for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(dst + j) =
            (has_work && ok) ? make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                           __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]))
                             : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (abort_flag) {  // uniform: no thread writes it after the barrier
    if (threadIdx.x == 0) drain_unconsumed(full, n_consumed, n_issued, stages, nullptr);
    __syncthreads();
  }
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
  }
}

// dw[co, (ky*3 + kx)*32 + c] = beta dw + sum over CTAs (in order) of part[cta][ky][kx][c][co]
__global__ void wgrad_halo_reduce_kernel(const float* __restrict__ part, int nctas, float* __restrict__ dw,
                                         int ldw, float beta) {
  DDPPO_PDL_ENTRY();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 32 * 288) return;
  const int co = i / 288, kk = i - co * 288;
  const int tap = kk / 32, c = kk - tap * 32;
  const int ky = tap / 3, kx = tap - ky * 3;
  float v = 0.f;
  for (int t = 0; t < nctas; ++t) v += part[((((size_t)t * 3 + ky) * 3 + kx) * 32 + c) * 32 + co];
  const size_t o = (size_t)co * ldw + kk;
  dw[o] = beta != 0.f ? beta * dw[o] + v : v;
}

// unit rows (RB), anchor pitch (Wp), stage strides and ring depth of the halo weight
// gradient; false when the shape is not covered or two stages do not fit
struct WgradHalo {
  int RB = 0, Wp = 0, stages = 0;
  uint32_t x_bytes = 0, dz_bytes = 0, x_stride = 0, dz_stride = 0;
  size_t smem = 0;
};
static bool wgrad_halo_geom(const ConvShape& c, WgradHalo* g) {
  if (c.C != 32 || c.Cout != 32 || c.k != 3 || c.s != 1 || c.p != 1 || c.Ho != c.H || c.Wo != c.W)
    return false;
  g->Wp = c.W + 2;
  if (g->Wp > 256) return false;
  int r = 1;
  while ((r * g->Wp) % 16 || r * g->Wp < 128) ++r;
  if (r + 3 > 256) return false;
  g->RB = r;
  // input box: the unit's rows, the filter halo above and below, and one more row -- the
  // tap atoms of the last K step read up to 3 anchors past the halo rows, and those
  // anchors (dz = 0 there) must meet finite values, never stale shared memory
  g->x_bytes = 64u * g->Wp * (r + 3);
  g->dz_bytes = 64u * g->Wp * r;
  g->x_stride = (g->x_bytes + 1023) / 1024 * 1024;
  g->dz_stride = (g->dz_bytes + 1023) / 1024 * 1024;
  for (int st = WH_STAGES; st >= 2; --st) {
    g->stages = st;
    g->smem = (size_t)st * (g->x_stride + g->dz_stride) + 1024;
    if (g->smem <= TC_SMEM_MAX) return true;
  }
  return false;
}

bool conv_wgrad_halo_ok(const ConvShape& c, const void* x, const void* dz) {
  WgradHalo g;
  return encode_fn() && !((uintptr_t)x & 15) && !((uintptr_t)dz & 15) && wgrad_halo_geom(c, &g);
}

// The paths and staging geometry a convolution and its weight gradient take (host only,
// no CUDA call): plan[0] 4-D gather forward path; plan[1] halo forward path, then its
// pitch Wp, padded height Hh, images per tile ni (0: tiles within one image), tiles per
// image tpi, box rows per image rows_box, rows allocated per ring stage, rows the box
// delivers, tiles; plan[10] 4-D gather weight gradient; plan[11] halo weight gradient,
// then unit rows RB, pitch Wp, input box rows, dz box rows, ring depth, shared memory
// bytes. 18 words.
void conv_plan(const ConvShape& c, int32_t* plan) {
  for (int i = 0; i < 18; ++i) plan[i] = 0;
  plan[0] = gather_ok(c) ? 1 : 0;
  ConvA ca;
  if (halo_geom(c, &ca)) {
    const int rb = ca.cbw * 2;
    plan[1] = ca.on == 4 ? 2 : 1;
    plan[2] = ca.Wp; plan[3] = ca.Hh; plan[4] = ca.ni; plan[5] = ca.tpi;
    plan[6] = ca.rows_box;
    plan[7] = (int32_t)(ca.halo_bytes / rb);
    plan[8] = (int32_t)(ca.box_bytes / rb);
    plan[9] = ca.tiles_m;
  }
  int hi = 0, ni = 0;
  plan[10] = ((c.C == 32 || (c.C > 0 && c.C % 64 == 0)) && c.k >= 1 && c.s >= 1 && c.s <= 8 &&
              c.N >= 1 && convw_geom(c, &hi, &ni)) ? 1 : 0;
  WgradHalo g;
  if (wgrad_halo_geom(c, &g)) {
    plan[11] = 1;
    plan[12] = g.RB; plan[13] = g.Wp;
    plan[14] = (int32_t)(g.x_bytes / (64u * g.Wp));
    plan[15] = (int32_t)(g.dz_bytes / (64u * g.Wp));
    plan[16] = g.stages;
    plan[17] = (int32_t)g.smem;
  }
}

int conv_wgrad_halo(const ConvShape& c, const void* x, const void* dz, float* dw, int ldw, float beta,
                    const GemmWorkspace& ws, cudaStream_t s) {
  WgradHalo g;
  if (!wgrad_halo_geom(c, &g)) {
    set_error("wgrad_halo: unsupported shape");
    return DDPPO_E_CONFIG;
  }
  const int RB = g.RB, Wp = g.Wp;
  auto fn = encode_fn();
  CUtensorMap mx, md;
  cuuint64_t dims[4] = {32, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.N};
  cuuint64_t strides[3] = {64, (cuuint64_t)c.W * 64, (cuuint64_t)c.H * c.W * 64};
  cuuint32_t boxx[4] = {32, (cuuint32_t)Wp, (cuuint32_t)(RB + 3), 1};
  cuuint32_t boxd[4] = {32, (cuuint32_t)Wp, (cuuint32_t)RB, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  if (!fn ||
      fn(&mx, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, boxx, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      fn(&md, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(dz), dims, strides, boxd, estr,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    set_error("wgrad_halo: tensor map encoding failed");
    return DDPPO_E_CUDA;
  }
  const int nrb = (c.H + RB - 1) / RB;
  const int nunits = c.N * nrb;
  int grid = std::min(nunits, ws.num_sms);
  const size_t per = (size_t)3 * 3 * 32 * 32;
  grid = (int)std::min<size_t>((size_t)grid, ws.partial_elems / per);
  if (grid < 1) {
    set_error("wgrad_halo: split-K workspace too small");
    return DDPPO_E_CONFIG;
  }
  static bool attr_done[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !attr_done[dev]) {
    DDPPO_CHECK_CUDA(cudaFuncSetAttribute(wgrad_halo_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)TC_SMEM_MAX));
    attr_done[dev] = true;
  }
  ::ddppo::launch_k(wgrad_halo_kernel, grid, WH_THREADS, g.smem, s, mx, md, Wp, RB, nrb, nunits, g.x_bytes,
                                                     g.dz_bytes, g.x_stride, g.dz_stride, g.stages,
                                                     ws.partial, ws.err);
  DDPPO_CHECK_LAUNCH();
  ::ddppo::launch_k(wgrad_halo_reduce_kernel, (32 * 288 + 255) / 256, 256, 0, s, ws.partial, grid, dw, ldw, beta);
  DDPPO_CHECK_LAUNCH();
  return DDPPO_OK;
}

}  // namespace ddppo
