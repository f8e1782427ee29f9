// Device helpers shared by the tcgen05 kernels (sm_103a): shared-memory addresses,
// mbarriers with bounded waits, the tcgen05 commit, the 128-byte-swizzled K-major shared
// memory descriptor, the kind::f16 / kind::f8f6f4 instruction descriptors and the MMA.
#pragma once

#include "common.cuh"

namespace ddppo {

constexpr uint32_t TC_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; on expiry marks the CTA aborted and raises the timeout flag
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          int32_t* err) {
  for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i) {
    if (mbar_try(bar, parity)) return true;
    if (*abort) return false;
    // another CTA already timed out: give up at once instead of waiting out the limit
    if ((i & 1023u) == 1023u && err && (*(volatile int32_t*)err & 2)) {
      *abort = 1;
      return false;
    }
  }
  *abort = 1;
  if (err) atomicOr(err, 2);
  return false;
}

// the drain after an abort: poll until the phase completes or the limit runs out (the
// abort flag is already set, so mbar_wait would return at once)
__device__ __forceinline__ bool mbar_drain_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < TC_SPIN_LIMIT; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

// shared-memory matrix descriptors, 128-byte swizzle.
// K-major tile: rows of 64 K-elements (128 B), 8-row groups 1024 B apart (SBO); the K
// offset of an MMA within the swizzle atom is added to the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version (tcgen05)
  d |= (uint64_t)2 << 61;              // SWIZZLE_128B
  return d;
}
// instruction descriptor, kind::f16: D f32, A/B bf16; a_mn / b_mn select MN-major operands
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N, int a_mn = 0, int b_mn = 0) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a_mn & 1) << 15) |
         ((uint32_t)(b_mn & 1) << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// instruction descriptor, kind::f8f6f4: D f32, A/B E4M3 (format code 0), both K-major
__host__ __device__ constexpr uint32_t f8_idesc(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// one MMA of the tile into TMEM: bf16 x bf16 (K = 16) or E4M3 x E4M3 (K = 32). Either way
// it consumes 32 bytes of every operand row, so the shared-memory layouts and descriptors
// are the same; acc = 0 overwrites the accumulator
__device__ __forceinline__ void tc_mma(uint32_t dacc, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t acc, int fp8) {
  if (fp8)
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}

}  // namespace ddppo
