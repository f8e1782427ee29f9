// PPO loss entry point that allocates nothing (ddppo_ppo_loss_static).
//
// Some callers cannot allocate device memory where they need the loss: code that runs
// while a stream is being captured into a CUDA graph in a capture mode that forbids
// cudaMalloc, or a process whose device memory all belongs to another allocator. The
// stateless ddppo_ppo_loss needs no scratch but reduces with a single thread block; this
// variant spreads the samples over one block per 256 and keeps the per-block partial
// sums in a library-owned array declared below, so it needs neither an allocation nor a
// worker context.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds
// it until the process exits. Host code cannot use its name as a device address, so the
// first call on each device looks the address up (cudaGetSymbolAddress, with that device
// current) and caches it; make that first call before any stream capture. All calls
// share the array: calls that overlap on the GPU (different streams, or concurrent host
// threads) race on it. Each call overwrites the partials it reads, so nothing has to be
// cleared between calls. The cached address outlives a cudaDeviceReset, which makes it
// stale: after a device reset, this entry point must not be called on that device again
// in the same process.
#include <mutex>

#include "rl.cuh"

namespace {
constexpr int kStaticLossMaxBlocks = 4096;                      // 256 samples per block
constexpr int kStaticLossMaxSamples = kStaticLossMaxBlocks * 256;  // 1,048,576
constexpr int kMaxDevices = 64;
__device__ __align__(256) float g_loss_partials[kStaticLossMaxBlocks * 5];  // 80 KiB
std::mutex g_mu;
float* g_partials_ptr[kMaxDevices] = {};
}  // namespace

using namespace ddppo;

extern "C" int ddppo_ppo_loss_static(int32_t n, const float* logits, const float* values,
                                     const int32_t* actions, const float* logp_old,
                                     const float* adv, const float* ret, float clip,
                                     float value_coef, float entropy_coef, float* stats,
                                     float* dlogits, float* dvalues, void* stream) {
  if (n < 0) {
    set_error("ppo_loss_static: negative size");
    return DDPPO_E_ARG;
  }
  if (n > kStaticLossMaxSamples) {
    set_error("ppo_loss_static: n = " + std::to_string(n) + " exceeds the static scratch limit of " +
              std::to_string(kStaticLossMaxSamples) + " samples; use ddppo_ppo_loss");
    return DDPPO_E_CONFIG;
  }
  if (n == 0) return DDPPO_OK;
  if (!logits || !values || !actions || !logp_old || !adv || !ret || !stats || !dlogits ||
      !dvalues) {
    set_error("ppo_loss_static: null argument");
    return DDPPO_E_ARG;
  }
  int dev = 0;
  DDPPO_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("ppo_loss_static: device ordinal out of range");
    return DDPPO_E_CONFIG;
  }
  float* part = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partials_ptr[dev]) {
      void* p = nullptr;
      DDPPO_CHECK_CUDA(cudaGetSymbolAddress(&p, g_loss_partials));
      g_partials_ptr[dev] = (float*)p;
    }
    part = g_partials_ptr[dev];
  }
  const int nb = (n + 255) / 256;
  return launch_ppo_loss_blocks(n, logits, values, actions, logp_old, adv, ret, clip, value_coef,
                                entropy_coef, stats, dlogits, dvalues, part, nb,
                                (cudaStream_t)stream);
}
