// Launchers of the learning-step kernels (rl.cu).
#pragma once

#include "common.cuh"

namespace ddppo {
int launch_ppo_loss(int n, const float* logits, const float* values, const int32_t* actions,
                    const float* logp_old, const float* adv, const float* ret, float clip, float cv,
                    float ce, float* stats, float* dlogits, float* dvalues, float* part,
                    size_t part_elems, cudaStream_t s);
// exactly nb blocks of 256 threads, partials part[nb * 5]
int launch_ppo_loss_blocks(int n, const float* logits, const float* values, const int32_t* actions,
                           const float* logp_old, const float* adv, const float* ret, float clip,
                           float cv, float ce, float* stats, float* dlogits, float* dvalues,
                           float* part, int nb, cudaStream_t s);
int launch_grad_norm(const float* g, size_t n, float* norm_out, float* part, size_t part_elems,
                     cudaStream_t s);
// Adam at step t = *t_dev + t_off (t_dev: device scalar, so a captured update replays with
// the current step)
int launch_adam(float* p, const float* g, float* m, float* v, size_t n, const float* norm,
                float max_norm, float lr, float b1, float b2, float eps, const int64_t* t_dev,
                int t_off, cudaStream_t s);
// env permutation of (seed, *update_dev, epoch); update_dev: device scalar
int launch_permutation(uint64_t seed, const int64_t* update_dev, int64_t epoch, int E,
                       int32_t* perm, cudaStream_t s);
int launch_normalize_adv(const float* adv, float* out, size_t n, float* scal2, float* part,
                         size_t part_elems, cudaStream_t s);
int launch_copy_scalar(float* dst, const float* src, cudaStream_t s);
}  // namespace ddppo
