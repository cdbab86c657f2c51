// Parameter layout of the proposal MLP (8 -> 64 -> 128 -> 64 -> 1) and the
// host launchers of its kernels.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tr_problem.h"

namespace tr {

constexpr int kW1 = 0;                 // [64][8]
constexpr int kB1 = kW1 + 64 * 8;      // [64]
constexpr int kW2 = kB1 + 64;          // [128][64]
constexpr int kB2 = kW2 + 128 * 64;    // [128]
constexpr int kW3 = kB2 + 128;         // [64][128]
constexpr int kB3 = kW3 + 64 * 128;    // [64]
constexpr int kW4 = kB3 + 64;          // [64]
constexpr int kB4 = kW4 + 64;          // [1]
constexpr int kMlpParams = kB4 + 1;    // 17217

cudaError_t mlp_setup();
void launch_mlp_round(const float* w, float* wbf, cudaStream_t s);
void launch_features(const Batch& b, cudaStream_t s);
void launch_mlp_proposal(const Batch& b, int total, const float* wbf, cudaStream_t s);
void launch_mlp_forward(const float* feat, int m, const float* wbf, float* prob, float* z4, __nv_bfloat16* h1,
                        __nv_bfloat16* h2, __nv_bfloat16* h3, uint32_t* err, cudaStream_t s);
void launch_mlp_backward(const float* feat, const float* label, int m, const float* wbf, const float* z4,
                         const __nv_bfloat16* h1, const __nv_bfloat16* h2, const __nv_bfloat16* h3, float* grad,
                         float* loss, uint32_t* err, cudaStream_t s);
void launch_mlp_adam(float* w, float* mom, float* vel, const float* g, float* wbf, int step, float lr,
                     cudaStream_t s);
void launch_learned_hist(const Batch& b, int total, int max_n, cudaStream_t s);

}  // namespace tr
