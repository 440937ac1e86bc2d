// hm_mlp.cuh -- learned rank model: MLP 8 -> 64 -> 64 -> 1 (ReLU), FP32.
#pragma once

#include "hm_internal.cuh"

namespace hm {

constexpr int MLP_F = 8;
constexpr int MLP_H = 64;
constexpr int MLP_NPARAM = MLP_H * MLP_F + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;  // 4801

void mlp_forward(const float* theta, const float* F, int64_t n, float* out, cudaStream_t s);
void mlp_loss_grad(const float* theta, const float* F, const float* target, int64_t n,
                   float* grad, float* loss, cudaStream_t s);
void mlp_adam(float* theta, const float* grad, float* m, float* v, int64_t t, float lr,
              float b1, float b2, float eps, cudaStream_t s);

}  // namespace hm
