// mlp.cuh -- the learned step-size proposer: a 12 -> 64 -> 64 -> 1 perceptron with GELU,
// bfloat16 operands and float32 accumulation, float32 master weights.
//
//   a1 = bf16(gelu(W1 bf16(x) + b1)),  a2 = bf16(gelu(W2 a1 + b2)),  m = W3 a2 + b3
//
// with W1, W2, W3 rounded to bfloat16.  m estimates log2 of the largest next step,
// relative to the last attempted one, that the corrector would accept.
// Parameter vector: W1 (64x12, row-major) | b1 | W2 (64x64) | b2 | W3 | b3 = 5,057 floats.
#pragma once
#include <cuda_bf16.h>

namespace hc {

#define MLP_IN 12
#define MLP_H 64
#define MLP_NP 5057
#define MLP_W1 0
#define MLP_B1 768
#define MLP_W2 832
#define MLP_B2 4928
#define MLP_W3 4992
#define MLP_B3 5056

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_df(float u)
{
    return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) + u * expf(-0.5f * u * u) * 0.39894228040143268f;
}

// One evaluation by a single thread (the tracker's proposal, once per corrector stage).
__device__ __forceinline__ float mlp_forward_thread(const float *__restrict__ p, const float *x_in)
{
    float x[MLP_IN], a1[MLP_H];
    for (int i = 0; i < MLP_IN; i++) x[i] = bf16r(x_in[i]);
    for (int o = 0; o < MLP_H; o++) {
        float u = p[MLP_B1 + o];
        for (int i = 0; i < MLP_IN; i++) u = fmaf(bf16r(p[MLP_W1 + o * MLP_IN + i]), x[i], u);
        a1[o] = bf16r(gelu_f(u));
    }
    float m = p[MLP_B3];
    for (int o = 0; o < MLP_H; o++) {
        float u = p[MLP_B2 + o];
        for (int i = 0; i < MLP_H; i++) u = fmaf(bf16r(p[MLP_W2 + o * MLP_H + i]), a1[i], u);
        m = fmaf(bf16r(p[MLP_W3 + o]), bf16r(gelu_f(u)), m);
    }
    return m;
}

}  // namespace hc
