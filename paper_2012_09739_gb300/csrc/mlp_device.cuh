// MLP surrogate inverse CDF used inside the level kernels.
//
// y(t) = W3 tanh(W2 tanh(W1 t + b1) + b2) + b3 approximates |Phi^-1(v)| for
// t = sqrt(-2 ln v), v = min(u, 1-u); Z~ = -y for u <= 1/2, +y above.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "device.cuh"

namespace mlmc {

constexpr int MLP_H = 32;
constexpr int MLP_NPARAMS = MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;   // 1153

// Device copy of the network: FP32 master weights in the 1153-value layout
// (W1, b1, W2 row-major [out][in], b2, W3, b3), and binary16 copies of W2
// for the tensor-core path.
struct MlpWeights {
    float w[MLP_NPARAMS + 3];     // padded to a multiple of 4
    __half w2h[MLP_H * MLP_H];    // W2 in binary16, [out][in]
};

__device__ __forceinline__ const float *mlp_W1(const MlpWeights *m) { return m->w; }
__device__ __forceinline__ const float *mlp_b1(const MlpWeights *m) { return m->w + 32; }
__device__ __forceinline__ const float *mlp_W2(const MlpWeights *m) { return m->w + 64; }
__device__ __forceinline__ const float *mlp_b2(const MlpWeights *m) { return m->w + 64 + 1024; }
__device__ __forceinline__ const float *mlp_W3(const MlpWeights *m) { return m->w + 64 + 1024 + 32; }
__device__ __forceinline__ float mlp_b3(const MlpWeights *m) { return m->w[64 + 1024 + 64]; }

// Scalar FP32 evaluation of y(t) for v in (0, 1/2].
__device__ __forceinline__ float mlp_y(const MlpWeights *m, float v) {
    const float t = sqrtf(-2.0f * logf(v));
    float h1[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) h1[j] = tanhf(fmaf(__ldg(mlp_W1(m) + j), t, __ldg(mlp_b1(m) + j)));
    float y = mlp_b3(m);
    for (int o = 0; o < MLP_H; ++o) {
        float acc = __ldg(mlp_b2(m) + o);
#pragma unroll
        for (int j = 0; j < MLP_H; ++j) acc = fmaf(__ldg(mlp_W2(m) + o * MLP_H + j), h1[j], acc);
        y = fmaf(__ldg(mlp_W3(m) + o), tanhf(acc), y);
    }
    return y;
}

// Z~ = -y for u <= 1/2, +y above.
__device__ __forceinline__ float mlp_z_from_v(const MlpWeights *m, float v, bool upper) {
    const float y = mlp_y(m, v);
    return upper ? y : -y;
}

__device__ __forceinline__ float mlp_z_scalar(const MlpWeights *m, uint32_t w) {
    return mlp_z_from_v(m, mirrored_v(w), (w & 0x80000000u) != 0);
}

__device__ __forceinline__ float2 mlp_z_pair(const MlpWeights *m, uint32_t w0, uint32_t w1) {
    return make_float2(mlp_z_scalar(m, w0), mlp_z_scalar(m, w1));
}

}  // namespace mlmc
