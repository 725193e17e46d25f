// Device copy of the MLP surrogate inverse CDF, and its inference.
//
// y(t) = W3 tanh(W2 tanh(W1 t + b1) + b2) + b3 approximates |Phi^-1(v)| for
// t = sqrt(-2 ln v), v = min(u, 1-u); Z~ = -y for u <= 1/2, +y above.
// Inference (mlp_eval16 below) is in binary16 inference arithmetic:
// binary16 weights W2, W3 and activations, every activation the tanh of a
// binary16 value correctly rounded to binary16, binary32 fused multiply-add
// accumulation in index order -- operations that each round once, so the
// result is defined bit for bit.  Training (mlp_train.cu) runs the same
// network on tensor cores (mlp_tc.cuh).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "device.cuh"

namespace mlmc {

constexpr int MLP_H = 32;
constexpr int MLP_NPARAMS = MLP_H + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;   // 1153

// The network's input v = min(u, 1 - u) takes 2^22 values on the 24-bit
// uniform grid u = (2 k + 1) 2^-24: v_k = (2 k + 1) 2^-24, k < 2^22.
constexpr uint32_t MLP_GRID = 1u << 22;

// The activation table: tanh of every binary16 value x >= 0 (bit patterns
// 0 .. 0x7FFF: zero, subnormals, normals, +inf, NaNs), the binary64 tanh
// rounded once to binary16 (nearest even), indexed by the pattern; odd
// symmetry gives x < 0.
constexpr uint32_t MLP_TANH16 = 0x8000;

// Device copy of the network: FP32 master weights in the 1153-value layout
// (W1, b1, W2 row-major [out][in], b2, W3, b3), the activation table, and
// the network's output y(v_k) on every grid point, evaluated by mlp_eval16
// whenever the weights change: the level kernels gather from it, which
// gives the value of evaluating the network for the sample (each grid
// point's evaluation depends on its own input only) for one load instead of
// 64 activations and 1,088 multiply-adds.
struct MlpWeights {
    float w[MLP_NPARAMS + 3];       // padded to a multiple of 4
    uint16_t tanh16[MLP_TANH16];    // 64 KiB
    float ygrid[MLP_GRID];          // y(v_k), 16 MiB
};

// Network input t = sqrt(-2 ln v) from v in [2^-24, 1/2], with binary32
// operations that each round once to nearest (so that the oracle can repeat
// them exactly): v = m 2^e with m in [1/sqrt2, sqrt2]; ln m = 2 z (1 + z^2/3
// + z^4/5 + z^6/7 + z^8/9) with z = (m - 1) / (m + 1), |z| <= 0.1716 (the
// atanh series; the next term is below 7e-10); t^2 = -2 e ln2 - 2 ln m by one
// FMA; t = sqrt(t^2) correctly rounded.
__device__ __forceinline__ float mlp_feature(float v) {
    const uint32_t b = __float_as_uint(v);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 1.41421354f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float z = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float w = __fmul_rn(z, z);
    float q = __fmaf_rn(1.0f / 9.0f, w, 1.0f / 7.0f);
    q = __fmaf_rn(q, w, 1.0f / 5.0f);
    q = __fmaf_rn(q, w, 1.0f / 3.0f);
    q = __fmaf_rn(q, w, 1.0f);
    const float lnm = __fmul_rn(__fmul_rn(2.0f, z), q);
    const float t2 = __fmaf_rn((float)(-2 * e), 0.693147182f, __fmul_rn(-2.0f, lnm));
    return __fsqrt_rn(t2);
}

// The network in shared memory for mlp_eval16: W2 and W3 rounded to
// binary16 (held as the binary32 values of those binary16 numbers).
struct alignas(16) MlpShared {
    float w1[MLP_H], b1[MLP_H], b2[MLP_H], w3h[MLP_H];
    float w2h[MLP_H * MLP_H];       // [out][in]
    float b3;
};

// Every thread of the block calls it; the caller synchronises the block.
__device__ __forceinline__ void mlp_stage(MlpShared &s, const MlpWeights *m) {
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x)
        s.w2h[i] = __half2float(__float2half_rn(m->w[2 * MLP_H + i]));
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        s.w1[i] = m->w[i];
        s.b1[i] = m->w[MLP_H + i];
        s.b2[i] = m->w[2 * MLP_H + MLP_H * MLP_H + i];
        s.w3h[i] = __half2float(__float2half_rn(m->w[3 * MLP_H + MLP_H * MLP_H + i]));
    }
    if (threadIdx.x == 0) s.b3 = m->w[4 * MLP_H + MLP_H * MLP_H];
}

// tanh16(R16(x)): x rounded to binary16 (nearest even; beyond the binary16
// range to +-inf, whose entry is +-1), then the table.
__device__ __forceinline__ float mlp_act16(const uint16_t *__restrict__ tanh16, float x) {
    const uint16_t b = __half_as_ushort(__float2half_rn(x));
    const uint16_t r = (uint16_t)(__ldg(tanh16 + (b & 0x7FFFu)) | (b & 0x8000u));
    return __half2float(__ushort_as_half(r));
}

// y(t) in binary16 inference arithmetic: h1_j = tanh16(fma(W1_j, t, b1_j));
// c_o = b2_o, then c_o = fma(W2_oi, h1_i, c_o) for i = 0 .. 31 in turn,
// h2_o = tanh16(c_o); y = b3, then y = fma(W3_o, h2_o, y) for o = 0 .. 31.
__device__ __forceinline__ float mlp_eval16(const MlpShared &s, const uint16_t *__restrict__ tanh16, float t) {
    float h1[MLP_H];
#pragma unroll
    for (int j = 0; j < MLP_H; ++j) h1[j] = mlp_act16(tanh16, __fmaf_rn(s.w1[j], t, s.b1[j]));
    float y = s.b3;
#pragma unroll 2
    for (int o = 0; o < MLP_H; ++o) {
        float c = s.b2[o];
#pragma unroll
        for (int i = 0; i < MLP_H; ++i) c = __fmaf_rn(s.w2h[o * MLP_H + i], h1[i], c);
        y = __fmaf_rn(s.w3h[o], mlp_act16(tanh16, c), y);
    }
    return y;
}

// Z~ of a word from the tabulated network: k = w >> 9 indexes u's grid
// point, v's index is k or 2^23 - 1 - k (k ^ 0x7FFFFF) above 1/2; -y for
// u <= 1/2 (bit 31 clear), +y above.
__device__ __forceinline__ float mlp_grid_z(const float *ygrid, uint32_t w) {
    const uint32_t k = w >> 9;
    const float y = __ldg(ygrid + (k ^ ((k >> 22) ? 0x7FFFFFu : 0u)));
    return __uint_as_float(__float_as_uint(y) ^ (~w & 0x80000000u));
}

}  // namespace mlmc
