// Device copy of the MLP surrogate inverse CDF.
//
// y(t) = W3 tanh(W2 tanh(W1 t + b1) + b2) + b3 approximates |Phi^-1(v)| for
// t = sqrt(-2 ln v), v = min(u, 1-u); Z~ = -y for u <= 1/2, +y above.  The
// evaluation (tensor cores, warp-cooperative) is in mlp_tc.cuh.
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

// Device copy of the network: FP32 master weights in the 1153-value layout
// (W1, b1, W2 row-major [out][in], b2, W3, b3), binary16 copies of W2, and
// the network's output y(v_k) on every grid point, evaluated by the
// tensor-core inference (mlp_tc.cuh) whenever the weights change: the level
// kernels gather from it, which gives the same value as evaluating the
// network for the sample (each row of the evaluation depends on its own
// input only) for one load instead of 64 activations and 40 mma per row.
struct MlpWeights {
    float w[MLP_NPARAMS + 3];     // padded to a multiple of 4
    __half w2h[MLP_H * MLP_H];    // W2 in binary16, [out][in]
    float ygrid[MLP_GRID];        // y(v_k), 16 MiB
};

// Z~ of a word from the tabulated network: k = w >> 9 indexes u's grid
// point, v's index is k or 2^23 - 1 - k (k ^ 0x7FFFFF) above 1/2; -y for
// u <= 1/2 (bit 31 clear), +y above.
__device__ __forceinline__ float mlp_grid_z(const float *ygrid, uint32_t w) {
    const uint32_t k = w >> 9;
    const float y = __ldg(ygrid + (k ^ ((k >> 22) ? 0x7FFFFFu : 0u)));
    return __uint_as_float(__float_as_uint(y) ^ (~w & 0x80000000u));
}

}  // namespace mlmc
