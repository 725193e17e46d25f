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

// Device copy of the network: FP32 master weights in the 1153-value layout
// (W1, b1, W2 row-major [out][in], b2, W3, b3), and binary16 copies of W2
// for the tensor-core path.
struct MlpWeights {
    float w[MLP_NPARAMS + 3];     // padded to a multiple of 4
    __half w2h[MLP_H * MLP_H];    // W2 in binary16, [out][in]
};

}  // namespace mlmc
