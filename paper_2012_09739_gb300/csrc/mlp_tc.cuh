// Warp-level FP16 tensor-core forward pass of the MLP surrogate
// (1 -> 32 -> 32 -> 1, tanh) with mma.sync.m16n8k16 (FP16 operands, FP32
// accumulation, tanh.approx activations), used by training (mlp_train.cu);
// inference is mlp_eval16 (mlp_device.cuh).
//
// A warp evaluates 64 rows at a time: lane L owns rows 16 i + q + 8 h for
// i = L % 4, q = L / 4 and h = 0, 1 (its two samples).  The rows are handled
// in four 16-row tiles m; in tile m the mma fragments of lane L cover rows
// 16 m + q and 16 m + q + 8 (the accumulator layout of one layer is the
// operand layout of the next, so activations stay in registers).
//   layer 1: h1 = tanh(W1 t + b1)      (FP32 FMA, tanh in f16x2)
//   layer 2: h2 = tanh(h1 W2^T + b2)   (8 mma per tile: 4 n-tiles x 2 k-chunks)
//   layer 3: y = h2 W3^T + b3          (2 mma per tile; W3 as the only non-zero
//                                       column of an 8-wide B operand)
// The input is t = sqrt(-2 ln v), v = min(u, 1-u), in FP32.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "device.cuh"
#include "mlp_device.cuh"

namespace mlmc {

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

__device__ __forceinline__ uint32_t tanh_h2(uint32_t x) {
    uint32_t r;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(r) : "r"(x));
    return r;
}

__device__ __forceinline__ float2 unpack_h2(uint32_t x) {
    return __half22float2(*reinterpret_cast<__half2 *>(&x));
}

// D = A B + C, m16n8k16, f16 x f16 -> f32 (not volatile: the outputs are
// used, and the compiler may interleave independent tiles).
__device__ __forceinline__ void mma16816(float &d0, float &d1, float &d2, float &d3, uint32_t a0, uint32_t a1,
                                         uint32_t a2, uint32_t a3, uint32_t b0, uint32_t b1, float c0, float c1,
                                         float c2, float c3) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%10,%11,%12,%13};"
        : "=f"(d0), "=f"(d1), "=f"(d2), "=f"(d3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(c0), "f"(c1), "f"(c2), "f"(c3));
}

// Per-lane register copy of the network in fragment form.
struct MlpFrags {
    float w1[8], b1[8];      // layer-1 weights of this lane's 8 columns, index (kc, hi, e) = 4 kc + 2 hi + e
    uint32_t w2[4][2][2];    // layer-2 B operand [n-tile][k-chunk][reg]: B[k=j][n=o] = W2[o][j]
    float b2[4][2];          // layer-2 bias of this lane's accumulator columns [n-tile][e]
    uint32_t w3[2][2];       // layer-3 B operand [k-chunk][reg] (zero except for lanes 0..3)
    float b3;

    // column of layer-1 index (kc, hi, e) for lane t = L % 4
    static __device__ __forceinline__ int col1(int kc, int hi, int e, int t) { return 16 * kc + 8 * hi + 2 * t + e; }

    __device__ __forceinline__ void load(const MlpWeights *m) {
        const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
        const float *W1 = m->w, *B1 = m->w + 32, *W2 = m->w + 64, *B2 = m->w + 64 + 1024;
        const float *W3 = m->w + 64 + 1024 + 32;
        for (int kc = 0; kc < 2; ++kc)
            for (int hi = 0; hi < 2; ++hi)
                for (int e = 0; e < 2; ++e) {
                    const int c = col1(kc, hi, e, t);
                    w1[4 * kc + 2 * hi + e] = W1[c];
                    b1[4 * kc + 2 * hi + e] = B1[c];
                }
        for (int nt = 0; nt < 4; ++nt) {
            const int o = 8 * nt + g;
            for (int kc = 0; kc < 2; ++kc) {
                const int j = 16 * kc + 2 * t;
                w2[nt][kc][0] = pack_h2(W2[o * 32 + j], W2[o * 32 + j + 1]);
                w2[nt][kc][1] = pack_h2(W2[o * 32 + j + 8], W2[o * 32 + j + 9]);
            }
            b2[nt][0] = B2[8 * nt + 2 * t];
            b2[nt][1] = B2[8 * nt + 2 * t + 1];
        }
        for (int kc = 0; kc < 2; ++kc) {
            const int j = 16 * kc + 2 * t;
            w3[kc][0] = g == 0 ? pack_h2(W3[j], W3[j + 1]) : 0u;
            w3[kc][1] = g == 0 ? pack_h2(W3[j + 8], W3[j + 9]) : 0u;
        }
        b3 = m->w[64 + 1024 + 64];
    }
};

// Layer 1 for one tile: A fragments of h1 for rows (r0, r1) with inputs (t0, t1).
__device__ __forceinline__ void mlp_layer1(const MlpFrags &F, float t0, float t1, uint32_t a[2][4]) {
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
        const float *w = F.w1 + 4 * kc, *b = F.b1 + 4 * kc;
        a[kc][0] = tanh_h2(pack_h2(fmaf(w[0], t0, b[0]), fmaf(w[1], t0, b[1])));
        a[kc][1] = tanh_h2(pack_h2(fmaf(w[0], t1, b[0]), fmaf(w[1], t1, b[1])));
        a[kc][2] = tanh_h2(pack_h2(fmaf(w[2], t0, b[2]), fmaf(w[3], t0, b[3])));
        a[kc][3] = tanh_h2(pack_h2(fmaf(w[2], t1, b[2]), fmaf(w[3], t1, b[3])));
    }
}

// Layer 2 for one tile: h2 in operand layout for layer 3, h[k-chunk][reg].
__device__ __forceinline__ void mlp_layer2(const MlpFrags &F, const uint32_t a[2][4], uint32_t h[2][4]) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
        float c0 = F.b2[nt][0], c1 = F.b2[nt][1], c2 = F.b2[nt][0], c3 = F.b2[nt][1];
        mma16816(c0, c1, c2, c3, a[0][0], a[0][1], a[0][2], a[0][3], F.w2[nt][0][0], F.w2[nt][0][1], c0, c1, c2, c3);
        mma16816(c0, c1, c2, c3, a[1][0], a[1][1], a[1][2], a[1][3], F.w2[nt][1][0], F.w2[nt][1][1], c0, c1, c2, c3);
        // n-tile nt covers columns 8 nt .. 8 nt + 7: k-chunk nt / 2, low or high half
        const int kc = nt >> 1, hi = nt & 1;
        h[kc][2 * hi + 0] = tanh_h2(pack_h2(c0, c1));
        h[kc][2 * hi + 1] = tanh_h2(pack_h2(c2, c3));
    }
}

// Layer 3 for one tile: y of rows r0 and r1, valid in lanes with L % 4 == 0.
__device__ __forceinline__ void mlp_layer3(const MlpFrags &F, const uint32_t h[2][4], float &y0, float &y1) {
    float c0 = F.b3, c1 = 0.0f, c2 = F.b3, c3 = 0.0f;
    mma16816(c0, c1, c2, c3, h[0][0], h[0][1], h[0][2], h[0][3], F.w3[0][0], F.w3[0][1], c0, c1, c2, c3);
    mma16816(c0, c1, c2, c3, h[1][0], h[1][1], h[1][2], h[1][3], F.w3[1][0], F.w3[1][1], c0, c1, c2, c3);
    y0 = c0;
    y1 = c2;
}

}  // namespace mlmc
