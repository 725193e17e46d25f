// Fixed-order FP64 reduction shared by the finalize kernels, so that a level
// launch and a batched launch add the same partials in the same order.
#pragma once

#include <cstdint>

namespace mlmc {

// A finalize sum covers at most FINALIZE_SPAN partials; more partials are
// first reduced span by span, then the span sums are reduced the same way.
constexpr uint64_t FINALIZE_SPAN = 8192;
constexpr int FINALIZE_THREADS = 1024;   // the strided sums of one fixed-order sum

// The fixed-order sum of p[0 .. n): FINALIZE_THREADS = 1024 strided sums
// (sum t adds p[t], p[t + 1024], ... in order, from 0.0), then a binary tree
// over them (level h = 512, 256, ..., 1: sum t += sum t + h for t < h).  A
// block of SUM_THREADS = 256 threads computes it: thread t holds the sums
// t, t + 256, t + 512, t + 768, so the levels 512 and 256 pair sums within a
// thread, 128 .. 32 go through shared memory and 16 .. 1 through shuffles.
// Every thread of the block must call it; thread 0 gets the result.
constexpr int SUM_THREADS = 256;

__device__ __forceinline__ double2 block_sum_fixed(const double2 *p, uint64_t n, double *r1, double *r2) {
    const uint32_t t = threadIdx.x;
    double x[4] = {0.0, 0.0, 0.0, 0.0}, y[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (uint64_t base = 0; base < n; base += FINALIZE_THREADS) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t i = base + t + SUM_THREADS * k;
            if (i < n) {
                const double2 v = p[i];
                x[k] += v.x;
                y[k] += v.y;
            }
        }
    }
    x[0] += x[2];       // level 512: sums t, t + 256 take t + 512, t + 768
    y[0] += y[2];
    x[1] += x[3];
    y[1] += y[3];
    x[0] += x[1];       // level 256
    y[0] += y[1];
    r1[t] = x[0];
    r2[t] = y[0];
    __syncthreads();
    for (int h = 128; h >= 32; h >>= 1) {
        if (t < h) {
            r1[t] += r1[t + h];
            r2[t] += r2[t + h];
        }
        __syncthreads();
    }
    double sx = 0.0, sy = 0.0;
    if (t < 32) {
        sx = r1[t];
        sy = r2[t];
#pragma unroll
        for (int h = 16; h > 0; h >>= 1) {
            sx += __shfl_down_sync(0xffffffffu, sx, h);
            sy += __shfl_down_sync(0xffffffffu, sy, h);
        }
    }
    __syncthreads();    // r1, r2 may be reused
    return make_double2(sx, sy);
}

}  // namespace mlmc
