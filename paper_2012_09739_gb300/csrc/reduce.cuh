// Fixed-order FP64 reduction shared by the finalize kernels, so that a level
// launch and a batched launch add the same partials in the same order.
#pragma once

#include <cstdint>

namespace mlmc {

// A finalize block adds at most FINALIZE_SPAN partials; more partials are
// first reduced span by span, then the span sums are reduced the same way.
constexpr uint64_t FINALIZE_SPAN = 8192;
constexpr int FINALIZE_THREADS = 1024;

// Sum of p[lo .. end) by a block of FINALIZE_THREADS threads: thread t adds
// p[lo + t], p[lo + t + 1024], ... in order, then a fixed binary tree over
// the threads' sums (r1, r2: FINALIZE_THREADS doubles of shared memory each).
// Every thread of the block must call it; all of them get the result.
__device__ __forceinline__ double2 block_sum_fixed(const double2 *p, uint64_t lo, uint64_t end, double *r1,
                                                   double *r2) {
    double t1 = 0.0, t2 = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < end; i += FINALIZE_THREADS) {
        t1 += p[i].x;
        t2 += p[i].y;
    }
    r1[threadIdx.x] = t1;
    r2[threadIdx.x] = t2;
    __syncthreads();
    for (int h = FINALIZE_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            r1[threadIdx.x] += r1[threadIdx.x + h];
            r2[threadIdx.x] += r2[threadIdx.x + h];
        }
        __syncthreads();
    }
    const double2 s = make_double2(r1[0], r2[0]);
    __syncthreads();    // r1, r2 may be reused
    return s;
}

}  // namespace mlmc
