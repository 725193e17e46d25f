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
                const double2 v = __ldcg(p + i);      // from L2: other SMs wrote them
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

// Strided sum J of a warp's lane (slot lane + 32 J: 0.0 plus its partial, if
// any) after the in-lane tree levels down to stride H: the level-H step adds
// sum J + H to sum J.  Evaluated depth first (few live values); each
// addition has the operands of the level-by-level order.
template <int J, int H>
__device__ __forceinline__ double2 strided_tree(const double2 *p, uint32_t n, uint32_t lane) {
    if constexpr (H == 32) {
        const uint32_t i = lane + 32u * J;
        double2 s = make_double2(0.0, 0.0);
        if (i < n) {
            const double2 v = __ldcg(p + i);      // written by other SMs in the same launch
            s.x += v.x;
            s.y += v.y;
        }
        return s;
    } else {
        // a subtree of empty slots sums to +0.0 exactly, and no sum here is
        // -0.0 (each slot is 0.0 plus its partial), so adding it changes
        // nothing: skipped (binary64 additions are slow on this GPU)
        const double2 a = strided_tree<J, 2 * H>(p, n, lane);
        if (lane + 32u * (J + H) >= n) return a;
        const double2 b = strided_tree<J + H, 2 * H>(p, n, lane);
        return make_double2(a.x + b.x, a.y + b.y);
    }
}

// The same fixed-order sum of p[0 .. n) for n <= FINALIZE_THREADS, by one
// warp: lane L holds the strided sums L + 32 j (j = 0 .. 31), each 0.0 plus
// its one partial, so the tree levels 512 .. 32 pair sums within a lane and
// 16 .. 1 go through the same shuffles: every addition of block_sum_fixed,
// on the same operands.  Every lane of the warp must call it; lane 0 gets
// the result.
__device__ __forceinline__ double2 warp_sum_fixed(const double2 *p, uint32_t n, uint32_t lane) {
    const double2 s = strided_tree<0, 1>(p, n, lane);
    double sx = s.x, sy = s.y;
#pragma unroll
    for (int h = 16; h > 0; h >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, h);
        sy += __shfl_down_sync(0xffffffffu, sy, h);
    }
    return make_double2(sx, sy);
}

}  // namespace mlmc
