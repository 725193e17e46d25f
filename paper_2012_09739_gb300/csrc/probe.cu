// Issue-rate probes of the non-tensor pipes (mlmc_peak_probe).
//
// Each thread runs eight independent dependency chains of one instruction
// kind, written as inline PTX so that the compiler neither removes nor fuses
// them; a full grid of resident blocks runs long enough (~10 ms) for the
// event timing to be accurate.  The result is thread-operations per second
// (an f16x2 FMA counts as two operations).
#include "api_internal.h"

namespace mlmc {

constexpr int PROBE_ITERS = 4096;
constexpr int PROBE_CHAINS = 8;

template <int KIND>
__global__ void __launch_bounds__(256) probe_kernel(uint32_t seed, uint32_t *sink) {
    uint32_t r[PROBE_CHAINS];
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) r[c] = seed + threadIdx.x * 7u + c * 0x9E3779B9u;
    const uint32_t k1 = seed | 1u, k2 = seed * 3u + 1u;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int c = 0; c < PROBE_CHAINS; ++c) {
            if (KIND == 0) {         // FP32 FMA
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+r"(r[c]) : "r"(0x3f7ffff0u), "r"(0x33800000u));
            } else if (KIND == 1) {  // f16x2 FMA
                asm volatile("fma.rn.f16x2 %0, %0, %1, %2;" : "+r"(r[c]) : "r"(0x3bff3bffu), "r"(0x10011001u));
            } else if (KIND == 2) {  // 32-bit integer multiply-add
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r[c]) : "r"(k1), "r"(k2));
            } else {                 // three-input logic op (XOR of three)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r[c]) : "r"(k1), "r"(k2));
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) acc ^= r[c];
    if (acc == 0x12345678u) sink[0] = acc;   // keeps the chains live
}

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_peak_probe(int kind, double *ops_per_s, void *stream) {
    if (kind < 0 || kind > 3) return fail(MLMC_EINVAL, "probe kind must be 0..3");
    if (!ops_per_s) return fail(MLMC_EINVAL, "ops_per_s is NULL");
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    void (*fn)(uint32_t, uint32_t *) = kind == 0 ? probe_kernel<0> : kind == 1 ? probe_kernel<1>
                                       : kind == 2 ? probe_kernel<2> : probe_kernel<3>;
    int bps = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "occupancy");
    const int grid = (bps > 0 ? bps : 1) * d->sm_count;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *sink = nullptr;
    if ((e = cudaMallocAsync(&sink, 4, s)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    fn<<<grid, 256, 0, s>>>(1u, sink);              // warm-up (clocks ramp)
    cudaEventRecord(a, s);
    const int reps = 5;
    for (int i = 0; i < reps; ++i) fn<<<grid, 256, 0, s>>>(2u + i, sink);
    cudaEventRecord(b, s);
    cudaFreeAsync(sink, s);
    e = cudaGetLastError();
    if (e == cudaSuccess) st = wait_event(b, wait_limit_s());
    else st = cuda_fail(e, "probe launch");
    if (!st) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        const double ops = (double)reps * grid * 256.0 * PROBE_ITERS * PROBE_CHAINS * (kind == 1 ? 2.0 : 1.0);
        *ops_per_s = ops / (ms * 1e-3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}
