// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mlmc.h"

namespace mlmc {

struct LevelArgs;
struct MlpWeights;
struct DevTables;
using LevelKernelFn = void (*)(LevelArgs);

LevelKernelFn level_kernel_f32(int mode, int kahan, int icdf, int sde);
LevelKernelFn level_kernel_f16(int mode, int kahan, int icdf, int sde);
LevelKernelFn level_kernel_bf16(int mode, int kahan, int icdf, int sde);

cudaError_t launch_build_table(DevTables *out, cudaStream_t s);
// out receives (sum, sum of squares); scratch holds finalize_scratch(count) double2.
uint64_t finalize_scratch(uint64_t count);
cudaError_t launch_finalize(const double2 *partials, uint64_t count, double *out, double2 *scratch, cudaStream_t s);
cudaError_t launch_philox_bulk(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t n, cudaStream_t s);
cudaError_t launch_uniform_bulk(const uint32_t *w, float *u, size_t n, cudaStream_t s);
cudaError_t launch_icdf_bulk(const float *u, void *z, size_t n, int icdf, int prec, const DevTables *tabs,
                             const MlpWeights *mlp, cudaStream_t s);

}  // namespace mlmc
