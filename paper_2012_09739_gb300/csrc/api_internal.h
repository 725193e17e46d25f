// Host-side state and helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"
#include "level_kernels.cuh"

namespace mlmc {

constexpr int MAX_DEVICES = 16;

struct BatchCache;   // batch.cu: device buffers of one batch plan (and its captured graph)
struct BatchGraphs;  // batch.cu: the captured graphs of mlmc_batch, by item-list shape

// Per-device library state: the piecewise-linear and cubic tables (FP64 and
// their binary32 / binary16 / bfloat16 roundings), the MLP weights, cached
// graphs.
struct DeviceState {
    bool ready = false;
    int device = -1;
    int sm_count = 0;
    DevTables *tabs = nullptr;
    MlpWeights *mlp = nullptr;
    bool mlp_ready = false;
    BatchGraphs *batch = nullptr;        // mlmc_batch: captured graphs and their buffers
    BatchCache *run_cache = nullptr;     // mlmc_run: buffers of its batched rounds
    cudaStream_t run_stream = nullptr;
    cudaEvent_t run_events[2] = {nullptr, nullptr};   // mlmc_run: around each round's launches
};

struct LaunchCfg {
    int grid = 1, block = 256;
};

mlmc_status fail(mlmc_status s, const char *fmt, ...);
mlmc_status cuda_fail(cudaError_t e, const char *where);
mlmc_status device_state(DeviceState **out);
mlmc_status wait_event(cudaEvent_t ev, double limit_s);
double wait_limit_s();
double *host_staging();
void level_moments(double s1, double s2, uint64_t n, double *mean, double *var);
mlmc_status check_params(const mlmc_sde_params *p);
mlmc_status check_level(int four, int l, uint64_t N, int prec, int icdf, const mlmc_sde_params *p);
LevelArgs make_level_args(const DeviceState &d, int four, int l, uint64_t N, int prec, int icdf, const mlmc_sde_params *p,
                          uint64_t seed, uint64_t path_offset, uint32_t set_id);
int kernel_sde(const mlmc_sde_params *p);
LevelKernelFn pick_level_kernel(int four, int prec, int kahan, int icdf, int sde);
LaunchCfg level_launch_cfg(const DeviceState &d, LevelKernelFn fn, uint64_t npairs);
mlmc_status enqueue_level(const DeviceState &d, int four, int l, uint64_t N, int prec, int kahan, int icdf,
                          const mlmc_sde_params *p, uint64_t seed, uint64_t path_offset, uint32_t set_id,
                          double *sums_dev, float *paths_dev, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1);
mlmc_status level_sync(int four, int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *p,
                       uint64_t seed, uint64_t path_offset, mlmc_sums *out, void *stream);
void release_device_extras(DeviceState &d);
BatchCache *batch_cache_create();
void batch_cache_destroy(BatchCache *c);
mlmc_status batch_round(const DeviceState &d, BatchCache &c, const mlmc_work *w, int n, uint64_t seed,
                        cudaStream_t s);
const double2 *batch_sums_host(const BatchCache &c);

}  // namespace mlmc
