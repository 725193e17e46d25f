// MLP weights on the device: the FP32 master copy, the binary16 activation
// table, and the network tabulated on the 24-bit uniform grid.
#include <vector>

#include "api_internal.h"
#include "mlp_device.cuh"

namespace mlmc {

// The activation table (independent of the weights; rebuilt with the grid).
__global__ void __launch_bounds__(256) mlp_tanh16_kernel(MlpWeights *m) {
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < MLP_TANH16; b += gridDim.x * blockDim.x) {
        const double x = (double)__half2float(__ushort_as_half((uint16_t)b));
        m->tanh16[b] = __half_as_ushort(__double2half(tanh(x)));
    }
}

// y(v_k) for every grid point v_k = (2 k + 1) 2^-24, k < 2^22, one point per
// thread and round (v_k is exact in binary32 and equal to mirrored_v of any
// word whose uniform is u_k or 1 - u_k).
__global__ void __launch_bounds__(256) mlp_grid_kernel(MlpWeights *m) {
    __shared__ MlpShared s;
    mlp_stage(s, m);
    __syncthreads();
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < MLP_GRID; k += gridDim.x * blockDim.x) {
        const float v = __fmul_rn((float)(2u * k + 1u), 0x1p-24f);
        m->ygrid[k] = mlp_eval16(s, m->tanh16, mlp_feature(v));
    }
}

// The weights' derived data: the activation table, then the tabulated
// network (a multiple of the SM count in blocks of 256).
cudaError_t mlp_refresh(MlpWeights *m, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    mlp_tanh16_kernel<<<MLP_TANH16 / 256, 256, 0, s>>>(m);
    mlp_grid_kernel<<<8 * sms, 256, 0, s>>>(m);
    return cudaGetLastError();
}

}  // namespace mlmc

using namespace mlmc;

extern "C" {

mlmc_status mlmc_mlp_set_weights(const float *w_host, size_t n) {
    if (!w_host || n != MLMC_MLP_PARAMS) return fail(MLMC_EINVAL, "expected %d weights", MLMC_MLP_PARAMS);
    for (size_t i = 0; i < n; ++i)
        if (!isfinite(w_host[i])) return fail(MLMC_EINVAL, "non-finite weight at %zu", i);
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    cudaError_t e = cudaMemcpy(d->mlp->w, w_host, n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = mlp_refresh(d->mlp, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "mlmc_mlp_set_weights");
    d->mlp_ready = true;
    return MLMC_OK;
}

mlmc_status mlmc_mlp_grid_table(float *y_host, size_t n) {
    if (!y_host || n != MLP_GRID) return fail(MLMC_EINVAL, "expected %u values", MLP_GRID);
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    if (!d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    cudaError_t e = cudaMemcpy(y_host, d->mlp->ygrid, n * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "mlmc_mlp_grid_table");
}

mlmc_status mlmc_mlp_get_weights(float *w_host, size_t n) {
    if (!w_host || n != MLMC_MLP_PARAMS) return fail(MLMC_EINVAL, "expected %d weights", MLMC_MLP_PARAMS);
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    if (!d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    cudaError_t e = cudaMemcpy(w_host, d->mlp->w, n * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "mlmc_mlp_get_weights");
}

}  // extern "C"
