// MLP weights on the device: the FP32 master copy and its binary16 W2.
#include <vector>

#include "api_internal.h"

namespace mlmc {

__global__ void mlp_refresh_half_kernel(MlpWeights *m) {
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) m->w2h[i] = __float2half_rn(m->w[64 + i]);
}

cudaError_t mlp_refresh_half(MlpWeights *m, cudaStream_t s) {
    mlp_refresh_half_kernel<<<1, 256, 0, s>>>(m);
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
    if (e == cudaSuccess) e = mlp_refresh_half(d->mlp, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "mlmc_mlp_set_weights");
    d->mlp_ready = true;
    return MLMC_OK;
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
