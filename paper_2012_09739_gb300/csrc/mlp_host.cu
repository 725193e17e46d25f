// MLP weights on the device: the FP32 master copy, its binary16 W2, and the
// network tabulated on the 24-bit uniform grid.
#include <vector>

#include "api_internal.h"
#include "mlp_tc.cuh"

namespace mlmc {

__global__ void mlp_refresh_half_kernel(MlpWeights *m) {
    for (int i = threadIdx.x; i < MLP_H * MLP_H; i += blockDim.x) m->w2h[i] = __float2half_rn(m->w[64 + i]);
}

// y(v_k) for every grid point v_k = (2 k + 1) 2^-24, k < 2^22, by the
// tensor-core inference: two points per lane, every lane of every warp
// active (the grid is a multiple of 64 rows).  v_k is exact in binary32 and
// equal to mirrored_v of any word whose uniform is u_k or 1 - u_k.
__global__ void __launch_bounds__(256) mlp_grid_kernel(MlpWeights *m) {
    MlpFrags F;
    F.load(m);
    const uint32_t k0 = 2u * (blockIdx.x * blockDim.x + threadIdx.x), k1 = k0 + 1u;
    const float v0 = __fmul_rn((float)(2u * k0 + 1u), 0x1p-24f), v1 = __fmul_rn((float)(2u * k1 + 1u), 0x1p-24f);
    const float2 y = mlp_eval_warp(F, mlp_feature(v0), mlp_feature(v1));
    m->ygrid[k0] = y.x;
    m->ygrid[k1] = y.y;
}

// The weights' derived data: binary16 W2, then the tabulated network.
cudaError_t mlp_refresh_half(MlpWeights *m, cudaStream_t s) {
    mlp_refresh_half_kernel<<<1, 256, 0, s>>>(m);
    mlp_grid_kernel<<<MLP_GRID / 512, 256, 0, s>>>(m);
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
