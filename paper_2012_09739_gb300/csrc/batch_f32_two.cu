// Instantiations of the batched kernel: two-way estimator, working precision f32.
#include "batch_kernels.cuh"

namespace mlmc {

#define MLMC_B(KAHAN, ICDF, SDE) &batch_kernel<MODE_TWO, P_F32, KAHAN, ICDF, SDE>
#define MLMC_SDES(KAHAN, ICDF) {MLMC_B(KAHAN, ICDF, SDE_GBM), MLMC_B(KAHAN, ICDF, SDE_OU), MLMC_B(KAHAN, ICDF, SDE_GBM_MIL)}

// [kahan][icdf][sde: GBM, OU, GBM with Milstein]
static const BatchKernelFn k_batch[2][5][3] = {
    {MLMC_SDES(false, ICDF_EXACT), MLMC_SDES(false, ICDF_TABLE), MLMC_SDES(false, ICDF_MLP),
     MLMC_SDES(false, ICDF_TABLE16), MLMC_SDES(false, ICDF_CUBIC)},
    {MLMC_SDES(true, ICDF_EXACT), MLMC_SDES(true, ICDF_TABLE), MLMC_SDES(true, ICDF_MLP),
     MLMC_SDES(true, ICDF_TABLE16), MLMC_SDES(true, ICDF_CUBIC)},
};

BatchKernelFn batch_kernel_f32_two(int kahan, int icdf, int sde) {
    if (icdf < 0 || icdf > 4 || sde < 0 || sde > 2) return nullptr;
    return k_batch[kahan ? 1 : 0][icdf][sde];
}

}  // namespace mlmc
