// Instantiations of the fused small-round kernel (batch_small_kernel) for the
// per-level choice's candidate rounds (MODE_CHOICE): every candidate variant
// of one approximate inverse CDF (the table, the table at 16-bit uniforms or
// the network's tabulation) and the standard exact-normal term in one
// launch, GBM with the Euler scheme (the Milstein ones in
// batch_small_choice_mil.cu).
#include "batch_kernels.cuh"
#include "internal.h"

namespace mlmc {

BatchSmallFn batch_small_choice_mil(int icdf);

static const BatchSmallFn k_small_choice[3] = {
    &batch_small_kernel<MODE_CHOICE, P_F32, false, ICDF_TABLE, SDE_GBM>,
    &batch_small_kernel<MODE_CHOICE, P_F32, false, ICDF_TABLE16, SDE_GBM>,
    &batch_small_kernel<MODE_CHOICE, P_F32, false, ICDF_MLP, SDE_GBM>,
};

BatchSmallFn batch_small_choice(int icdf, int sde) {
    if (sde == SDE_GBM_MIL) return batch_small_choice_mil(icdf);
    if (sde != SDE_GBM) return nullptr;
    if (icdf == MLMC_ICDF_TABLE) return k_small_choice[0];
    if (icdf == MLMC_ICDF_TABLE16) return k_small_choice[1];
    if (icdf == MLMC_ICDF_MLP) return k_small_choice[2];
    return nullptr;
}

}  // namespace mlmc
