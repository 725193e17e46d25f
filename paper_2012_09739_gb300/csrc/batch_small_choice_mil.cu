// Instantiations of the fused choice kernel (batch_small_kernel, MODE_CHOICE)
// for GBM with the Milstein scheme: the per-level choice's candidate rounds
// of Milstein runs in one launch (the Euler ones in batch_small_choice.cu).
#include "batch_kernels.cuh"
#include "internal.h"

namespace mlmc {

static const BatchSmallFn k_small_choice_mil[2] = {
    &batch_small_kernel<MODE_CHOICE, P_F32, false, ICDF_TABLE, SDE_GBM_MIL>,
    &batch_small_kernel<MODE_CHOICE, P_F32, false, ICDF_TABLE16, SDE_GBM_MIL>,
};

BatchSmallFn batch_small_choice_mil(int icdf) {
    if (icdf == MLMC_ICDF_TABLE) return k_small_choice_mil[0];
    if (icdf == MLMC_ICDF_TABLE16) return k_small_choice_mil[1];
    return nullptr;
}

}  // namespace mlmc
