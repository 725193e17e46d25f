// Instantiations of the fused small-round kernel (batch_small_kernel) for the
// adaptive driver's standard-estimator rounds: two-way, binary32, exact
// normals, with and without Kahan, GBM (Euler and Milstein) and OU.
#include "batch_kernels.cuh"
#include "internal.h"

namespace mlmc {

#define MLMC_ST(KAHAN, SDE) &batch_small_kernel<MODE_TWO, P_F32, KAHAN, ICDF_EXACT, SDE>

// [kahan][sde: GBM, OU, GBM-Milstein]
static const BatchSmallFn k_small_two[2][3] = {
    {MLMC_ST(false, SDE_GBM), MLMC_ST(false, SDE_OU), MLMC_ST(false, SDE_GBM_MIL)},
    {MLMC_ST(true, SDE_GBM), MLMC_ST(true, SDE_OU), MLMC_ST(true, SDE_GBM_MIL)},
};

BatchSmallFn batch_small_two(int prec, int kahan, int icdf, int sde) {
    if (prec != MLMC_F32 || icdf != MLMC_ICDF_EXACT || sde < SDE_GBM || sde > SDE_GBM_MIL) return nullptr;
    return k_small_two[kahan ? 1 : 0][sde];
}

}  // namespace mlmc
