// Instantiations of the fused small-round kernel (batch_small_kernel) for the
// adaptive driver's nested rounds: both estimators' items of one variant in
// one launch (MODE_MIXED), binary16 and binary32, with and without Kahan,
// table and 16-bit-uniform table normals, GBM with the Euler scheme.
#include "batch_kernels.cuh"
#include "internal.h"

namespace mlmc {

#define MLMC_SM(P, KAHAN, ICDF) &batch_small_kernel<MODE_MIXED, P, KAHAN, ICDF, SDE_GBM>

// [prec: F32, F16][kahan][icdf: TABLE, TABLE16]
static const BatchSmallFn k_small_mixed[2][2][2] = {
    {{MLMC_SM(P_F32, false, ICDF_TABLE), MLMC_SM(P_F32, false, ICDF_TABLE16)},
     {MLMC_SM(P_F32, true, ICDF_TABLE), MLMC_SM(P_F32, true, ICDF_TABLE16)}},
    {{MLMC_SM(P_F16, false, ICDF_TABLE), MLMC_SM(P_F16, false, ICDF_TABLE16)},
     {MLMC_SM(P_F16, true, ICDF_TABLE), MLMC_SM(P_F16, true, ICDF_TABLE16)}},
};

BatchSmallFn batch_small_mixed(int prec, int kahan, int icdf, int sde) {
    if (sde != SDE_GBM || (prec != MLMC_F32 && prec != MLMC_F16)) return nullptr;
    if (icdf != MLMC_ICDF_TABLE && icdf != MLMC_ICDF_TABLE16) return nullptr;
    return k_small_mixed[prec == MLMC_F16 ? 1 : 0][kahan ? 1 : 0][icdf == MLMC_ICDF_TABLE ? 0 : 1];
}

}  // namespace mlmc
