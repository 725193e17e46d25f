// Instantiations of the level kernels in working precision f32.
#include "level_kernels.cuh"

namespace mlmc {

#define MLMC_K(MODE, KAHAN, ICDF, SDE) &level_kernel<MODE, P_F32, KAHAN, ICDF, SDE>
#define MLMC_SDES(MODE, KAHAN, ICDF) \
    {MLMC_K(MODE, KAHAN, ICDF, SDE_GBM), MLMC_K(MODE, KAHAN, ICDF, SDE_OU), MLMC_K(MODE, KAHAN, ICDF, SDE_GBM_MIL)}

// [mode][kahan][icdf][sde: GBM, OU, GBM with Milstein]; the four-way difference needs approximate normals
// on its bar pair, so its EXACT slot is empty.
static const LevelKernelFn k_table[2][2][5][3] = {
    {{MLMC_SDES(MODE_TWO, false, ICDF_EXACT), MLMC_SDES(MODE_TWO, false, ICDF_TABLE), MLMC_SDES(MODE_TWO, false, ICDF_MLP),
      MLMC_SDES(MODE_TWO, false, ICDF_TABLE16),
      MLMC_SDES(MODE_TWO, false, ICDF_CUBIC)},
     {MLMC_SDES(MODE_TWO, true, ICDF_EXACT), MLMC_SDES(MODE_TWO, true, ICDF_TABLE), MLMC_SDES(MODE_TWO, true, ICDF_MLP),
      MLMC_SDES(MODE_TWO, true, ICDF_TABLE16),
      MLMC_SDES(MODE_TWO, true, ICDF_CUBIC)}},
    {{{nullptr, nullptr, nullptr}, MLMC_SDES(MODE_FOUR, false, ICDF_TABLE), MLMC_SDES(MODE_FOUR, false, ICDF_MLP),
      MLMC_SDES(MODE_FOUR, false, ICDF_TABLE16),
      MLMC_SDES(MODE_FOUR, false, ICDF_CUBIC)},
     {{nullptr, nullptr, nullptr}, MLMC_SDES(MODE_FOUR, true, ICDF_TABLE), MLMC_SDES(MODE_FOUR, true, ICDF_MLP),
      MLMC_SDES(MODE_FOUR, true, ICDF_TABLE16),
      MLMC_SDES(MODE_FOUR, true, ICDF_CUBIC)}},
};

LevelKernelFn level_kernel_f32(int mode, int kahan, int icdf, int sde) {
    if (mode < 0 || mode > 1 || icdf < 0 || icdf > 4 || sde < 0 || sde > 2) return nullptr;
    return k_table[mode][kahan ? 1 : 0][icdf][sde];
}

}  // namespace mlmc
