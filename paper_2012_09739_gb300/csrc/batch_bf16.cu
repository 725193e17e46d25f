// Instantiations of the batched kernel in working precision bf16.
#include "batch_kernels.cuh"

namespace mlmc {

static const BatchKernelFn k_batch[2][5] = {
    {&batch_kernel<P_BF16, false, ICDF_EXACT>, &batch_kernel<P_BF16, false, ICDF_TABLE>, &batch_kernel<P_BF16, false, ICDF_MLP>,
     &batch_kernel<P_BF16, false, ICDF_TABLE16>,
     &batch_kernel<P_BF16, false, ICDF_CUBIC>},
    {&batch_kernel<P_BF16, true, ICDF_EXACT>, &batch_kernel<P_BF16, true, ICDF_TABLE>, &batch_kernel<P_BF16, true, ICDF_MLP>,
     &batch_kernel<P_BF16, true, ICDF_TABLE16>,
     &batch_kernel<P_BF16, true, ICDF_CUBIC>},
};

BatchKernelFn batch_kernel_bf16(int kahan, int icdf) {
    if (icdf < 0 || icdf > 4) return nullptr;
    return k_batch[kahan ? 1 : 0][icdf];
}

}  // namespace mlmc
