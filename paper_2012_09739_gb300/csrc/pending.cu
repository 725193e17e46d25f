// Entry points whose device side is not built yet: they validate nothing
// and report that the feature is unavailable.
#include "api_internal.h"

using namespace mlmc;

namespace mlmc {
void release_device_extras(DeviceState &d) { (void)d; }
}

extern "C" {

mlmc_status mlmc_mlp_grad(const float *, const float *, size_t, float *, float *, void *) {
    return fail(MLMC_EINVAL, "mlmc_mlp_grad: not available in this build");
}
mlmc_status mlmc_mlp_train(const float *, const float *, size_t, const mlmc_train_opts *, float *, void *) {
    return fail(MLMC_EINVAL, "mlmc_mlp_train: not available in this build");
}
mlmc_status mlmc_batch(const mlmc_work *, int, uint64_t, mlmc_sums *, void *) {
    return fail(MLMC_EINVAL, "mlmc_batch: not available in this build");
}
mlmc_status mlmc_run(double, const mlmc_sde_params *, const mlmc_run_opts *, mlmc_run_result *) {
    return fail(MLMC_EINVAL, "mlmc_run: not available in this build");
}
mlmc_status mlmc_peak_probe(int, double *, void *) {
    return fail(MLMC_EINVAL, "mlmc_peak_probe: not available in this build");
}

}  // extern "C"
