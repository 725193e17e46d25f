// Allocation-free level estimate (mlmc_level_noalloc).
//
// Some callers cannot allocate device memory at the time they want a level
// estimate: a service that reserves all of HBM at start-up for its own
// allocator, a latency-critical loop where cudaMalloc/cudaMallocAsync could
// synchronise the device or fail under memory pressure, or a host framework
// whose policy forbids allocation outside its own pools.  For them this file
// keeps everything the level kernels need in file-scope device arrays that
// exist from the moment the library's module is loaded on a GPU until the
// process exits: the per-block scratch of partial sums and a private copy of
// the piecewise-linear table.  No cudaMalloc, cudaFree or allocating library
// routine is called here.
#include <mutex>

#include "api_internal.h"

namespace mlmc {

// Scratch: one (sum D, sum D^2) pair per block.  The launch uses one sample
// pair per thread, so a call needs ceil(ceil(N/2) / 256) blocks; the array
// holds NOALLOC_MAX_BLOCKS of them (64 KiB), i.e. N <= 2,097,152 samples.
constexpr int NOALLOC_BLOCK = 256;
constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr uint64_t NOALLOC_MAX_N = (uint64_t)NOALLOC_MAX_BLOCKS * NOALLOC_BLOCK * 2;

static __device__ __align__(256) double2 g_noalloc_partials[NOALLOC_MAX_BLOCKS];
// Private tables (same construction as the per-device tables of the other entry points).
static __device__ __align__(256) DevTables g_noalloc_tabs;

// Device addresses of the arrays above, looked up once per device with that
// device current.  In host code the array names are host-side stand-ins, not
// device addresses, so kernels only ever receive these looked-up pointers.
struct NoallocState {
    bool ready = false;
    double2 *partials = nullptr;
    DevTables *tabs = nullptr;
};
static std::mutex g_noalloc_mu;
static NoallocState g_noalloc[MAX_DEVICES];

// Every call looks the array addresses up again (no allocation, a table
// lookup in the runtime): if the module was loaded anew since the last call
// on this device -- after a reset of the device's primary context, say --
// the arrays have moved and hold no table, so the private table is built
// again.  A (re)build runs on `s` and waits for it, so the first call on a
// device should come before any stream capture that includes this entry
// point.
static mlmc_status noalloc_setup(int dev, cudaStream_t s, NoallocState **out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocState &st = g_noalloc[dev];
    cudaError_t e;
    double2 *partials = nullptr;
    DevTables *tabs = nullptr;
    if ((e = cudaGetSymbolAddress((void **)&partials, g_noalloc_partials)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    if ((e = cudaGetSymbolAddress((void **)&tabs, g_noalloc_tabs)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress(table)");
    if (!st.ready || partials != st.partials || tabs != st.tabs) {
        st.ready = false;
        st.partials = partials;
        st.tabs = tabs;
        if ((e = launch_build_table(st.tabs, s)) != cudaSuccess)
            return cuda_fail(e, "build_table");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "build_table");
        st.ready = true;
    }
    *out = &st;
    return MLMC_OK;
}

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_level_noalloc(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                                          const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset,
                                          double *sums_dev, void *stream) {
    mlmc_status st = check_level(four, l, N, prec, icdf, params);
    if (st) return st;
    if (!sums_dev) return fail(MLMC_EINVAL, "sums_dev is NULL");
    if (icdf == MLMC_ICDF_MLP)
        return fail(MLMC_EINVAL, "mlmc_level_noalloc supports the exact and table inverse CDFs only");
    if (N > NOALLOC_MAX_N)
        return fail(MLMC_EINVAL, "mlmc_level_noalloc: N = %llu exceeds its fixed scratch (at most %llu samples)",
                    (unsigned long long)N, (unsigned long long)NOALLOC_MAX_N);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return fail(MLMC_EINVAL, "device %d out of range", dev);
    cudaStream_t s = (cudaStream_t)stream;
    NoallocState *na;
    if ((st = noalloc_setup(dev, s, &na))) return st;

    LevelKernelFn fn = pick_level_kernel(four ? 1 : 0, prec, kahan, icdf, kernel_sde(params));
    if (!fn) return fail(MLMC_EINVAL, "no kernel for this variant");
    // make_level_args only reads the table pointers from the state it is given
    DeviceState view;
    view.tabs = na->tabs;
    LevelArgs a = make_level_args(view, four ? 1 : 0, l, N, prec, icdf, params, seed, path_offset, 0);
    a.partials = na->partials;
    a.paths_out = nullptr;
    const int grid = (int)((a.npairs + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
    fn<<<grid, NOALLOC_BLOCK, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "level kernel launch");
    // grid <= 4096 partials: one finalize block, no finalize scratch
    if ((e = launch_finalize(na->partials, grid, sums_dev, nullptr, s)) != cudaSuccess) return cuda_fail(e, "finalize");
    return MLMC_OK;
}
