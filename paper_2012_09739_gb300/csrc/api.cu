// C ABI of the library (include/mlmc.h): argument checking, per-device
// state, launch configuration, and the host side of every entry point.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "api_internal.h"
#include "level_kernels.cuh"

namespace mlmc {

// ---------------------------------------------------------------- errors
static thread_local char g_last_error[512] = "";

mlmc_status fail(mlmc_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

mlmc_status cuda_fail(cudaError_t e, const char *where) {
    return fail(e == cudaErrorMemoryAllocation ? MLMC_ENOMEM : MLMC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// ---------------------------------------------------------------- device state
static std::mutex g_mu;
static DeviceState g_dev[MAX_DEVICES];

mlmc_status device_state(DeviceState **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return fail(MLMC_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceState &d = g_dev[dev];
    if (!d.ready) {
        if ((e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        if ((e = cudaMalloc(&d.tabs, sizeof(DevTables))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(table)");
        if ((e = cudaMalloc(&d.mlp, sizeof(MlpWeights))) != cudaSuccess) return cuda_fail(e, "cudaMalloc(mlp)");
        if ((e = cudaMemset(d.mlp, 0, sizeof(MlpWeights))) != cudaSuccess) return cuda_fail(e, "cudaMemset(mlp)");
        if ((e = launch_build_table(d.tabs, 0)) != cudaSuccess)
            return cuda_fail(e, "build_table");
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "build_table");
        d.device = dev;
        d.ready = true;
    }
    *out = &d;
    return MLMC_OK;
}

// ---------------------------------------------------------------- waiting
double wait_limit_s() {
    static double limit = [] {
        const char *s = getenv("MLMC_TIMEOUT_S");
        double v = s ? atof(s) : 0.0;
        return v > 0.0 ? v : 600.0;
    }();
    return limit;
}

// Polls the event: yields the core for the first 2 ms (short GPU work is
// picked up within a poll), then sleeps 20 us between polls.
mlmc_status wait_event(cudaEvent_t ev, double limit_s) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return MLMC_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "wait");
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit_s) return fail(MLMC_ETIMEOUT, "wait exceeded %.1f s", limit_s);
        if (el < 2e-3) std::this_thread::yield();
        else std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// ---------------------------------------------------------------- validation
mlmc_status check_params(const mlmc_sde_params *p) {
    if (!p) return fail(MLMC_EINVAL, "params is NULL");
    if (p->sde != MLMC_GBM && p->sde != MLMC_OU) return fail(MLMC_EINVAL, "unknown sde %d", p->sde);
    if (p->payoff != MLMC_PAYOFF_X && p->payoff != MLMC_PAYOFF_CALL) return fail(MLMC_EINVAL, "unknown payoff");
    if (p->scheme != MLMC_EULER && p->scheme != MLMC_MILSTEIN) return fail(MLMC_EINVAL, "unknown scheme %d", p->scheme);
    if (p->reserved != 0) return fail(MLMC_EINVAL, "reserved field must be 0");
    const double v[] = {p->p0, p->p1, p->p2, p->x0, p->T, p->K, p->disc};
    for (double x : v)
        if (!isfinite(x)) return fail(MLMC_EINVAL, "non-finite SDE parameter");
    if (!(p->T > 0.0)) return fail(MLMC_EINVAL, "T must be > 0");
    if (p->sde == MLMC_GBM && !(p->p1 > 0.0)) return fail(MLMC_EINVAL, "GBM sigma must be > 0");
    if (p->sde == MLMC_OU && !(p->p2 > 0.0)) return fail(MLMC_EINVAL, "OU s must be > 0");
    return MLMC_OK;
}

mlmc_status check_level(int four, int l, uint64_t N, int prec, int icdf, const mlmc_sde_params *p) {
    if (l < 0 || l > 18) return fail(MLMC_EINVAL, "level %d outside 0..18", l);
    if (N == 0) return fail(MLMC_EINVAL, "N must be >= 1");
    if (N > (1ull << 40)) return fail(MLMC_EINVAL, "N too large");
    if (prec != MLMC_F32 && prec != MLMC_F16 && prec != MLMC_BF16) return fail(MLMC_EINVAL, "unknown precision %d", prec);
    if (icdf < 0 || icdf > 4) return fail(MLMC_EINVAL, "unknown icdf %d", icdf);
    if (four && icdf == MLMC_ICDF_EXACT) return fail(MLMC_EINVAL, "four-way difference needs approximate normals");
    return check_params(p);
}

// ---------------------------------------------------------------- launches
// A binary64 constant rounded once to nearest even, as the pair bits of the
// working precision (CUDA's host conversions to binary16 / bfloat16 round
// directly from binary64).
static uint32_t pair_bits(double v, int prec) {
    if (prec == MLMC_F16) {
        const __half_raw h = __double2half(v);
        return (uint32_t)h.x | ((uint32_t)h.x << 16);
    }
    if (prec == MLMC_BF16) {
        const __nv_bfloat16_raw b = __double2bfloat16(v);
        return (uint32_t)b.x | ((uint32_t)b.x << 16);
    }
    const float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

LevelArgs make_level_args(const DeviceState &d, int four, int l, uint64_t N, int prec, int icdf,
                          const mlmc_sde_params *p, uint64_t seed, uint64_t path_offset, uint32_t set_id) {
    LevelArgs a;
    memset(&a, 0, sizeof a);
    const double delta_f = ldexp(p->T, -l);
    const double sq = sqrt(delta_f);
    a.l = l;
    a.payoff = p->payoff;
    a.mode = four ? MODE_FOUR : MODE_TWO;
    a.sde = kernel_sde(p);
    a.prec = prec;
    a.icdf = icdf;
    a.N = N;
    a.unit = unit_pairs(a.mode, icdf, l);
    a.npairs = (N + 2 * a.unit - 1) / (2 * a.unit);
    a.path_offset = path_offset;
    const uint32_t kind = four ? 2u : (icdf == MLMC_ICDF_EXACT ? 0u : 1u);
    a.tag = kind | ((uint32_t)l << 8) | (set_id << 16);
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.rk = philox_round_keys(a.k0, a.k1);
    a.drift_f = p->p0 * delta_f;
    a.drift_c = p->p0 * (2.0 * delta_f);
    if (p->sde == MLMC_GBM) {
        a.diff = p->p1 * sq;
        a.mean = 0.0;
        a.mil = 0.5 * p->p1 * p->p1 * delta_f;
    } else {
        a.diff = p->p2 * sq;
        a.mean = p->p1;
    }
    a.x0 = p->x0;
    a.K = p->K;
    a.disc = p->disc;
    const double cv[8] = {a.drift_f, a.drift_c, a.diff, a.mean, a.x0, a.mil, 1.0, 2.0};
    for (int i = 0; i < 8; ++i) {
        a.cw[i] = pair_bits(cv[i], prec);
        a.c32[i] = (float)cv[i];
    }
    a.K32 = (float)p->K;
    a.disc32 = (float)p->disc;
    a.tabs = d.tabs;
    a.mlp = d.mlp;
    return a;
}

// Kernel SDE kind: Milstein only changes GBM (b' = 0 for OU).
int kernel_sde(const mlmc_sde_params *p) {
    if (p->sde == MLMC_OU) return SDE_OU;
    return p->scheme == MLMC_MILSTEIN ? SDE_GBM_MIL : SDE_GBM;
}

LevelKernelFn pick_level_kernel(int four, int prec, int kahan, int icdf, int sde) {
    return prec == MLMC_F32   ? level_kernel_f32(four, kahan, icdf, sde)
           : prec == MLMC_F16 ? level_kernel_f16(four, kahan, icdf, sde)
                              : level_kernel_bf16(four, kahan, icdf, sde);
}

static int env_int(const char *name, int dflt) {
    const char *s = getenv(name);
    return s ? atoi(s) : dflt;
}

// Launch shape: a persistent grid of every resident block (256 threads, the
// occupancy limit of blocks per SM) when the chunks outnumber the resident
// warps, else one block per 8 chunks.  MLMC_BLOCK / MLMC_BLOCKS_PER_SM
// override the block size and the blocks per SM.
LaunchCfg level_launch_cfg(const DeviceState &d, LevelKernelFn fn, uint64_t npairs) {
    LaunchCfg c;
    int bt = env_int("MLMC_BLOCK", 256);
    if (bt < 32 || bt > 256 || bt % 32) bt = 256;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, bt, 0) != cudaSuccess || occ < 1) occ = 1;
    const int k = env_int("MLMC_BLOCKS_PER_SM", 0);
    if (k > 0 && k < occ) occ = k;
    const uint64_t chunks = (npairs + 31) / 32, per_block = (uint64_t)bt / 32;
    const uint64_t resident = (uint64_t)occ * d.sm_count;
    c.block = bt;
    c.grid = (int)std::max<uint64_t>(1, std::min(resident, (chunks + per_block - 1) / per_block));
    return c;
}

// Chunk groups up to which each group gets its own partial sum.
constexpr uint64_t MAX_CHUNK_PARTIALS = 1ull << 22;

mlmc_status enqueue_level(const DeviceState &d, int four, int l, uint64_t N, int prec, int kahan, int icdf,
                          const mlmc_sde_params *p, uint64_t seed, uint64_t path_offset, uint32_t set_id,
                          double *sums_dev, float *paths_dev, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    LevelKernelFn fn = pick_level_kernel(four, prec, kahan, icdf, kernel_sde(p));
    if (!fn) return fail(MLMC_EINVAL, "no kernel for this variant");
    LevelArgs a = make_level_args(d, four, l, N, prec, icdf, p, seed, path_offset, set_id);
    const LaunchCfg cfg = level_launch_cfg(d, fn, a.npairs);
    const uint64_t chunks = (a.npairs + 31) / 32;
    const uint64_t G = chunk_group(l, chunks);
    const uint64_t groups = (chunks + G - 1) / G;
    a.chunk_partials = groups <= MAX_CHUNK_PARTIALS ? 1 : 0;
    const uint64_t slots = a.chunk_partials ? groups : (uint64_t)cfg.grid;
    const uint64_t fin = finalize_scratch(slots);
    double2 *partials = nullptr;
    // partial slots, the chunk counter (zeroed), the finalize scratch
    cudaError_t e = cudaMallocAsync(&partials, (slots + 1 + fin) * sizeof(double2), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(partials)");
    a.partials = partials;
    a.counter = reinterpret_cast<unsigned long long *>(partials + slots);
    if (a.chunk_partials && (e = cudaMemsetAsync(a.counter, 0, 8, s)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync");
    a.paths_out = paths_dev;
    if (ev0) cudaEventRecord(ev0, s);
    fn<<<cfg.grid, cfg.block, 0, s>>>(a);
    e = cudaGetLastError();
    if (ev1) cudaEventRecord(ev1, s);
    if (e == cudaSuccess && sums_dev) e = launch_finalize(partials, slots, sums_dev, partials + slots + 1, s);
    cudaError_t e2 = cudaFreeAsync(partials, s);
    if (e != cudaSuccess) return cuda_fail(e, "level kernel launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFreeAsync");
    return MLMC_OK;
}

// Sample mean and unbiased variance of a level's differences from their
// FP64 sums (Sec. 3); every result struct and the adaptive driver use it.
void level_moments(double s1, double s2, uint64_t n, double *mean, double *var) {
    const double m = s1 / (double)n;
    *mean = m;
    *var = n > 1 ? fmax((s2 - s1 * m) / (double)(n - 1), 0.0) : 0.0;
}

// Per-thread pinned staging for small device->host results.
double *host_staging() {
    static thread_local double *buf = nullptr;
    if (!buf && cudaMallocHost(&buf, 64 * sizeof(double)) != cudaSuccess) buf = nullptr;
    return buf;
}

mlmc_status level_sync(int four, int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *p,
                       uint64_t seed, uint64_t path_offset, mlmc_sums *out, void *stream) {
    mlmc_status st = check_level(four, l, N, prec, icdf, p);
    if (st) return st;
    if (!out) return fail(MLMC_EINVAL, "out_host is NULL");
    DeviceState *d;
    if ((st = device_state(&d))) return st;
    if (icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    cudaStream_t s = (cudaStream_t)stream;
    // the finalize kernel writes the two sums straight into pinned host
    // memory (device-accessible under unified addressing); the events are
    // the calling thread's own, created once
    double *host = host_staging();
    if (!host) return fail(MLMC_ENOMEM, "cudaMallocHost");
    struct Events {
        cudaEvent_t t0 = nullptr, t1 = nullptr, done = nullptr;
    };
    static thread_local Events evs[MAX_DEVICES];
    Events &E = evs[d->device];
    if (!E.done) {
        if (cudaEventCreate(&E.t0) != cudaSuccess || cudaEventCreate(&E.t1) != cudaSuccess ||
            cudaEventCreateWithFlags(&E.done, cudaEventDisableTiming) != cudaSuccess) {
            E.done = nullptr;
            return fail(MLMC_ECUDA, "cudaEventCreate");
        }
    }
    cudaEvent_t ev0 = E.t0, ev1 = E.t1, done = E.done;
    st = enqueue_level(*d, four, l, N, prec, kahan, icdf, p, seed, path_offset, 0, host, nullptr, s, ev0, ev1);
    cudaEventRecord(done, s);
    if (st == MLMC_OK) st = wait_event(done, wait_limit_s());
    if (st == MLMC_OK) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        out->s1 = host[0];
        out->s2 = host[1];
        out->n = N;
        out->cost_ns = (double)ms * 1e6;
        level_moments(out->s1, out->s2, N, &out->mean, &out->var);
    }
    return st;
}

}  // namespace mlmc

using namespace mlmc;

extern "C" {

mlmc_status mlmc_level(int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *params, uint64_t seed,
                       uint64_t path_offset, mlmc_sums *out_host, void *stream) {
    return level_sync(0, l, N, prec, kahan, icdf, params, seed, path_offset, out_host, stream);
}

mlmc_status mlmc_nested_level(int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *params,
                              uint64_t seed, uint64_t path_offset, mlmc_sums *out_host, void *stream) {
    return level_sync(1, l, N, prec, kahan, icdf, params, seed, path_offset, out_host, stream);
}

mlmc_status mlmc_level_async(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                             const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset, double *sums_dev,
                             void *stream) {
    mlmc_status st = check_level(four, l, N, prec, icdf, params);
    if (st) return st;
    if (!sums_dev) return fail(MLMC_EINVAL, "sums_dev is NULL");
    DeviceState *d;
    if ((st = device_state(&d))) return st;
    if (icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    return enqueue_level(*d, four ? 1 : 0, l, N, prec, kahan, icdf, params, seed, path_offset, 0, sums_dev, nullptr,
                         (cudaStream_t)stream, nullptr, nullptr);
}

mlmc_status mlmc_level_paths(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                             const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset, float *out_dev,
                             void *stream) {
    mlmc_status st = check_level(four, l, N, prec, icdf, params);
    if (st) return st;
    if (!out_dev) return fail(MLMC_EINVAL, "out_dev is NULL");
    DeviceState *d;
    if ((st = device_state(&d))) return st;
    if (icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    return enqueue_level(*d, four ? 1 : 0, l, N, prec, kahan, icdf, params, seed, path_offset, 0, nullptr, out_dev,
                         (cudaStream_t)stream, nullptr, nullptr);
}

mlmc_status approx_icdf(const float *u_dev, void *z_dev, size_t n, int icdf, int prec, void *stream) {
    if (icdf < 0 || icdf > 4) return fail(MLMC_EINVAL, "unknown icdf %d", icdf);
    if (prec != MLMC_F32 && prec != MLMC_F16 && prec != MLMC_BF16) return fail(MLMC_EINVAL, "unknown precision %d", prec);
    if (n == 0) return MLMC_OK;
    if (!u_dev || !z_dev) return fail(MLMC_EINVAL, "NULL buffer");
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    if (icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    cudaError_t e = launch_icdf_bulk(u_dev, z_dev, n, icdf, prec, d->tabs, d->mlp, (cudaStream_t)stream);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "approx_icdf");
}

mlmc_status mlmc_philox4x32_10(const uint32_t *ctr_dev, const uint32_t *key_dev, uint32_t *out_dev, size_t n,
                               void *stream) {
    if (n == 0) return MLMC_OK;
    if (!ctr_dev || !key_dev || !out_dev) return fail(MLMC_EINVAL, "NULL buffer");
    if (((uintptr_t)ctr_dev | (uintptr_t)out_dev) & 15) return fail(MLMC_EINVAL, "ctr/out must be 16-byte aligned");
    if ((uintptr_t)key_dev & 7) return fail(MLMC_EINVAL, "key must be 8-byte aligned");
    cudaError_t e = launch_philox_bulk(ctr_dev, key_dev, out_dev, n, (cudaStream_t)stream);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "philox");
}

mlmc_status mlmc_uniforms(const uint32_t *w_dev, float *u_dev, size_t n, void *stream) {
    if (n == 0) return MLMC_OK;
    if (!w_dev || !u_dev) return fail(MLMC_EINVAL, "NULL buffer");
    cudaError_t e = launch_uniform_bulk(w_dev, u_dev, n, (cudaStream_t)stream);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "uniforms");
}

// Table entry (biased binary32 exponent E of v, minus 103) that holds
// 0-based interval i: E = 125 - i for i < 15, any E <= 110 for the last.
static int interval_entry(int i) { return i < 15 ? 22 - i : 0; }

static mlmc_status fetch_tables(DevTables *h) {
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    cudaError_t e = cudaMemcpy(h, d->tabs, sizeof(DevTables), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? MLMC_OK : cuda_fail(e, "copy of the tables");
}

mlmc_status mlmc_icdf_table(double *c_host, float *c32_host, uint16_t *c16_host, uint16_t *cbf16_host) {
    DevTables t;
    mlmc_status st = fetch_tables(&t);
    if (st) return st;
    for (int i = 0; i < 16; ++i) {
        const int entry = interval_entry(i);
        if (c_host) {
            c_host[2 * i] = t.lin64[2 * i];
            c_host[2 * i + 1] = t.lin64[2 * i + 1];
        }
        if (c32_host) {
            c32_host[2 * i] = t.e.c32[entry].x;
            c32_host[2 * i + 1] = t.e.c32[entry].y;
        }
        if (c16_host) {
            __half2_raw r = *reinterpret_cast<__half2_raw *>(&t.e.c16[entry]);
            c16_host[2 * i] = r.x;
            c16_host[2 * i + 1] = r.y;
        }
        if (cbf16_host) {
            cbf16_host[2 * i] = (uint16_t)(t.e.cb16[entry] & 0xFFFFu);
            cbf16_host[2 * i + 1] = (uint16_t)(t.e.cb16[entry] >> 16);
        }
    }
    return MLMC_OK;
}

mlmc_status mlmc_icdf_cubic(double *d_host, float *d32_host, uint16_t *d16_host, uint16_t *dbf16_host) {
    DevTables t;
    mlmc_status st = fetch_tables(&t);
    if (st) return st;
    for (int i = 0; i < 16; ++i) {
        const int entry = interval_entry(i);
        const float4 q = t.e.q32[entry];
        const float q32[4] = {q.x, q.y, q.z, q.w};
        const uint2 h = t.e.q16[entry], b = t.e.qbf[entry];
        const uint32_t h16[4] = {h.x & 0xFFFFu, h.x >> 16, h.y & 0xFFFFu, h.y >> 16};
        const uint32_t b16[4] = {b.x & 0xFFFFu, b.x >> 16, b.y & 0xFFFFu, b.y >> 16};
        for (int j = 0; j < 4; ++j) {
            if (d_host) d_host[4 * i + j] = t.cub64[4 * i + j];
            if (d32_host) d32_host[4 * i + j] = q32[j];
            if (d16_host) d16_host[4 * i + j] = (uint16_t)h16[j];
            if (dbf16_host) dbf16_host[4 * i + j] = (uint16_t)b16[j];
        }
    }
    return MLMC_OK;
}

mlmc_status mlmc_moments(const double *sums_host, uint64_t n, double *mean_host, double *var_host) {
    if (!sums_host || !mean_host || !var_host || n == 0) return fail(MLMC_EINVAL, "bad arguments");
    level_moments(sums_host[0], sums_host[1], n, mean_host, var_host);
    return MLMC_OK;
}

mlmc_status mlmc_optimal_samples(const double *V, const double *C, int n, double eps, uint64_t *N_out) {
    if (!V || !C || !N_out || n <= 0) return fail(MLMC_EINVAL, "bad arguments");
    if (!(eps > 0.0) || !isfinite(eps)) return fail(MLMC_EINVAL, "eps must be > 0");
    double total = 0.0;
    for (int i = 0; i < n; ++i) {
        if (!(V[i] >= 0.0) || !(C[i] > 0.0) || !isfinite(V[i]) || !isfinite(C[i]))
            return fail(MLMC_EINVAL, "V must be >= 0 and C > 0");
        total += sqrt(V[i] * C[i]);
    }
    for (int i = 0; i < n; ++i) {
        const double Ni = ceil(2.0 / (eps * eps) * sqrt(V[i] / C[i]) * total);
        N_out[i] = Ni < 1.0 ? 1 : (Ni > 1.8e19 ? (uint64_t)1.8e19 : (uint64_t)Ni);
    }
    return MLMC_OK;
}

const char *mlmc_strerror(mlmc_status s) {
    switch (s) {
    case MLMC_OK: return "ok";
    case MLMC_EINVAL: return "invalid argument";
    case MLMC_ECUDA: return "CUDA error";
    case MLMC_ETIMEOUT: return "timeout";
    case MLMC_ENOMEM: return "out of memory";
    case MLMC_ENOTCONV: return "not converged";
    case MLMC_ENOTREADY: return "MLP weights not set";
    }
    return "unknown status";
}

const char *mlmc_last_error(void) { return g_last_error; }

const char *mlmc_version(void) { return "mlmc-gb300 0.1 (sm_103a)"; }

mlmc_status mlmc_shutdown(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (int i = 0; i < MAX_DEVICES; ++i) {
        DeviceState &d = g_dev[i];
        if (!d.ready) continue;
        cudaSetDevice(i);
        release_device_extras(d);
        cudaFree(d.tabs);
        cudaFree(d.mlp);
        d = DeviceState();
    }
    cudaSetDevice(cur);
    return MLMC_OK;
}

}  // extern "C"
