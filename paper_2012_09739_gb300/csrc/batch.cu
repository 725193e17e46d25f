// Host side of mlmc_batch: warp tiles in longest-first order, one persistent
// launch per working-precision variant, a finalize kernel, all captured in a
// CUDA graph that is replayed while the item list is unchanged, and an
// autotuner for the tile size.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "batch_kernels.cuh"

namespace mlmc {

BatchKernelFn batch_kernel_f32(int kahan, int icdf);
BatchKernelFn batch_kernel_f16(int kahan, int icdf);
BatchKernelFn batch_kernel_bf16(int kahan, int icdf);

// Sums each item's tile partials in a fixed order, one warp per item, FP64.
__global__ void batch_finalize_kernel(const double2 *tile_partials, const uint32_t *start, const uint32_t *list,
                                      int nitems, double2 *sums) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= nitems) return;
    double s1 = 0.0, s2 = 0.0;
    for (uint32_t i = start[warp] + lane; i < start[warp + 1]; i += 32) {
        const double2 p = tile_partials[list[i]];
        s1 += p.x;
        s2 += p.y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    }
    if (lane == 0) sums[warp] = make_double2(s1, s2);
}

namespace {

struct Group {
    int prec, kahan, icdf;
    std::vector<Tile> tiles;
    uint32_t tile_base = 0;        // offset of this group's tiles in the device array
};

struct Plan {
    std::vector<LevelArgs> items;
    std::vector<Group> groups;
    std::vector<uint32_t> start, list;   // per-item tile lists (global tile indices)
    std::vector<double> weight;          // share of the launch's work per item
    uint32_t ntiles = 0;
};

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

double item_work(const mlmc_work &w) {
    return ldexp((double)((w.N + 1) / 2), w.l) * (w.kind ? 2.2 : 1.0);
}

// Tiles of `lane_pairs_log2` controls the work per lane per tile: a lane takes
// max(1, 2^lane_work_log2 / 2^l) pairs of an item at level l.
Plan make_plan(const DeviceState &d, const mlmc_work *w, int n, uint64_t seed, int lane_work_log2) {
    Plan plan;
    plan.items.resize(n);
    std::vector<std::vector<uint32_t>> per_item(n);
    double total = 0.0;
    for (int i = 0; i < n; ++i) total += item_work(w[i]);
    for (int i = 0; i < n; ++i) {
        plan.items[i] = make_level_args(d, w[i].kind, w[i].l, w[i].N, w[i].prec, w[i].icdf, &w[i].params, seed,
                                        w[i].path_offset, (uint32_t)w[i].set_id);
        plan.weight.push_back(total > 0 ? item_work(w[i]) / total : 0.0);
        Group *g = nullptr;
        for (auto &gg : plan.groups)
            if (gg.prec == w[i].prec && gg.kahan == (w[i].kahan ? 1 : 0) && gg.icdf == w[i].icdf) g = &gg;
        if (!g) {
            plan.groups.push_back(Group{w[i].prec, w[i].kahan ? 1 : 0, w[i].icdf, {}, 0});
            g = &plan.groups.back();
        }
        const uint64_t np = (w[i].N + 1) / 2;
        const uint64_t per_lane = std::max<uint64_t>(1, (1ull << lane_work_log2) >> w[i].l);
        const uint64_t per_tile = 32 * per_lane;
        for (uint64_t first = 0; first < np; first += per_tile)
            g->tiles.push_back(Tile{(uint32_t)i, (uint32_t)std::min<uint64_t>(per_tile, np - first), first});
    }
    uint32_t base = 0;
    for (auto &g : plan.groups) {
        // longest first: lane rounds x steps per pair, four-way weighted
        std::stable_sort(g.tiles.begin(), g.tiles.end(), [&](const Tile &a, const Tile &b) {
            const LevelArgs &ia = plan.items[a.item], &ib = plan.items[b.item];
            const double ca = ldexp((double)((a.npairs + 31) / 32), ia.l) * (ia.mode ? 2.2 : 1.0);
            const double cb = ldexp((double)((b.npairs + 31) / 32), ib.l) * (ib.mode ? 2.2 : 1.0);
            return ca > cb;
        });
        g.tile_base = base;
        for (uint32_t k = 0; k < g.tiles.size(); ++k) per_item[g.tiles[k].item].push_back(base + k);
        base += (uint32_t)g.tiles.size();
    }
    plan.ntiles = base;
    plan.start.push_back(0);
    for (int i = 0; i < n; ++i) {
        for (uint32_t t : per_item[i]) plan.list.push_back(t);
        plan.start.push_back((uint32_t)plan.list.size());
    }
    return plan;
}

BatchKernelFn pick_batch_kernel(int prec, int kahan, int icdf) {
    return prec == MLMC_F32 ? batch_kernel_f32(kahan, icdf)
                            : prec == MLMC_F16 ? batch_kernel_f16(kahan, icdf) : batch_kernel_bf16(kahan, icdf);
}

template <typename T>
cudaError_t grow(T **p, size_t *cap, size_t n) {
    if (n <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    size_t want = std::max<size_t>(n, 64);
    cudaError_t e = cudaMalloc(p, want * sizeof(T));
    if (e == cudaSuccess) *cap = want;
    return e;
}

}  // namespace

struct BatchCache {
    // descriptors, uploaded by one copy: items, tiles, per-item tile lists
    // and the schedule counters (zeroed by the same copy), 16-byte aligned
    unsigned char *blob = nullptr;
    size_t blob_cap = 0;
    LevelArgs *items = nullptr;
    Tile *tiles = nullptr;
    uint32_t *start = nullptr, *list = nullptr;
    uint32_t *counters = nullptr;
    double2 *partials = nullptr;
    size_t partials_cap = 0;
    double2 *sums = nullptr;
    size_t sums_cap = 0;
    double2 *sums_host = nullptr;
    size_t sums_host_cap = 0;
    unsigned char *stage = nullptr;      // pinned staging of the descriptors
    size_t stage_cap = 0;
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t sig = 0;
    std::vector<double> weight;
    std::map<uint64_t, int> tuned;       // item-list signature -> lane_work_log2
    std::map<const void *, int> occupancy;   // batch kernel -> resident blocks per SM
};

BatchCache *batch_cache_create() { return new BatchCache(); }

void batch_cache_destroy(BatchCache *c) {
    if (!c) return;
    if (c->exec) cudaGraphExecDestroy(c->exec);
    cudaFree(c->blob);
    cudaFree(c->partials);
    cudaFree(c->sums);
    if (c->sums_host) cudaFreeHost(c->sums_host);
    if (c->stage) cudaFreeHost(c->stage);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    delete c;
}

void release_device_extras(DeviceState &d) {
    batch_cache_destroy(d.batch);
    batch_cache_destroy(d.run_cache);
    if (d.run_stream) cudaStreamDestroy(d.run_stream);
    d.batch = d.run_cache = nullptr;
    d.run_stream = nullptr;
}

namespace {

// Uploads the plan into the cache's device buffers: the descriptors and the
// zeroed schedule counters are packed into pinned staging memory and copied
// to the device in one asynchronous copy on s (the buffers only grow, with
// cudaMalloc, when a larger batch arrives).
mlmc_status upload(BatchCache &c, const Plan &p, cudaStream_t s) {
    cudaError_t e;
    const size_t n = p.items.size();
    if ((e = grow(&c.partials, &c.partials_cap, p.ntiles)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if ((e = grow(&c.sums, &c.sums_cap, n)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if (c.sums_host_cap < n) {
        if (c.sums_host) cudaFreeHost(c.sums_host);
        c.sums_host = nullptr;
        c.sums_host_cap = 0;
        if ((e = cudaMallocHost(&c.sums_host, n * sizeof(double2))) != cudaSuccess) return cuda_fail(e, "pinned");
        c.sums_host_cap = n;
    }
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t b_items = n * sizeof(LevelArgs), b_tiles = (size_t)p.ntiles * sizeof(Tile);
    const size_t b_start = p.start.size() * 4, b_list = std::max<size_t>(p.list.size(), 1) * 4;
    const size_t b_cnt = p.groups.size() * 4;
    const size_t o_tiles = up16(b_items), o_start = o_tiles + up16(b_tiles), o_list = o_start + up16(b_start);
    const size_t o_cnt = o_list + up16(b_list), total = o_cnt + up16(b_cnt);
    if ((e = grow(&c.blob, &c.blob_cap, total)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if (c.stage_cap < total) {
        if (c.stage) cudaFreeHost(c.stage);
        c.stage = nullptr;
        c.stage_cap = 0;
        if ((e = cudaMallocHost(&c.stage, total * 2)) != cudaSuccess) return cuda_fail(e, "pinned");
        c.stage_cap = total * 2;
    }
    // the previous round's copy out of the staging buffer must be done
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "upload");
    c.items = reinterpret_cast<LevelArgs *>(c.blob);
    c.tiles = reinterpret_cast<Tile *>(c.blob + o_tiles);
    c.start = reinterpret_cast<uint32_t *>(c.blob + o_start);
    c.list = reinterpret_cast<uint32_t *>(c.blob + o_list);
    c.counters = reinterpret_cast<uint32_t *>(c.blob + o_cnt);
    unsigned char *h = c.stage;
    memset(h, 0, total);
    memcpy(h, p.items.data(), b_items);
    size_t off = o_tiles;
    for (const auto &g : p.groups) {
        memcpy(h + off, g.tiles.data(), g.tiles.size() * sizeof(Tile));
        off += g.tiles.size() * sizeof(Tile);
    }
    memcpy(h + o_start, p.start.data(), b_start);
    if (!p.list.empty()) memcpy(h + o_list, p.list.data(), p.list.size() * 4);
    if ((e = cudaMemcpyAsync(c.blob, h, total, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(e, "upload");
    return MLMC_OK;
}

// Enqueues the whole batch on stream s (also used inside graph capture).
// zero_counters: reset the schedule counters on the stream (a replayed graph
// needs it; a fresh upload has zeroed them already).
mlmc_status enqueue(const DeviceState &d, BatchCache &c, const Plan &p, cudaStream_t s, bool copy_out,
                    bool zero_counters) {
    cudaError_t e;
    if (zero_counters && (e = cudaMemsetAsync(c.counters, 0, p.groups.size() * sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "memset");
    for (size_t gi = 0; gi < p.groups.size(); ++gi) {
        const Group &g = p.groups[gi];
        BatchKernelFn fn = pick_batch_kernel(g.prec, g.kahan, g.icdf);
        int bps = 0;
        auto it = c.occupancy.find((const void *)fn);
        if (it != c.occupancy.end()) {
            bps = it->second;
        } else {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 256, 0) != cudaSuccess || bps < 1) bps = 1;
            c.occupancy[(const void *)fn] = bps;
        }
        const uint32_t warps_needed = (uint32_t)g.tiles.size();
        uint32_t grid = (uint32_t)bps * d.sm_count;
        grid = std::min<uint32_t>(grid, (warps_needed + 7) / 8);
        fn<<<grid ? grid : 1, 256, 0, s>>>(c.items, c.tiles + g.tile_base, (uint32_t)g.tiles.size(), c.counters + gi,
                                           c.partials + g.tile_base, d.tabs);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch kernel");
    }
    const int n = (int)p.items.size();
    // copy_out: the finalize kernel writes the sums straight into the pinned
    // host buffer (device-accessible under unified addressing), no copy
    double2 *dst = copy_out ? c.sums_host : c.sums;
    batch_finalize_kernel<<<(n * 32 + 255) / 256, 256, 0, s>>>(c.partials, c.start, c.list, n, dst);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch finalize");
    return MLMC_OK;
}

int env_int(const char *name, int dflt) {
    const char *s = getenv(name);
    return s ? atoi(s) : dflt;
}

// Times each candidate tile size once on the real batch and keeps the fastest.
// Tile size (log2 of the path-steps per lane) for a batch's total work:
// about four tiles per resident lane, clamped to [4, 12].
int work_lane_log2(const DeviceState &d, const mlmc_work *w, int n) {
    double steps = 0.0;
    for (int i = 0; i < n; ++i) steps += ldexp((double)((w[i].N + 1) / 2), w[i].l);
    const double lanes = (double)d.sm_count * 24 * 32;
    const int lw = (int)floor(log2(std::max(steps / (4.0 * lanes), 1.0)));
    return std::min(12, std::max(4, lw));
}

mlmc_status autotune(const DeviceState &d, BatchCache &c, const mlmc_work *w, int n, uint64_t seed, int *best) {
    // candidates around the work-based size (large batches favour longer tiles)
    const int base = work_lane_log2(d, w, n);
    const int cands[] = {base - 1, base, base + 1, base + 2};
    float best_ms = 1e30f;
    *best = base;
    cudaStream_t s = c.capture_stream;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    mlmc_status st = MLMC_OK;
    for (int lw : cands) {
        Plan p = make_plan(d, w, n, seed, lw);
        if ((st = upload(c, p, s))) break;
        cudaEventRecord(a, s);
        if ((st = enqueue(d, c, p, s, false, true))) break;
        cudaEventRecord(b, s);
        if ((st = wait_event(b, wait_limit_s()))) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best_ms) {
            best_ms = ms;
            *best = lw;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

}  // namespace

// One round of a caller that owns its own cache (the adaptive driver):
// descriptors, persistent kernels, finalize and the copy of all sums into
// c.sums_host, enqueued on s.  The caller waits on s before reading.
// The tile size follows the round's total work: about four tiles per
// resident lane, each at least 16 and at most 4096 steps long per lane.
mlmc_status batch_round(const DeviceState &d, BatchCache &c, const mlmc_work *w, int n, uint64_t seed,
                        cudaStream_t s) {
    Plan p = make_plan(d, w, n, seed, work_lane_log2(d, w, n));
    mlmc_status st = upload(c, p, s);
    if (st) return st;
    return enqueue(d, c, p, s, true, false);
}

const double2 *batch_sums_host(const BatchCache &c) { return c.sums_host; }

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_batch(const mlmc_work *items, int n_items, uint64_t seed, mlmc_sums *out_host,
                                  void *stream) {
    if (!items || n_items <= 0 || !out_host) return fail(MLMC_EINVAL, "bad batch arguments");
    for (int i = 0; i < n_items; ++i) {
        const mlmc_work &w = items[i];
        if (w.kind != 0 && w.kind != 1) return fail(MLMC_EINVAL, "item %d: kind must be 0 or 1", i);
        if (w.set_id < 0 || w.set_id > 0xFFFF) return fail(MLMC_EINVAL, "item %d: set_id outside 0..65535", i);
        if (w.N > 0xFFFFFFFFull * 32) return fail(MLMC_EINVAL, "item %d: N too large for a batch", i);
        mlmc_status st = check_level(w.kind, w.l, w.N, w.prec, w.icdf, &w.params);
        if (st) return fail(st, "item %d: %s", i, mlmc_last_error());
    }
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    // one batch at a time per process: the cached graph and buffers are shared
    static std::mutex batch_mu;
    std::lock_guard<std::mutex> lock(batch_mu);
    for (int i = 0; i < n_items; ++i)
        if (items[i].icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    if (!d->batch) {
        d->batch = new BatchCache();
        cudaError_t e = cudaStreamCreateWithFlags(&d->batch->capture_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    }
    BatchCache &c = *d->batch;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t sig = fnv1a(items, sizeof(mlmc_work) * n_items, fnv1a(&seed, sizeof seed));
    sig = fnv1a(&n_items, sizeof n_items, sig);

    if (!(c.exec && c.sig == sig)) {
        int lw = env_int("MLMC_BATCH_LANE_WORK_LOG2", 0);
        if (lw < 6 || lw > 20) {
            auto it = c.tuned.find(sig);
            if (it != c.tuned.end()) {
                lw = it->second;
            } else if (env_int("MLMC_AUTOTUNE", 1)) {
                // the capture stream must see the caller's prior work first
                cudaEvent_t ev;
                cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                cudaEventRecord(ev, s);
                cudaStreamWaitEvent(c.capture_stream, ev, 0);
                cudaEventDestroy(ev);
                if ((st = autotune(*d, c, items, n_items, seed, &lw))) return st;
                c.tuned[sig] = lw;
            } else {
                lw = 12;
            }
        }
        Plan p = make_plan(*d, items, n_items, seed, lw);
        if ((st = upload(c, p, c.capture_stream))) return st;
        // the graph is launched on the caller's stream: the descriptors must have landed
        cudaError_t ue = cudaStreamSynchronize(c.capture_stream);
        if (ue != cudaSuccess) return cuda_fail(ue, "upload");
        if (c.exec) {
            cudaGraphExecDestroy(c.exec);
            c.exec = nullptr;
        }
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(c.capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
        st = enqueue(*d, c, p, c.capture_stream, true, true);
        e = cudaStreamEndCapture(c.capture_stream, &g);
        if (st) return st;
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        c.sig = sig;
        c.weight = p.weight;
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    cudaError_t e = cudaGraphLaunch(c.exec, s);
    cudaEventRecord(b, s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaGraphLaunch");
    if (!st) st = wait_event(b, wait_limit_s());
    if (!st) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        for (int i = 0; i < n_items; ++i) {
            out_host[i].s1 = c.sums_host[i].x;
            out_host[i].s2 = c.sums_host[i].y;
            out_host[i].n = items[i].N;
            out_host[i].cost_ns = (double)ms * 1e6 * c.weight[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}
