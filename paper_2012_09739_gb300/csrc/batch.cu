// Host side of mlmc_batch: warp tiles in longest-first (or interleaved)
// order (one span of tiles per item, never listed one by one); one
// persistent launch per group of items sharing estimator, working-precision
// variant and SDE scheme, the groups running concurrently; a finalize
// kernel; CUDA graphs of recent item-list shapes, replayed; and an autotuner
// for the tile size, block shape and span order.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "api_internal.h"
#include "batch_kernels.cuh"
#include "reduce.cuh"

namespace mlmc {

BatchKernelFn batch_kernel_f32_two(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_f16_two(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_bf16_two(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_f32_four(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_f16_four(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_bf16_four(int kahan, int icdf, int sde);
BatchKernelFn batch_kernel_mixed(int prec, int kahan, int icdf, int sde);
BatchSmallFn batch_small_mixed(int prec, int kahan, int icdf, int sde);
BatchSmallFn batch_small_two(int prec, int kahan, int icdf, int sde);
BatchSmallFn batch_small_choice(int icdf, int sde);

// The batch finalize adds an item's group partials exactly as the level
// finalize does (block_sum_fixed over at most FINALIZE_SPAN partials, or one
// per span and one over the span sums): one block per item or span, all of
// them in parallel.

// First pass, items of more than FINALIZE_SPAN partials: job j = (first
// partial, count, scratch slot) writes one span's sum.
__global__ void __launch_bounds__(SUM_THREADS) batch_span_kernel(double2 *partials, const uint32_t *jobs) {
    __shared__ double r1[SUM_THREADS], r2[SUM_THREADS];
    const uint32_t j = blockIdx.x;
    const double2 s = block_sum_fixed(partials + jobs[3 * j], jobs[3 * j + 1], r1, r2);
    if (threadIdx.x == 0) partials[jobs[3 * j + 2]] = s;
}

// Each item's sums: over its group partials (fin[3i] .. + fin[3i+1]) when
// they fit one span, else over its span sums (from fin[3i+2]).
__global__ void __launch_bounds__(SUM_THREADS) batch_finalize_kernel(const double2 *partials, const uint32_t *fin,
                                                                     double2 *sums) {
    __shared__ double r1[SUM_THREADS], r2[SUM_THREADS];
    const uint32_t w = blockIdx.x;
    const uint64_t first = fin[3 * w], count = fin[3 * w + 1], scratch = fin[3 * w + 2];
    const double2 s =
        count <= FINALIZE_SPAN
            ? block_sum_fixed(partials + first, count, r1, r2)
            : block_sum_fixed(partials + scratch, (count + FINALIZE_SPAN - 1) / FINALIZE_SPAN, r1, r2);
    if (threadIdx.x == 0) sums[w] = s;
}

namespace {

int env_int(const char *name, int dflt);

// Work (pair-cost units: fine-step equivalents of a two-way pair) below
// which a batch is latency-sized: about 50 us on GB300.
constexpr double SMALL_BATCH_WORK = 2e7;

struct Group {
    int mode, prec, kahan, icdf, sde;
    std::vector<TileSpan> spans;   // in the plan's span order (ORDER_*)
    std::vector<double> tile_cost;  // per span: cost of one full tile
    uint32_t span_base = 0;        // offset of this group's spans in the device array
    uint32_t ntiles = 0;
    double work = 0.0;
};

struct Plan {
    std::vector<LevelArgs> items;
    std::vector<Group> groups;
    std::vector<uint32_t> fin;           // per item: first group partial, partials, finalize scratch
    std::vector<uint32_t> jobs;          // span jobs of the finalize's first pass: first, count, scratch slot
    std::vector<double> weight;          // share of the launch's work per item
    uint32_t nspans = 0;
    uint64_t npartials = 0;              // group partials and finalize scratch, all items
    double work = 0.0;
    bool too_large = false;              // tiles or partials beyond 32-bit indices
    int block = 256;                     // threads per block of the batch kernels (256 or 128)
};

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char *c = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    return h;
}

// Cost of one sample pair on one lane in fine-step units: 2^l steps plus the
// per-sample work (counter set-up, payoffs, accumulation), which at level 0
// is about three steps' worth; a four-way pair costs about 2.2 two-way pairs.
constexpr double PAIR_OVERHEAD_STEPS = 3.0;
double pair_cost(int l, int four) { return (ldexp(1.0, l) + PAIR_OVERHEAD_STEPS) * (four ? 2.2 : 1.0); }

double item_work(const mlmc_work &w) { return (double)((w.N + 1) / 2) * pair_cost(w.l, w.kind); }

// Span orders: by the cost of their tiles, longest first; or interleaved
// from both ends of that order (longest, shortest, second longest, ...), so
// that warps taking consecutive tiles mix long and short ones.
enum { ORDER_LONGEST_FIRST = 0, ORDER_INTERLEAVED = 1 };

// Tiles: a lane takes max(1, 2^lane_work_log2 / (2^l + overhead)) pairs of an
// item at level l, rounded up to whole chunk groups of the level kernel; a
// tile is 32 such lanes.  Every item is one span of consecutive tiles; each
// group's spans are ordered by the cost of their tiles (ORDER_*), so the
// host work is per item, not per tile.  Each item owns one partial per chunk
// group and, above FINALIZE_SPAN of them, scratch for the finalize's span sums.
Plan make_plan(const DeviceState &d, const mlmc_work *w, int n, uint64_t seed, int lane_work_log2,
               int block = 256, int span_order = ORDER_LONGEST_FIRST, bool choice = false) {
    Plan plan;
    plan.block = block;
    plan.items.resize(n);
    plan.fin.assign(3 * (size_t)n, 0);
    for (int i = 0; i < n; ++i) plan.work += item_work(w[i]);
    for (int i = 0; i < n; ++i) {
        plan.items[i] = make_level_args(d, w[i].kind, w[i].l, w[i].N, w[i].prec, w[i].icdf, &w[i].params, seed,
                                        w[i].path_offset, (uint32_t)w[i].set_id);
        plan.items[i].kahan = w[i].kahan ? 1 : 0;
    }
    // a latency-sized batch puts both estimators' items of one variant into
    // one launch where a mixed kernel exists (MLMC_BATCH_MIXED=0 disables it)
    const bool mixed = plan.work < SMALL_BATCH_WORK && env_int("MLMC_BATCH_MIXED", 1) != 0;
    // and (choice: an adaptive round) the items of several variants, or of
    // one without a mixed kernel, where all are candidates of the per-level
    // choice (binary16 with or without Kahan, or binary32, with one
    // approximate inverse CDF; or the standard binary32 exact-normal two-way
    // term), into one launch of the fused choice kernel
    int choice_icdf = -1;
    bool use_choice = choice && mixed && n <= SMALL_ITEMS && env_int("MLMC_ROUND_FUSED", 1) != 0;
    bool several = false;
    const int choice_sde = n > 0 ? plan.items[0].sde : SDE_GBM;
    for (int i = 0; i < n && use_choice; ++i) {
        const mlmc_work &x = w[i];
        if (plan.items[i].sde != choice_sde) {
            use_choice = false;
        } else if (x.icdf == MLMC_ICDF_EXACT) {
            use_choice = x.kind == 0 && x.prec == MLMC_F32 && x.kahan;
        } else if (choice_icdf >= 0 && x.icdf != choice_icdf) {
            use_choice = false;
        } else {
            choice_icdf = x.icdf;
            use_choice = x.prec == MLMC_F16 || (x.prec == MLMC_F32 && !x.kahan);
        }
        several |= x.prec != w[0].prec || (x.kahan != 0) != (w[0].kahan != 0) || x.icdf != w[0].icdf;
    }
    // (one variant: where no mixed kernel takes both estimators' items)
    if (use_choice && !several) use_choice = !batch_kernel_mixed(w[0].prec, w[0].kahan ? 1 : 0, w[0].icdf, choice_sde);
    use_choice = use_choice && choice_icdf >= 0 && batch_small_choice(choice_icdf, choice_sde) != nullptr;
    for (int i = 0; i < n; ++i) {
        plan.weight.push_back(plan.work > 0 ? item_work(w[i]) / plan.work : 0.0);
        int kahan = w[i].kahan ? 1 : 0, sde = plan.items[i].sde, prec = w[i].prec, icdf = w[i].icdf;
        int mode = mixed && batch_kernel_mixed(prec, kahan, icdf, sde) ? (int)MODE_MIXED : w[i].kind;
        if (use_choice) {
            mode = MODE_CHOICE;
            prec = kahan = -1;
            icdf = choice_icdf;
        }
        size_t gi = 0;
        while (gi < plan.groups.size()) {
            const Group &g = plan.groups[gi];
            if (g.mode == mode && g.prec == prec && g.kahan == kahan && g.icdf == icdf && g.sde == sde) break;
            ++gi;
        }
        if (gi == plan.groups.size()) plan.groups.push_back(Group{mode, prec, kahan, icdf, sde});
        Group &g = plan.groups[gi];
        // lane slots: pairs, or units of pairs at the coarsest two-way levels
        const uint64_t np = plan.items[i].npairs, nchunks = (np + 31) / 32;
        const uint32_t G = chunk_group(w[i].l, nchunks);
        const uint64_t ngroups = (nchunks + G - 1) / G;
        const double pc = pair_cost(w[i].l, w[i].kind) * plan.items[i].unit;
        uint64_t per_lane = std::max<uint64_t>(1, (uint64_t)(ldexp(1.0, lane_work_log2) / (pc / (w[i].kind ? 2.2 : 1.0))));
        per_lane = (per_lane + G - 1) / G * G;
        const uint64_t per_tile = 32 * per_lane;
        const uint64_t count = (np + per_tile - 1) / per_tile;
        const uint64_t rounds = (std::min(per_tile, np) + 31) / 32;
        plan.fin[3 * i] = (uint32_t)plan.npartials;
        plan.fin[3 * i + 1] = (uint32_t)ngroups;
        g.spans.push_back(TileSpan{(uint32_t)i, (uint32_t)per_tile, 0, (uint32_t)count, (uint32_t)plan.npartials, G});
        plan.npartials += ngroups;
        if (plan.npartials > 0xFFFFFFFFull || count > 0xFFFFFFFFull) plan.too_large = true;
        g.tile_cost.push_back((double)rounds * pc);
        g.work += item_work(w[i]);
    }
    for (int i = 0; i < n; ++i) {          // finalize scratch and span jobs for items above one span
        const uint64_t first = plan.fin[3 * i], cnt = plan.fin[3 * i + 1];
        plan.fin[3 * i + 2] = (uint32_t)plan.npartials;
        if (cnt <= FINALIZE_SPAN) continue;
        for (uint64_t lo = 0; lo < cnt; lo += FINALIZE_SPAN) {
            plan.jobs.push_back((uint32_t)(first + lo));
            plan.jobs.push_back((uint32_t)std::min<uint64_t>(FINALIZE_SPAN, cnt - lo));
            plan.jobs.push_back((uint32_t)plan.npartials++);
        }
    }
    if (plan.npartials > 0xFFFFFFFFull) plan.too_large = true;
    uint32_t span_base = 0;
    for (auto &g : plan.groups) {
        std::vector<uint32_t> order(g.spans.size());
        for (uint32_t k = 0; k < order.size(); ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return g.tile_cost[a] > g.tile_cost[b]; });
        if (span_order == ORDER_INTERLEAVED) {
            std::vector<uint32_t> both_ends;
            for (size_t lo = 0, hi = order.size(); lo < hi;) {
                both_ends.push_back(order[lo++]);
                if (lo < hi) both_ends.push_back(order[--hi]);
            }
            order.swap(both_ends);
        }
        std::vector<TileSpan> spans;
        std::vector<double> cost;
        uint64_t begin = 0;
        for (uint32_t k : order) {
            TileSpan sp = g.spans[k];
            sp.begin = (uint32_t)begin;
            begin += sp.count;
            spans.push_back(sp);
            cost.push_back(g.tile_cost[k]);
        }
        g.spans.swap(spans);
        g.tile_cost.swap(cost);
        g.ntiles = (uint32_t)begin;
        g.span_base = span_base;
        span_base += (uint32_t)g.spans.size();
        if (begin > 0xFFFFFFFFull) plan.too_large = true;
    }
    plan.nspans = span_base;
    // the choice kernel runs only as one fused launch (small_round)
    if (use_choice && (!plan.jobs.empty() || plan.too_large || block != SUM_THREADS))
        return make_plan(d, w, n, seed, lane_work_log2, block, span_order, false);
    return plan;
}

BatchKernelFn pick_batch_kernel(const Group &g) {
    if (g.mode == MODE_CHOICE) return nullptr;      // fused launches only
    if (g.mode == MODE_MIXED) return batch_kernel_mixed(g.prec, g.kahan, g.icdf, g.sde);
    if (g.mode == MODE_TWO)
        return g.prec == MLMC_F32   ? batch_kernel_f32_two(g.kahan, g.icdf, g.sde)
               : g.prec == MLMC_F16 ? batch_kernel_f16_two(g.kahan, g.icdf, g.sde)
                                    : batch_kernel_bf16_two(g.kahan, g.icdf, g.sde);
    return g.prec == MLMC_F32   ? batch_kernel_f32_four(g.kahan, g.icdf, g.sde)
           : g.prec == MLMC_F16 ? batch_kernel_f16_four(g.kahan, g.icdf, g.sde)
                                : batch_kernel_bf16_four(g.kahan, g.icdf, g.sde);
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

struct ShapeKey {
    int32_t l, kind, prec, kahan, icdf, sde, scheme, zero;
    uint64_t N;
};
// compared with memcmp: neither may hold padding bytes
static_assert(sizeof(ShapeKey) == 40, "ShapeKey has no padding");
static_assert(sizeof(mlmc_work) == sizeof(mlmc_sde_params) + 6 * 4 + 2 * 8 && sizeof(mlmc_sde_params) == 72,
              "mlmc_work has no padding");

struct BatchCache {
    // descriptors, uploaded by one copy: items, tile spans, per-item partial
    // ranges, the finalize's span jobs and the schedule counters (zeroed by
    // the same copy), each 16-byte aligned
    unsigned char *blob = nullptr;
    size_t blob_cap = 0;
    LevelArgs *items = nullptr;
    TileSpan *spans = nullptr;
    uint32_t *fin = nullptr;             // per item: first partial, partials, finalize scratch
    uint32_t *jobs = nullptr;            // the finalize's span jobs
    uint32_t *counters = nullptr;
    double2 *partials = nullptr;
    size_t partials_cap = 0;
    double2 *sums = nullptr;
    size_t sums_cap = 0;
    double2 *sums_host = nullptr;
    size_t sums_host_cap = 0;
    unsigned char *stage = nullptr;      // pinned staging of the descriptors
    size_t stage_cap = 0;
    std::map<std::pair<const void *, int>, int> occupancy;   // (batch kernel, block) -> resident blocks per SM
    uint32_t *small_counters = nullptr;  // the fused small-round kernel's counters (zero between rounds)
    // streams of the concurrent groups (created on first use)
    static constexpr size_t MAX_SIDE = 7;
    cudaStream_t side[MAX_SIDE] = {};
    cudaEvent_t fork = nullptr, join[MAX_SIDE] = {};
    // mlmc_batch graph entry: the captured graph of one item-list shape
    cudaGraphExec_t exec = nullptr;
    std::vector<ShapeKey> shape;         // the item-list shape the graph was captured for
    uint64_t graph_seed = 0;             // and the seed: the two-way kernels take its key as launch parameters
    std::vector<mlmc_work> staged_items; // the items the device descriptors hold
    uint64_t last_use = 0;
    size_t items_bytes = 0;      // the LevelArgs part of the descriptors
    cudaEvent_t done = nullptr;  // after the entry's last launch and sums copy
    cudaEvent_t staged = nullptr;    // after the last descriptor copy out of `stage`
    bool launched = false, restaged = false;
    std::vector<double> weight;
};

// A plan's shape: tile size (log2 of the fine-step equivalents per lane and
// tile), block threads and span order (ORDER_*).
struct Tuning {
    int lw, block, order;
};

// The graph entries of mlmc_batch / mlmc_batch_async on one device.
struct BatchGraphs {
    std::vector<BatchCache *> entries;   // at most MAX_ENTRIES, least recently used evicted
    cudaStream_t capture_stream = nullptr;
    std::map<uint64_t, Tuning> tuned;   // hash of the item-list shape -> its tuned plan shape
    uint64_t clock = 0;
    static constexpr size_t MAX_ENTRIES = 8;
};

BatchCache *batch_cache_create() { return new BatchCache(); }

void batch_cache_destroy(BatchCache *c) {
    if (!c) return;
    if (c->done) cudaEventSynchronize(c->done);
    if (c->exec) cudaGraphExecDestroy(c->exec);
    cudaFree(c->blob);
    cudaFree(c->small_counters);
    cudaFree(c->partials);
    cudaFree(c->sums);
    if (c->sums_host) cudaFreeHost(c->sums_host);
    if (c->stage) cudaFreeHost(c->stage);
    if (c->done) cudaEventDestroy(c->done);
    if (c->staged) cudaEventDestroy(c->staged);
    for (size_t k = 0; k < BatchCache::MAX_SIDE; ++k) {
        if (c->side[k]) cudaStreamSynchronize(c->side[k]);
        if (c->side[k]) cudaStreamDestroy(c->side[k]);
        if (c->join[k]) cudaEventDestroy(c->join[k]);
    }
    if (c->fork) cudaEventDestroy(c->fork);
    delete c;
}

void release_device_extras(DeviceState &d) {
    if (d.batch) {
        for (BatchCache *c : d.batch->entries) batch_cache_destroy(c);
        if (d.batch->capture_stream) cudaStreamDestroy(d.batch->capture_stream);
        delete d.batch;
    }
    batch_cache_destroy(d.run_cache);
    if (d.run_stream) cudaStreamDestroy(d.run_stream);
    for (cudaEvent_t &ev : d.run_events) {
        if (ev) cudaEventDestroy(ev);
        ev = nullptr;
    }
    d.batch = nullptr;
    d.run_cache = nullptr;
    d.run_stream = nullptr;
}

namespace {

// Uploads the plan into the cache's device buffers: the descriptors and the
// zeroed schedule counters are packed into pinned staging memory and copied
// to the device in one asynchronous copy on s (the buffers only grow, with
// cudaMalloc, when a larger batch arrives).
// stage_idle: the caller knows that no copy out of the staging buffer is
// still in flight (it waited for the previous round), so no stream sync.
mlmc_status upload(BatchCache &c, const Plan &p, cudaStream_t s, bool stage_idle = false) {
    cudaError_t e;
    const size_t n = p.items.size();
    if (p.too_large) return fail(MLMC_EINVAL, "batch needs more than 2^32 - 1 tiles or partials");
    if ((e = grow(&c.partials, &c.partials_cap, p.npartials)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if ((e = grow(&c.sums, &c.sums_cap, n)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if (c.sums_host_cap < n) {
        if (c.sums_host) cudaFreeHost(c.sums_host);
        c.sums_host = nullptr;
        c.sums_host_cap = 0;
        if ((e = cudaMallocHost(&c.sums_host, n * sizeof(double2))) != cudaSuccess) return cuda_fail(e, "pinned");
        c.sums_host_cap = n;
    }
    auto up16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t b_items = n * sizeof(LevelArgs), b_spans = (size_t)p.nspans * sizeof(TileSpan);
    const size_t b_fin = p.fin.size() * 4, b_jobs = p.jobs.size() * 4, b_cnt = p.groups.size() * 4;
    const size_t o_spans = up16(b_items), o_fin = o_spans + up16(b_spans), o_jobs = o_fin + up16(b_fin);
    const size_t o_cnt = o_jobs + up16(b_jobs), total = o_cnt + up16(b_cnt);
    if ((e = grow(&c.blob, &c.blob_cap, total)) != cudaSuccess) return cuda_fail(e, "batch buffers");
    if (c.stage_cap < total) {
        if (c.stage) cudaFreeHost(c.stage);
        c.stage = nullptr;
        c.stage_cap = 0;
        if ((e = cudaMallocHost(&c.stage, total * 2)) != cudaSuccess) return cuda_fail(e, "pinned");
        c.stage_cap = total * 2;
    }
    // the previous round's copy out of the staging buffer must be done
    if (!stage_idle && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "upload");
    c.items = reinterpret_cast<LevelArgs *>(c.blob);
    c.spans = reinterpret_cast<TileSpan *>(c.blob + o_spans);
    c.fin = reinterpret_cast<uint32_t *>(c.blob + o_fin);
    c.jobs = reinterpret_cast<uint32_t *>(c.blob + o_jobs);
    c.counters = reinterpret_cast<uint32_t *>(c.blob + o_cnt);
    unsigned char *h = c.stage;
    memset(h, 0, total);
    memcpy(h, p.items.data(), b_items);
    for (const auto &g : p.groups)
        memcpy(h + o_spans + g.span_base * sizeof(TileSpan), g.spans.data(), g.spans.size() * sizeof(TileSpan));
    memcpy(h + o_fin, p.fin.data(), b_fin);
    if (b_jobs) memcpy(h + o_jobs, p.jobs.data(), b_jobs);
    if ((e = cudaMemcpyAsync(c.blob, h, total, cudaMemcpyHostToDevice, s)) != cudaSuccess) return cuda_fail(e, "upload");
    return MLMC_OK;
}

// Resident blocks per SM of a batch kernel at a block size (cached).
template <class Fn>
int blocks_per_sm(BatchCache &c, Fn fn, int block) {
    const auto key = std::make_pair((const void *)fn, block);
    auto it = c.occupancy.find(key);
    if (it != c.occupancy.end()) return it->second;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, 0) != cudaSuccess || bps < 1) bps = 1;
    c.occupancy[key] = bps;
    return bps;
}

// Enqueues the whole batch on stream s (also used inside graph capture).
// Groups run concurrently: the first on s, the others on side streams forked
// from s and joined back before the finalize.  A lone group gets every
// resident block; with several, each gets a share of the GPU proportional to
// its work, but at least one warp for each of its tiles that is longer than
// the whole batch's ideal time per warp (their tiles are the critical path).
// zero_counters: reset the schedule counters on the stream (a replayed graph
// needs it; a fresh upload has zeroed them already).
mlmc_status enqueue(const DeviceState &d, BatchCache &c, const Plan &p, cudaStream_t s, bool copy_out,
                    bool zero_counters) {
    cudaError_t e;
    const size_t ng = p.groups.size();
    if (zero_counters && (e = cudaMemsetAsync(c.counters, 0, ng * sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "memset");
    std::vector<BatchKernelFn> fns(ng);
    std::vector<int> bps(ng);
    int bps_min = 1 << 20;
    for (size_t gi = 0; gi < ng; ++gi) {
        if (!(fns[gi] = pick_batch_kernel(p.groups[gi]))) return fail(MLMC_EINVAL, "no batch kernel for this variant");
        bps[gi] = blocks_per_sm(c, fns[gi], p.block);
        bps_min = std::min(bps_min, bps[gi]);
    }
    // Groups one after another on s, each with the whole GPU, unless the
    // batch is latency-sized (below about 50 us of work: the second launch
    // would wait for the first) or the groups' longest tiles dominate.  In
    // per-lane step units, a group alone takes about max(ideal, tail) (its
    // work spread over all resident lanes, or its longest tile); in sequence
    // the groups add up, concurrently they share the GPU, at about 1.2 times
    // the ideal sum (measured), and overlap their tails.  On GB300 adaptive
    // rounds of 0.5-15 ms ran 10-30 % faster in sequence (RMSE 3e-6, a
    // 15.4 ms concurrent round took 11.9 ms), the batching workload's
    // single-pair deep items twice as fast concurrently.
    // MLMC_BATCH_CONCURRENT = 0 / 1 forces either.
    double seq = 0.0, ideal_sum = 0.0, tail_max = 0.0;
    for (size_t gi = 0; gi < ng; ++gi) {
        const Group &g = p.groups[gi];
        const double ideal_g = g.work / ((double)bps[gi] * d.sm_count * p.block);
        const double tail_g = g.tile_cost.empty() ? 0.0 : *std::max_element(g.tile_cost.begin(), g.tile_cost.end());
        seq += std::max(ideal_g, tail_g);
        ideal_sum += ideal_g;
        tail_max = std::max(tail_max, tail_g);
    }
    const int conc_env = env_int("MLMC_BATCH_CONCURRENT", -1);
    const bool concurrent =
        ng > 1 && (conc_env == 1 || (conc_env != 0 && (p.work < SMALL_BATCH_WORK ||
                                                        1.2 * std::max(ideal_sum, tail_max) < seq)));
    const size_t nside = concurrent ? std::min<size_t>(ng - 1, BatchCache::MAX_SIDE) : 0;
    if (nside > 0) {
        if (!c.fork && (e = cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate");
        for (size_t k = 0; k < nside; ++k) {
            if (!c.side[k] && (e = cudaStreamCreateWithFlags(&c.side[k], cudaStreamNonBlocking)) != cudaSuccess)
                return cuda_fail(e, "cudaStreamCreate");
            if (!c.join[k] && (e = cudaEventCreateWithFlags(&c.join[k], cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "cudaEventCreate");
        }
        if ((e = cudaEventRecord(c.fork, s)) != cudaSuccess) return cuda_fail(e, "fork");
        for (size_t k = 0; k < nside; ++k)
            if ((e = cudaStreamWaitEvent(c.side[k], c.fork, 0)) != cudaSuccess) return cuda_fail(e, "fork");
    }
    const int wpb = p.block / 32;
    const double ideal = p.work / ((double)bps_min * d.sm_count * wpb);
    for (size_t gi = 0; gi < ng; ++gi) {
        const Group &g = p.groups[gi];
        const uint64_t full = (uint64_t)bps[gi] * d.sm_count;
        uint64_t grid = full;
        if (concurrent) {
            uint64_t long_tiles = 0;
            for (size_t k = 0; k < g.spans.size(); ++k)
                if (g.tile_cost[k] > ideal) long_tiles += g.spans[k].count;
            const uint64_t share = (uint64_t)ceil(g.work / p.work * (double)full);
            grid = std::min(full, std::max(share, (long_tiles + wpb - 1) / wpb));
        }
        grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, ((uint64_t)g.ntiles + wpb - 1) / wpb));
        cudaStream_t gs = gi == 0 || !concurrent ? s : c.side[(gi - 1) % BatchCache::MAX_SIDE];
        fns[gi]<<<(unsigned)grid, p.block, 0, gs>>>(c.items, c.spans + g.span_base, (uint32_t)g.spans.size(), g.ntiles,
                                                 c.counters + gi, c.partials, d.tabs, p.items[0].rk);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch kernel");
    }
    for (size_t k = 0; k < nside; ++k) {
        if ((e = cudaEventRecord(c.join[k], c.side[k])) != cudaSuccess) return cuda_fail(e, "join");
        if ((e = cudaStreamWaitEvent(s, c.join[k], 0)) != cudaSuccess) return cuda_fail(e, "join");
    }
    const int n = (int)p.items.size();
    // copy_out: the finalize kernel writes the sums straight into the pinned
    // host buffer (device-accessible under unified addressing), no copy
    double2 *dst = copy_out ? c.sums_host : c.sums;
    const uint32_t njobs = (uint32_t)(p.jobs.size() / 3);
    if (njobs) {
        batch_span_kernel<<<njobs, SUM_THREADS, 0, s>>>(c.partials, c.jobs);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch finalize");
    }
    batch_finalize_kernel<<<n, SUM_THREADS, 0, s>>>(c.partials, c.fin, dst);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "batch finalize");
    return MLMC_OK;
}

int env_int(const char *name, int dflt) {
    const char *s = getenv(name);
    return s ? atoi(s) : dflt;
}

// Tile size (log2 of the fine-step equivalents per lane and tile) for a
// batch's total work: about four tiles per resident lane, clamped to [4, 12].
int work_lane_log2(const DeviceState &d, const mlmc_work *w, int n) {
    double steps = 0.0;
    for (int i = 0; i < n; ++i) steps += (double)((w[i].N + 1) / 2) * pair_cost(w[i].l, 0);
    const double lanes = (double)d.sm_count * 24 * 32;
    const int lw = (int)floor(log2(std::max(steps / (4.0 * lanes), 1.0)));
    return std::min(12, std::max(4, lw));
}

// Tunes a batch shape on the real batch: tile size (log2 of the fine-step
// equivalents per lane and tile, five candidates around the work-based size
// of about four tiles per resident lane) x block shape (256 threads, or
// 128 -- more, smaller blocks per SM at the same register budget) with the
// spans longest first, then the best of those with the spans interleaved.
// Each candidate runs three times after the plan is uploaded; the median
// device time decides (ties to the earlier candidate).  MLMC_TUNE_LOG=1
// prints every candidate's times and the choice on stderr.
mlmc_status autotune(const DeviceState &d, BatchCache &c, const mlmc_work *w, int n, uint64_t seed, cudaStream_t s,
                     Tuning *best) {
    const int base = work_lane_log2(d, w, n);
    const int lws[] = {base - 3, base - 2, base - 1, base, base + 1};
    const int blocks[] = {256, 128};
    const bool log = env_int("MLMC_TUNE_LOG", 0) > 0;
    float best_ms = 1e30f;
    *best = Tuning{base, 256, ORDER_LONGEST_FIRST};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    auto trial = [&](const Tuning &tu) -> mlmc_status {
        Plan p = make_plan(d, w, n, seed, tu.lw, tu.block, tu.order);
        mlmc_status st = upload(c, p, s);
        if (st) return st;
        float t[3];
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a, s);
            if ((st = enqueue(d, c, p, s, false, true))) return st;
            cudaEventRecord(b, s);
            if ((st = wait_event(b, wait_limit_s()))) return st;
            cudaEventElapsedTime(&t[rep], a, b);
        }
        std::sort(t, t + 3);
        if (log)
            fprintf(stderr, "{\"mlmc_tune\": {\"items\": %d, \"lane_work_log2\": %d, \"block\": %d, "
                            "\"order\": %d, \"ms\": [%.4f, %.4f, %.4f]}}\n", n, tu.lw, tu.block, tu.order, t[0], t[1],
                    t[2]);
        if (t[1] < best_ms) {
            best_ms = t[1];
            *best = tu;
        }
        return MLMC_OK;
    };
    mlmc_status st = MLMC_OK;
    for (int block : blocks)
        for (int lw : lws)
            if (!st) st = trial(Tuning{lw, block, ORDER_LONGEST_FIRST});
    if (!st) st = trial(Tuning{best->lw, best->block, ORDER_INTERLEAVED});
    if (log && !st)
        fprintf(stderr, "{\"mlmc_tune_choice\": {\"items\": %d, \"lane_work_log2\": %d, \"block\": %d, "
                        "\"order\": %d, \"median_ms\": %.4f}}\n", n, best->lw, best->block, best->order, best_ms);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

}  // namespace

// A latency-sized round of one group in one launch of the fused small-round
// kernel (descriptors as a kernel parameter, finalized in the launch, sums
// straight into the pinned host buffer); false (nothing enqueued) where the
// round does not qualify: several groups, more than SMALL_ITEMS items, an
// item above one finalize span, not latency-sized, or no such kernel for the
// variant.  MLMC_ROUND_FUSED=0 turns it off.
bool small_round(const DeviceState &d, BatchCache &c, const Plan &p, cudaStream_t s, mlmc_status *st) {
    if (p.groups.size() != 1 || p.items.size() > (size_t)SMALL_ITEMS || !p.jobs.empty() || p.too_large ||
        p.block != SUM_THREADS || p.work >= SMALL_BATCH_WORK || env_int("MLMC_ROUND_FUSED", 1) == 0)
        return false;
    const Group &g = p.groups[0];
    const BatchSmallFn fn = g.mode == MODE_CHOICE ? batch_small_choice(g.icdf, g.sde)
                            : g.mode == MODE_MIXED ? batch_small_mixed(g.prec, g.kahan, g.icdf, g.sde)
                            : g.mode == MODE_TWO ? batch_small_two(g.prec, g.kahan, g.icdf, g.sde)
                                                 : nullptr;
    if (!fn) return false;
    cudaError_t e;
    *st = MLMC_OK;
    if (!c.small_counters) {
        if ((e = cudaMalloc(&c.small_counters, SMALL_COUNTERS * sizeof(uint32_t))) != cudaSuccess ||
            (e = cudaMemsetAsync(c.small_counters, 0, SMALL_COUNTERS * sizeof(uint32_t), s)) != cudaSuccess) {
            *st = cuda_fail(e, "batch buffers");
            return true;
        }
    }
    if ((e = grow(&c.partials, &c.partials_cap, p.npartials)) != cudaSuccess) {
        *st = cuda_fail(e, "batch buffers");
        return true;
    }
    const size_t n = p.items.size();
    if (c.sums_host_cap < n) {
        if (c.sums_host) cudaFreeHost(c.sums_host);
        c.sums_host = nullptr;
        c.sums_host_cap = 0;
        if ((e = cudaMallocHost(&c.sums_host, SMALL_ITEMS * sizeof(double2))) != cudaSuccess) {
            *st = cuda_fail(e, "pinned");
            return true;
        }
        c.sums_host_cap = SMALL_ITEMS;
    }
    SmallRound r;
    memset(&r, 0, sizeof r);
    for (size_t i = 0; i < n; ++i) {
        r.items[i] = p.items[i];
        r.first[i] = p.fin[3 * i];
        r.count[i] = p.fin[3 * i + 1];
    }
    for (size_t k = 0; k < g.spans.size(); ++k) r.spans[k] = g.spans[k];
    r.nitems = (uint32_t)n;
    r.nspans = (uint32_t)g.spans.size();
    r.ntiles = g.ntiles;
    r.keys = p.items[0].rk;
    const int wpb = SUM_THREADS / 32;
    const uint64_t full = (uint64_t)blocks_per_sm(c, fn, SUM_THREADS) * d.sm_count;
    const uint64_t grid = std::max<uint64_t>(1, std::min<uint64_t>(full, ((uint64_t)g.ntiles + wpb - 1) / wpb));
    r.tail = grid * wpb < (uint64_t)g.ntiles;
    for (size_t i = 0; i < n; ++i) r.tail |= r.count[i] > (uint32_t)FINALIZE_THREADS;
    fn<<<(unsigned)grid, SUM_THREADS, 0, s>>>(r, c.small_counters, c.partials, c.sums_host, d.tabs);
    if ((e = cudaGetLastError()) != cudaSuccess) *st = cuda_fail(e, "batch small-round kernel");
    return true;
}

// One round of a caller that owns its own cache (the adaptive driver):
// descriptors, persistent kernels, finalize and the copy of all sums into
// c.sums_host, enqueued on s.  The caller waits on s before reading.
// The tile size follows the round's total work: about sixteen tiles per
// resident lane (every round has a new shape, so nothing is tuned), each at
// least 4 steps long per lane; the dynamic schedule then leaves a last wave
// of at most a sixteenth of a group's time.  A latency-sized round, which
// fills a fraction of the GPU, gets the shortest tiles (a pair or two per
// lane): its time is its longest tile's.
mlmc_status batch_round(const DeviceState &d, BatchCache &c, const mlmc_work *w, int n, uint64_t seed,
                        cudaStream_t s) {
    Plan p = make_plan(d, w, n, seed, std::max(2, work_lane_log2(d, w, n) - 2), SUM_THREADS, ORDER_LONGEST_FIRST,
                       true);
    mlmc_status st = MLMC_OK;
    if (small_round(d, c, p, s, &st)) return st;
    // the driver waits for every round before it plans the next one
    st = upload(c, p, s, true);
    if (st) return st;
    return enqueue(d, c, p, s, true, false);
}

const double2 *batch_sums_host(const BatchCache &c) { return c.sums_host; }

namespace {

mlmc_status check_items(const mlmc_work *items, int n_items) {
    if (!items || n_items <= 0) return fail(MLMC_EINVAL, "bad batch arguments");
    for (int i = 0; i < n_items; ++i) {
        const mlmc_work &w = items[i];
        if (w.kind != 0 && w.kind != 1) return fail(MLMC_EINVAL, "item %d: kind must be 0 or 1", i);
        if (w.set_id < 0 || w.set_id > 0xFFFF) return fail(MLMC_EINVAL, "item %d: set_id outside 0..65535", i);
        if (w.N > 0xFFFFFFFFull * 32) return fail(MLMC_EINVAL, "item %d: N too large for a batch", i);
        mlmc_status st = check_level(w.kind, w.l, w.N, w.prec, w.icdf, &w.params);
        if (st) return fail(st, "item %d: %s", i, mlmc_last_error());
    }
    return MLMC_OK;
}

// What the tiles, the kernel groups and so the captured graph of an item
// depend on: level, estimator, variant, SDE type and scheme, N.  Parameter
// values, payoffs, set ids, path offsets and the seed only change the
// LevelArgs, which are re-staged.
std::vector<ShapeKey> shape_of(const mlmc_work *items, int n) {
    std::vector<ShapeKey> k((size_t)n);
    for (int i = 0; i < n; ++i) {
        const mlmc_work &w = items[i];
        k[i] = ShapeKey{w.l, w.kind, w.prec, w.kahan, w.icdf, (int32_t)w.params.sde, (int32_t)w.params.scheme, 0, w.N};
    }
    return k;
}

std::mutex g_batch_mu;   // one enqueue at a time per process: the entries are shared

// Builds a graph entry: tile size (tuned once per shape), plan, descriptor
// upload and the captured graph (batch kernels and finalize into c.sums).
mlmc_status build_entry(DeviceState &d, BatchGraphs &G, BatchCache &c, const mlmc_work *items, int n_items,
                        uint64_t seed, std::vector<ShapeKey> &&shape, cudaStream_t s) {
    const uint64_t shape_hash = fnv1a(shape.data(), shape.size() * sizeof(ShapeKey));
    cudaError_t e;
    mlmc_status st;
    if ((e = cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&c.staged, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    // the capture stream must see the caller's prior work first
    cudaEvent_t ev;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e, "event");
    cudaEventRecord(ev, s);
    cudaStreamWaitEvent(G.capture_stream, ev, 0);
    cudaEventDestroy(ev);
    // MLMC_BATCH_LANE_WORK_LOG2 (6..20) forces the tile size, with 256-thread
    // blocks and MLMC_BATCH_ORDER's span order (default longest first)
    Tuning tu{env_int("MLMC_BATCH_LANE_WORK_LOG2", 0), 256,
              env_int("MLMC_BATCH_ORDER", 0) == ORDER_INTERLEAVED ? ORDER_INTERLEAVED : ORDER_LONGEST_FIRST};
    if (tu.lw < 6 || tu.lw > 20) {
        auto it = G.tuned.find(shape_hash);
        if (it != G.tuned.end()) {
            tu = it->second;
        } else if (env_int("MLMC_AUTOTUNE", 1)) {
            if ((st = autotune(d, c, items, n_items, seed, G.capture_stream, &tu))) return st;
            G.tuned[shape_hash] = tu;
        } else {
            tu = Tuning{12, 256, ORDER_LONGEST_FIRST};
        }
    }
    Plan p = make_plan(d, items, n_items, seed, tu.lw, tu.block, tu.order);
    if ((st = upload(c, p, G.capture_stream))) return st;
    // the graph is launched on the caller's stream: the descriptors must have landed
    if ((e = cudaStreamSynchronize(G.capture_stream)) != cudaSuccess) return cuda_fail(e, "upload");
    cudaGraph_t g;
    if ((e = cudaStreamBeginCapture(G.capture_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamBeginCapture");
    st = enqueue(d, c, p, G.capture_stream, false, true);
    e = cudaStreamEndCapture(G.capture_stream, &g);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c.exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    c.shape = std::move(shape);
    c.graph_seed = seed;
    c.staged_items.assign(items, items + n_items);
    c.items_bytes = p.items.size() * sizeof(LevelArgs);
    c.weight = p.weight;
    return MLMC_OK;
}

// Finds or builds the graph entry of this item-list shape and seed and
// enqueues one replay on s: waits (on s) for the entry's previous launch,
// re-stages the descriptors if the items changed since then (parameter
// values, payoffs, set ids, path offsets), launches the graph and copies the
// item sums to dst (device or pinned host memory; NULL: the entry's pinned
// host buffer), then records the entry's done event.  t0/t1 (optional)
// bracket the graph.
mlmc_status batch_enqueue(DeviceState &d, const mlmc_work *items, int n_items, uint64_t seed, void *dst,
                          cudaStream_t s, cudaEvent_t t0, cudaEvent_t t1, BatchCache **used) {
    cudaError_t e;
    mlmc_status st;
    if (!d.batch) {
        d.batch = new BatchGraphs();
        if ((e = cudaStreamCreateWithFlags(&d.batch->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "cudaStreamCreate");
    }
    BatchGraphs &G = *d.batch;
    std::vector<ShapeKey> shape = shape_of(items, n_items);
    BatchCache *c = nullptr;
    for (BatchCache *x : G.entries)
        if (x->graph_seed == seed && x->shape.size() == shape.size() &&
            memcmp(x->shape.data(), shape.data(), shape.size() * sizeof(ShapeKey)) == 0)
            c = x;
    if (!c) {
        if (G.entries.size() >= BatchGraphs::MAX_ENTRIES) {
            auto lru = std::min_element(G.entries.begin(), G.entries.end(),
                                        [](const BatchCache *x, const BatchCache *y) { return x->last_use < y->last_use; });
            // its last launch must be done with the buffers (bounded wait)
            if ((*lru)->launched && (st = wait_event((*lru)->done, wait_limit_s()))) return st;
            batch_cache_destroy(*lru);
            G.entries.erase(lru);
        }
        c = new BatchCache();
        if ((st = build_entry(d, G, *c, items, n_items, seed, std::move(shape), s))) {
            batch_cache_destroy(c);
            return st;
        }
        G.entries.push_back(c);
    }
    c->last_use = ++G.clock;
    // the previous launch of this entry (on any stream) must be done with
    // the descriptors, the partials and the sums before they are reused
    if (c->launched && (e = cudaStreamWaitEvent(s, c->done, 0)) != cudaSuccess) return cuda_fail(e, "wait");
    if (memcmp(c->staged_items.data(), items, (size_t)n_items * sizeof(mlmc_work)) != 0) {
        // same shape and seed, new parameters, payoffs, set ids or offsets: only the LevelArgs change
        if (c->restaged && (st = wait_event(c->staged, wait_limit_s()))) return st;
        LevelArgs *h = reinterpret_cast<LevelArgs *>(c->stage);
        for (int i = 0; i < n_items; ++i)
            h[i] = make_level_args(d, items[i].kind, items[i].l, items[i].N, items[i].prec, items[i].icdf,
                                   &items[i].params, seed, items[i].path_offset, (uint32_t)items[i].set_id);
        if ((e = cudaMemcpyAsync(c->items, h, c->items_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "descriptor upload");
        cudaEventRecord(c->staged, s);
        c->restaged = true;
        c->staged_items.assign(items, items + n_items);
    }
    if (t0) cudaEventRecord(t0, s);
    if ((e = cudaGraphLaunch(c->exec, s)) != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    if (t1) cudaEventRecord(t1, s);
    void *out = dst ? dst : (void *)c->sums_host;
    if ((e = cudaMemcpyAsync(out, c->sums, (size_t)n_items * sizeof(double2), cudaMemcpyDefault, s)) != cudaSuccess)
        return cuda_fail(e, "sums copy");
    if ((e = cudaEventRecord(c->done, s)) != cudaSuccess) return cuda_fail(e, "event");
    c->launched = true;
    if (used) *used = c;
    return MLMC_OK;
}

}  // namespace

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_batch(const mlmc_work *items, int n_items, uint64_t seed, mlmc_sums *out_host,
                                  void *stream) {
    mlmc_status st = check_items(items, n_items);
    if (st) return st;
    if (!out_host) return fail(MLMC_EINVAL, "out_host is NULL");
    DeviceState *d;
    if ((st = device_state(&d))) return st;
    for (int i = 0; i < n_items; ++i)
        if (items[i].icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    // held to the end: the entry's pinned sums are read after the wait
    std::lock_guard<std::mutex> lock(g_batch_mu);
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        if (a) cudaEventDestroy(a);
        return fail(MLMC_ECUDA, "cudaEventCreate");
    }
    BatchCache *c = nullptr;
    st = batch_enqueue(*d, items, n_items, seed, nullptr, s, a, b, &c);
    if (!st) st = wait_event(c->done, wait_limit_s());
    if (!st) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        for (int i = 0; i < n_items; ++i) {
            out_host[i].s1 = c->sums_host[i].x;
            out_host[i].s2 = c->sums_host[i].y;
            out_host[i].n = items[i].N;
            out_host[i].cost_ns = (double)ms * 1e6 * c->weight[i];
            level_moments(out_host[i].s1, out_host[i].s2, items[i].N, &out_host[i].mean, &out_host[i].var);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

extern "C" mlmc_status mlmc_batch_async(const mlmc_work *items, int n_items, uint64_t seed, double *sums_dev,
                                        void *stream) {
    mlmc_status st = check_items(items, n_items);
    if (st) return st;
    if (!sums_dev) return fail(MLMC_EINVAL, "sums_dev is NULL");
    DeviceState *d;
    if ((st = device_state(&d))) return st;
    for (int i = 0; i < n_items; ++i)
        if (items[i].icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");
    std::lock_guard<std::mutex> lock(g_batch_mu);
    return batch_enqueue(*d, items, n_items, seed, sums_dev, (cudaStream_t)stream, nullptr, nullptr, nullptr);
}

extern "C" size_t mlmc_batch_descriptor_bytes(void) { return sizeof(LevelArgs); }
