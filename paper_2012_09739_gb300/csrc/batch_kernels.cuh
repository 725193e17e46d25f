// Persistent batched level kernel: many (parameter set, level) items of one
// estimator, working-precision variant and SDE scheme in one launch.
//
// Every item is cut into warp tiles (a contiguous range of sample pairs; one
// pair per lane per round) of one size per item: a span of consecutive tile
// indices.  The host orders the spans by tile length (longest first, or
// interleaved long and short); it never lists the tiles.  Each warp of a
// grid of resident blocks repeatedly takes the next tile index from an
// atomic counter, finds its span and simulates the tile with the same
// per-pair code as the level kernels.
//
// A tile covers whole chunk groups of the level kernel (32 pairs per chunk,
// chunk_group(l, chunks) chunks per group) and accumulates exactly as the
// level kernel does: per lane in FP32 with Kahan over a group's chunks, then
// a warp sum, one FP64 (sum D, sum D^2) per group.  The finalize kernel adds
// an item's group partials with the level finalize's fixed-order tree, so an
// item's sums equal those of the level entry points bit for bit, whatever
// the tile size.  No warp ever waits on another warp or block.
#pragma once

#include <type_traits>

#include "level_kernels.cuh"
#include "reduce.cuh"

namespace mlmc {

struct TileSpan {
    uint32_t item;       // index into the item array
    uint32_t per_tile;   // pairs per tile, a multiple of 32 * group (the item's last tile may be shorter)
    uint32_t begin;      // first tile index of the item (within its launch)
    uint32_t count;      // tiles of the item
    uint32_t part;       // the item's first group partial
    uint32_t group;      // chunks per group partial: chunk_group(l, chunks)
};

// Index of the span holding tile t: the largest k with spans[k].begin <= t
// (spans[0].begin = 0, begins strictly increasing).  Warp-cooperative: each
// pass tests 32 evenly spaced spans and keeps the last one that starts at or
// before t, shrinking the range 32-fold; the whole warp must call it.
__device__ __forceinline__ uint32_t find_span(const TileSpan *spans, uint32_t n, uint32_t t, uint32_t lane) {
    uint32_t lo = 0, hi = n;     // spans[lo].begin <= t, and t < spans[hi].begin unless hi = n
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) >> 5;
        const uint32_t k = lo + lane * step;
        const bool ok = k < hi && spans[k].begin <= t;
        const uint32_t m = __ballot_sync(0xffffffffu, ok);    // a prefix of the lanes; lane 0 always
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    return lo;
}

// Warp-cooperative simulation of one pair of samples (the deep levels of a
// batch hold items of one or two samples whose 2^l dependent steps would
// otherwise run on one lane).  Per block of 32 fine steps the lanes compute
// the Philox words and the normals of the 32 steps in parallel, then lane 0
// advances the paths through them with exactly the arithmetic of
// simulate_pair, so the results are identical.  Needs 2^l >= 32.
constexpr int SEQ_MIN_LEVEL = 10;

template <int P>
struct SeqScratch {
    uint32_t w[2][40];         // the block's uniforms' words of paths p0, p1 (five per call, or halves)
    Pair<P> zb[32];            // approximate normals of the 32 steps (both paths)
    Pair<P_F32> zh[32];        // exact normals (four-way)
};

template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__device__ void simulate_pair_seq(const LevelArgs &a, const PhiloxKeys &K, const SmemTable &tab, const float *mlp,
                                  uint64_t g, float &d0, float &d1, SeqScratch<P> &sc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nf = 1u << a.l;
    const uint64_t p0 = a.path_offset + 2 * g, p1 = p0 + 1;
    // 16-bit uniforms on a two-way path: two steps per word, 4 calls per
    // block; otherwise five uniforms per call, calls c0 .. c0 + 7 with
    // c0 = 32 blk / 5 cover the block's steps (its first step is uniform
    // 32 blk - 5 c0 of call c0)
    constexpr bool U16 = ICDF == ICDF_TABLE16 && MODE == MODE_TWO;
    constexpr uint32_t CALLS = U16 ? 4u : 8u;
    PathPair<P, KAHAN, SDE> fine, coarse;
    fine.template init<false>(a, false);
    coarse.template init<false>(a, true);
    PathPair<P_F32, true, SDE> hfine, hcoarse;
    if (MODE == MODE_FOUR) {
        hfine.template init<true>(a, false);
        hcoarse.template init<true>(a, true);
    }
    Pair<P> zprev;
    Pair<P_F32> zhprev;
    for (uint32_t blk = 0; blk < (nf >> 5); ++blk) {
        const uint32_t c0 = U16 ? blk * CALLS : (32u * blk) / 5u;
        if (lane < 2 * CALLS) {
            const uint64_t path = lane < CALLS ? p0 : p1;
            const uint32_t j = c0 + (lane % CALLS);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)path, (uint32_t)(path >> 32), j, a.tag), K);
            uint32_t *dst = &sc.w[lane < CALLS ? 0 : 1][(U16 ? 4u : 5u) * (lane % CALLS)];
            dst[0] = r.x;
            dst[1] = r.y;
            dst[2] = r.z;
            dst[3] = r.w;
            if (!U16) dst[4] = spare_word(r);
        }
        __syncwarp();
        if constexpr (U16) {
            const uint32_t w0 = sc.w[0][lane >> 1], w1 = sc.w[1][lane >> 1];
            const uint32_t f0 = (lane & 1) ? half16_bits<true>(w0) : half16_bits<false>(w0);
            const uint32_t f1 = (lane & 1) ? half16_bits<true>(w1) : half16_bits<false>(w1);
            sc.zb[lane] = table_pair<P, true>(tab, f0, f1, mirrored_v16(f0), mirrored_v16(f1));
        } else {
            const uint32_t k = 32u * blk + lane - 5u * c0;
            const uint32_t w0 = sc.w[0][k], w1 = sc.w[1][k];
            sc.zb[lane] = icdf_pair<P, ICDF>(tab, mlp, w0, w1);
            if (MODE == MODE_FOUR) sc.zh[lane] = Pair<P_F32>::of2(exact_z(tab, w0), exact_z(tab, w1));
        }
        __syncwarp();
        if (lane == 0) {
            for (int k = 0; k < 32; ++k) {
                const Pair<P> z = sc.zb[k];
                fine.step(z);
                if (k & 1) coarse.step(add(zprev, z));
                else zprev = z;
                if (MODE == MODE_FOUR) {
                    const Pair<P_F32> zh = sc.zh[k];
                    hfine.step(zh);
                    if (k & 1) hcoarse.step(add(zhprev, zh));
                    else zhprev = zh;
                }
            }
        }
        __syncwarp();
    }
    float out0[5], out1[5];
    pair_result<MODE>(a, fine, coarse, hfine, hcoarse, d0, d1, out0, out1);
}

// One warp tile t of span sp: its chunk groups (the last one of the item may
// be short), each accumulated and summed as the level kernel does, one FP64
// partial per group; a single deep pair warp-cooperatively.
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__device__ __forceinline__ void run_tile(const LevelArgs &a, const PhiloxKeys &keys, const SmemTable &tab,
                                         const float *mlp, const TileSpan &sp, uint32_t t, uint32_t lane,
                                         double2 *partials, SeqScratch<P> &seq) {
    const uint64_t first = (uint64_t)(t - sp.begin) * sp.per_tile;
    const uint32_t npairs = a.npairs - first < sp.per_tile ? (uint32_t)(a.npairs - first) : sp.per_tile;
    const uint64_t chunk0 = first >> 5;        // the tile's first chunk, the start of a group
    KahanF32 s1, s2;
    if (npairs == 1 && a.l >= SEQ_MIN_LEVEL) {
        // one pair, long paths: the warp generates the normals, lane 0 steps
        float d0, d1;
        simulate_pair_seq<MODE, P, KAHAN, ICDF, SDE>(a, keys, tab, mlp, first, d0, d1, seq);
        if (lane == 0) {
            s1.add(d0);
            s2.add(d0 * d0);
            if (2 * first + 1 < a.N) {
                s1.add(d1);
                s2.add(d1 * d1);
            }
            partials[sp.part + chunk0 / sp.group] = make_double2((double)s1.value(), (double)s2.value());
        }
        return;
    }
    const uint32_t rounds = (npairs + 31u) >> 5;
    uint32_t grp = sp.part + (uint32_t)chunk0 / sp.group;    // chunks < 2^31 (N < 2^37)
    for (uint32_t r = 0; r < rounds; ++grp) {
        const uint32_t r1 = r + sp.group < rounds ? r + sp.group : rounds;
        for (; r < r1; ++r) {
            const uint32_t k = (r << 5) + lane;
            const bool active = k < npairs;
            run_slot<MODE, P, KAHAN, ICDF, SDE>(a, keys, tab, mlp, first + (active ? k : npairs - 1), active, s1, s2);
        }
        const float w1 = warp_sum(s1.value()), w2 = warp_sum(s2.value());
        if (lane == 0) partials[grp] = make_double2((double)w1, (double)w2);
        s1 = KahanF32();
        s2 = KahanF32();
    }
}

// MODE_MIXED: one kernel for the two-way and four-way items of one variant
// (each tile dispatched on its item's mode), for latency-sized batches such
// as the rounds of an adaptive run at large RMSE, where one launch instead of
// two matters more than the four-way register budget the two-way tiles then
// run at.  Accumulation as in the single-mode kernels, so sums are the same.
enum { MODE_MIXED = 2 };

// MODE_CHOICE: a candidate round of the adaptive driver's per-level choice of
// working precision -- the two-way and four-way items of binary16 with and
// without Kahan and binary32 with one approximate inverse CDF, and the standard
// binary32 exact-normal two-way term -- in one launch, each tile dispatched
// on its item's variant (LevelArgs prec, kahan, icdf).  Accumulation as in
// the single-variant kernels, so the sums are the same.
enum { MODE_CHOICE = 3 };

// Scratch of the warp-cooperative single pairs for either working precision.
union ChoiceScratch {
    SeqScratch<P_F32> f32;
    SeqScratch<P_F16> f16;
};

template <int MODE, int P>
using TileScratch = std::conditional_t<MODE == MODE_CHOICE, ChoiceScratch, SeqScratch<P>>;

// The tile loop of a persistent batch kernel: each warp takes the next tile
// index from the counter until the tiles run out; or (STATIC) warp w of W
// first takes tile w and then W + the counter's next value, so that a
// launch of at most one tile per warp needs no atomic at all.  A tile's
// partials do not depend on which warp runs it.  The whole warp calls
// after(span) once each tile's partials are written.
template <bool STATIC, int MODE, int P, bool KAHAN, int ICDF, int SDE, class After>
__device__ __forceinline__ void tile_loop(const LevelArgs *items, const TileSpan *spans, uint32_t nspans,
                                          uint32_t ntiles, uint32_t *counter, double2 *partials,
                                          const SmemTable &tab, const PhiloxKeys &keys, TileScratch<MODE, P> &seq,
                                          After after) {
    const float *mlp = ICDF == ICDF_MLP ? items[0].mlp->ygrid : nullptr;
    const uint32_t lane = threadIdx.x & 31;
    auto tile = [&](uint32_t t) {
        const TileSpan sp = spans[find_span(spans, nspans, t, lane)];
        // every item has the batch's seed: its round keys come from the
        // launch parameters
        const LevelArgs a = items[sp.item];
        if constexpr (MODE == MODE_CHOICE) {
            auto either = [&](auto p, auto kahan, auto &sc) {
                constexpr int PP = decltype(p)::value;
                constexpr bool KK = decltype(kahan)::value;
                if (a.mode == MODE_FOUR)
                    run_tile<MODE_FOUR, PP, KK, ICDF, SDE>(a, keys, tab, mlp, sp, t, lane, partials, sc);
                else
                    run_tile<MODE_TWO, PP, KK, ICDF, SDE>(a, keys, tab, mlp, sp, t, lane, partials, sc);
            };
            if (a.icdf == ICDF_EXACT)
                run_tile<MODE_TWO, P_F32, true, ICDF_EXACT, SDE>(a, keys, tab, mlp, sp, t, lane, partials, seq.f32);
            else if (a.prec == P_F32)
                either(std::integral_constant<int, P_F32>(), std::false_type(), seq.f32);
            else if (a.kahan)
                either(std::integral_constant<int, P_F16>(), std::true_type(), seq.f16);
            else
                either(std::integral_constant<int, P_F16>(), std::false_type(), seq.f16);
        } else if constexpr (MODE == MODE_MIXED) {
            if (a.mode == MODE_FOUR)
                run_tile<MODE_FOUR, P, KAHAN, ICDF, SDE>(a, keys, tab, mlp, sp, t, lane, partials, seq);
            else
                run_tile<MODE_TWO, P, KAHAN, ICDF, SDE>(a, keys, tab, mlp, sp, t, lane, partials, seq);
        } else {
            run_tile<MODE, P, KAHAN, ICDF, SDE>(a, keys, tab, mlp, sp, t, lane, partials, seq);
        }
        after(sp);
    };
    if constexpr (STATIC) {
        uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        while (t < ntiles) {
            tile(t);
            const uint32_t warps = gridDim.x * (blockDim.x >> 5);
            if (warps >= ntiles) break;
            uint32_t k = 0;
            if (lane == 0) k = atomicAdd(counter, 1u);
            t = warps + __shfl_sync(0xffffffffu, k, 0);
        }
    } else {
        for (;;) {
            uint32_t t = 0;
            if (lane == 0) t = atomicAdd(counter, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= ntiles) break;
            tile(t);
        }
    }
}

// One kernel per (MODE, P, KAHAN, ICDF, SDE), like the level kernels and with
// their register budgets, so that a batch runs at the level kernels'
// occupancy; the host launches one per group of items that share them.
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__global__ void __launch_bounds__(256, MODE == MODE_TWO ? 4 : 3)
batch_kernel(const LevelArgs *items, const TileSpan *spans, uint32_t nspans, uint32_t ntiles, uint32_t *counter,
             double2 *partials, const DevTables *tabs, const PhiloxKeys keys) {
    __shared__ SmemTable tab;
    __shared__ SeqScratch<P> seq[8];           // one per warp (warp-cooperative single pairs)
    stage_table(tab, tabs);
    __syncthreads();
    tile_loop<false, MODE, P, KAHAN, ICDF, SDE>(items, spans, nspans, ntiles, counter, partials, tab, keys,
                                         seq[threadIdx.x >> 5], [](const TileSpan &) {});
}

// A latency-sized round of one group (an adaptive run's round at large
// RMSE): its descriptors travel in the kernel's parameter space, so the
// round needs no descriptor copy, and its sums are finalized inside the
// launch with the finalize's fixed-order sums (so they equal those of the
// two-kernel path bit for bit), written to `sums`.  A warp's first tile is
// its own index (no atomic).  Each item counts its finished tiles: the warp
// that finishes an item's last tile adds the item's partials (at most 1024:
// warp_sum_fixed, the same tree) while other warps still simulate, and
// zeroes the item's count; if an item has more partials, or the grid has
// fewer warps than tiles (tail), the last block to finish adds the partials
// of larger items with the whole block and zeroes the tile and block counts
// for the next round on the stream.  One launch per round instead of a
// copy and two launches.
//
// counters: [0] tiles taken, [1] blocks done, [2 + i] tiles done of item i.
constexpr int SMALL_ITEMS = 24;
constexpr int SMALL_COUNTERS = 2 + SMALL_ITEMS;

struct SmallRound {
    LevelArgs items[SMALL_ITEMS];
    TileSpan spans[SMALL_ITEMS];
    uint32_t first[SMALL_ITEMS];   // per item: its first group partial
    uint32_t count[SMALL_ITEMS];   // and how many (at most FINALIZE_SPAN)
    uint32_t nitems, nspans, ntiles;
    uint32_t tail;                 // 1: an item above 1024 partials, or more tiles than warps
    PhiloxKeys keys;
};

// atomicAdd with acquire-release semantics at GPU scope: the calling
// thread's earlier writes are visible to whoever acquires this location
// later, and whatever the earlier writers to it released is visible to the
// caller.  In place of __threadfence() (a sequentially consistent fence)
// and a relaxed atomicAdd: the release covers only the caller's own writes,
// which is all a count of one warp's tile needs.
__device__ __forceinline__ uint32_t atomic_add_acq_rel(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

// A latency-sized round fills a fraction of one wave, so the kernel takes a
// register budget of two blocks per SM instead of the occupancy the bulk
// kernels need.
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__global__ void __launch_bounds__(256, 2)
batch_small_kernel(const __grid_constant__ SmallRound r, uint32_t *counters, double2 *partials, double2 *sums,
                   const DevTables *tabs) {
    __shared__ SmemTable tab;
    __shared__ TileScratch<MODE, P> seq[8];
    __shared__ double r1[SUM_THREADS], r2[SUM_THREADS];
    __shared__ uint32_t last;
    stage_table(tab, tabs);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31;
    // lane 0 wrote the tile's partials and counts the tile with release
    // semantics; the count that completes the item also acquires the other
    // tiles' partials, and __syncwarp passes them on to the whole warp,
    // which reads them from L2 (warp_sum_fixed)
    auto item_done = [&](const TileSpan &sp) {
        uint32_t done = 0;
        if (lane == 0) {
            done = atomic_add_acq_rel(counters + 2 + sp.item, 1u) == sp.count - 1;
            if (done) counters[2 + sp.item] = 0u;
        }
        if (!__shfl_sync(0xffffffffu, done, 0) || r.count[sp.item] > (uint32_t)FINALIZE_THREADS) return;
        __syncwarp();
        const double2 v = warp_sum_fixed(partials + r.first[sp.item], r.count[sp.item], lane);
        if (lane == 0) sums[sp.item] = v;
    };
    tile_loop<true, MODE, P, KAHAN, ICDF, SDE>(r.items, r.spans, r.nspans, r.ntiles, counters, partials, tab, r.keys,
                                         seq[threadIdx.x >> 5], item_done);
    // without larger items or a shared tile counter to reset, the items'
    // warps have finished the round
    if (!r.tail) return;
    // the block's partials were released by its warps (item_done) before
    // this barrier; thread 0's count releases them again for the last block
    __syncthreads();
    if (threadIdx.x == 0) last = atomic_add_acq_rel(counters + 1, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    for (uint32_t i = 0; i < r.nitems; ++i) {
        if (r.count[i] <= (uint32_t)FINALIZE_THREADS) continue;
        const double2 v = block_sum_fixed(partials + r.first[i], r.count[i], r1, r2);
        if (threadIdx.x == 0) sums[i] = v;
    }
    if (threadIdx.x == 0) {
        counters[0] = 0u;
        counters[1] = 0u;
    }
}

using BatchSmallFn = void (*)(SmallRound, uint32_t *, double2 *, double2 *, const DevTables *);

using BatchKernelFn = void (*)(const LevelArgs *, const TileSpan *, uint32_t, uint32_t, uint32_t *, double2 *,
                               const DevTables *, const PhiloxKeys);

}  // namespace mlmc
