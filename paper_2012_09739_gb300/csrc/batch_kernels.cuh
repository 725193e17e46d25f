// Persistent batched level kernel: many (parameter set, level, estimator)
// items of one working-precision variant in one launch.
//
// The host cuts every item into warp tiles (a contiguous range of sample
// pairs; one pair per lane per round) and orders all tiles longest first.
// Each warp of a grid of resident blocks repeatedly takes the next tile from
// an atomic counter, simulates it with the same per-pair code as the level
// kernels, and writes the tile's (sum D, sum D^2) to its own slot; a finalize
// kernel then sums each item's slots in a fixed order.  No warp ever waits on
// another warp or block.
#pragma once

#include "level_kernels.cuh"

namespace mlmc {

struct Tile {
    uint32_t item;     // index into the item array
    uint32_t npairs;   // pairs in this tile
    uint64_t first;    // first pair index within the item
};

// Warp-cooperative simulation of one pair of samples (the deep levels of a
// batch hold items of one or two samples whose 2^l dependent steps would
// otherwise run on one lane).  Per block of 32 fine steps the lanes compute
// the Philox words and the normals of the 32 steps in parallel, then lane 0
// advances the paths through them with exactly the arithmetic of
// simulate_pair, so the results are identical.  Needs 2^l >= 32.
constexpr int SEQ_MIN_LEVEL = 10;

template <int P>
struct SeqScratch {
    uint32_t w[2][32];         // the block's Philox words of paths p0, p1
    Pair<P> zb[32];            // approximate normals of the 32 steps (both paths)
    Pair<P_F32> zh[32];        // exact normals (four-way)
};

template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__device__ void simulate_pair_seq(const LevelArgs &a, const SmemTable &tab, const MlpFrags &mlp, uint64_t g,
                                  float &d0, float &d1, SeqScratch<P> &sc) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nf = 1u << a.l;
    const uint64_t p0 = a.path_offset + 2 * g, p1 = p0 + 1;
    // 16-bit uniforms on a two-way path: two steps per word, 4 calls per block
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
        if (lane < 2 * CALLS) {
            const uint64_t path = lane < CALLS ? p0 : p1;
            const uint32_t j = blk * CALLS + (lane % CALLS);
            const uint4 r = philox4x32_10(make_uint4((uint32_t)path, (uint32_t)(path >> 32), j, a.tag), a.k0, a.k1);
            uint32_t *dst = &sc.w[lane < CALLS ? 0 : 1][4 * (lane % CALLS)];
            dst[0] = r.x;
            dst[1] = r.y;
            dst[2] = r.z;
            dst[3] = r.w;
        }
        __syncwarp();
        if constexpr (U16) {
            const uint32_t w0 = sc.w[0][lane >> 1], w1 = sc.w[1][lane >> 1];
            const uint32_t f0 = (lane & 1) ? half16_bits<true>(w0) : half16_bits<false>(w0);
            const uint32_t f1 = (lane & 1) ? half16_bits<true>(w1) : half16_bits<false>(w1);
            sc.zb[lane] = table_pair<P, true>(tab, f0, f1, mirrored_v16(f0), mirrored_v16(f1));
        } else {
            const uint32_t w0 = sc.w[0][lane], w1 = sc.w[1][lane];
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

template <int P, bool KAHAN, int ICDF>
__global__ void __launch_bounds__(256) batch_kernel(const LevelArgs *items, const Tile *tiles, uint32_t ntiles,
                                                    uint32_t *counter, double2 *tile_partials,
                                                    const DevTables *tabs) {
    __shared__ SmemTable tab;
    __shared__ SeqScratch<P> seq[8];           // one per warp (warp-cooperative single pairs)
    stage_table(tab, tabs);
    __syncthreads();
    MlpFrags mlp;
    if (ICDF == ICDF_MLP) mlp.load(items[0].mlp);
    const uint32_t lane = threadIdx.x & 31;
    for (;;) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(counter, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= ntiles) break;
        const Tile tl = tiles[t];
        const LevelArgs a = items[tl.item];
        KahanF32 s1, s2;
        if (tl.npairs == 1 && a.l >= SEQ_MIN_LEVEL) {
            // one pair, long paths: the warp generates the normals, lane 0 steps
            SeqScratch<P> &sc = seq[threadIdx.x >> 5];
            float d0, d1;
            if (a.mode == MODE_TWO) {
                if (a.sde == SDE_GBM) simulate_pair_seq<MODE_TWO, P, KAHAN, ICDF, SDE_GBM>(a, tab, mlp, tl.first, d0, d1, sc);
                else if (a.sde == SDE_OU) simulate_pair_seq<MODE_TWO, P, KAHAN, ICDF, SDE_OU>(a, tab, mlp, tl.first, d0, d1, sc);
                else simulate_pair_seq<MODE_TWO, P, KAHAN, ICDF, SDE_GBM_MIL>(a, tab, mlp, tl.first, d0, d1, sc);
            } else {
                if (a.sde == SDE_GBM) simulate_pair_seq<MODE_FOUR, P, KAHAN, ICDF, SDE_GBM>(a, tab, mlp, tl.first, d0, d1, sc);
                else if (a.sde == SDE_OU) simulate_pair_seq<MODE_FOUR, P, KAHAN, ICDF, SDE_OU>(a, tab, mlp, tl.first, d0, d1, sc);
                else simulate_pair_seq<MODE_FOUR, P, KAHAN, ICDF, SDE_GBM_MIL>(a, tab, mlp, tl.first, d0, d1, sc);
            }
            if (lane == 0) {
                s1.add(d0);
                s2.add(d0 * d0);
                if (2 * tl.first + 1 < a.N) {
                    s1.add(d1);
                    s2.add(d1 * d1);
                }
                tile_partials[t] = make_double2((double)s1.value(), (double)s2.value());
            }
            continue;
        }
        const uint32_t rounds = (tl.npairs + 31u) >> 5;
        for (uint32_t r = 0; r < rounds; ++r) {
            const uint32_t k = (r << 5) + lane;
            const bool active = k < tl.npairs;
            const uint64_t g = tl.first + (active ? k : tl.npairs - 1);
            float d0, d1, o0[5], o1[5];
            if (a.mode == MODE_TWO) {
                if (a.sde == SDE_GBM) simulate_pair<MODE_TWO, P, KAHAN, ICDF, SDE_GBM>(a, tab, mlp, g, d0, d1, o0, o1);
                else if (a.sde == SDE_OU) simulate_pair<MODE_TWO, P, KAHAN, ICDF, SDE_OU>(a, tab, mlp, g, d0, d1, o0, o1);
                else simulate_pair<MODE_TWO, P, KAHAN, ICDF, SDE_GBM_MIL>(a, tab, mlp, g, d0, d1, o0, o1);
            } else {
                if (a.sde == SDE_GBM) simulate_pair<MODE_FOUR, P, KAHAN, ICDF, SDE_GBM>(a, tab, mlp, g, d0, d1, o0, o1);
                else if (a.sde == SDE_OU) simulate_pair<MODE_FOUR, P, KAHAN, ICDF, SDE_OU>(a, tab, mlp, g, d0, d1, o0, o1);
                else simulate_pair<MODE_FOUR, P, KAHAN, ICDF, SDE_GBM_MIL>(a, tab, mlp, g, d0, d1, o0, o1);
            }
            if (!active) continue;
            s1.add(d0);
            s2.add(d0 * d0);
            if (2 * g + 1 < a.N) {
                s1.add(d1);
                s2.add(d1 * d1);
            }
        }
        const float w1 = warp_sum(s1.value()), w2 = warp_sum(s2.value());
        if (lane == 0) tile_partials[t] = make_double2((double)w1, (double)w2);
    }
}

using BatchKernelFn = void (*)(const LevelArgs *, const Tile *, uint32_t, uint32_t *, double2 *,
                               const DevTables *);

}  // namespace mlmc
