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

template <int P, bool KAHAN, int ICDF>
__global__ void __launch_bounds__(256) batch_kernel(const LevelArgs *items, const Tile *tiles, uint32_t ntiles,
                                                    uint32_t *counter, double2 *tile_partials,
                                                    const DevTables *tabs) {
    __shared__ SmemTable tab;
    if (ICDF == ICDF_TABLE || ICDF == ICDF_TABLE16 || ICDF == ICDF_CUBIC) {
        stage_table(tab, tabs);
        __syncthreads();
    }
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
