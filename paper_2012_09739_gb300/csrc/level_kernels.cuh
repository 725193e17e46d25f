// Level kernels: two-way and four-way MLMC differences (Sec. 3).
//
// One thread carries a pair of samples (paths 2g and 2g+1 of the level), so
// that binary16 arithmetic runs packed as f16x2.  Path state lives in
// registers for all 2^l fine steps; the piecewise-linear table sits in
// shared memory; per-thread sums are reduced with warp shuffles in FP32,
// across warps in FP64, and one FP64 (sum D, sum D^2) pair per block goes
// to global memory for the finalize kernel.
//
// Every warp runs the same number of pair iterations (lanes past the end
// simulate a clamped pair and discard it), so warp-cooperative steps such as
// the MLP's tensor-core evaluation see all 32 lanes.
#pragma once

#include "device.cuh"
#include "mlp_device.cuh"

namespace mlmc {

enum { MODE_TWO = 0, MODE_FOUR = 1 };
enum { SDE_GBM = 0, SDE_OU = 1, SDE_GBM_MIL = 2 };   // GBM with Milstein
enum { PAYOFF_X = 0, PAYOFF_CALL = 1 };
enum { CI_DRIFT_F = 0, CI_DRIFT_C = 1, CI_DIFF = 2, CI_MEAN = 3, CI_X0 = 4, CI_MIL = 5, CI_ONE = 6, CI_TWO = 7 };

struct LevelArgs {
    int l;                    // level: 2^l fine steps
    int payoff;
    int mode, sde;            // MODE_*, SDE_* (read by the batched kernel)
    int prec, kahan, icdf;    // working precision (P_*), Kahan flag, ICDF_* (read by the choice kernel)
    uint64_t npairs;          // lane slots: ceil(N / 2) pairs, or ceil(N / (2 unit)) units
    int unit;                 // pairs per slot: 1, or 2 / 4 at the coarsest levels (unit_pairs)
    uint64_t N;
    uint64_t path_offset;
    uint32_t tag, k0, k1;     // Philox counter tag and key (seed)
    PhiloxKeys rk;            // the key's ten round keys (level launches read them from here)
    // per-level coefficients in FP64, rounded once to the working precision
    // in the kernel: GBM drift = mu delta_f (fine) / mu 2 delta_f (coarse),
    // diff = sigma sqrt(delta_f), Milstein mil = sigma^2 delta_f / 2; OU
    // drift = theta delta, diff = s sqrt(delta_f), mean = m.
    double drift_f, drift_c, diff, mean, x0, mil;
    double K, disc;
    // The same coefficients rounded once, on the host, to nearest even from
    // FP64: cw in the approximate paths' working precision as pair bits
    // (binary32: the value's bits; binary16 / bfloat16: the value in both
    // halves), c32 in binary32 for the exact-normal paths.  Index: CI_*.
    uint32_t cw[8];
    float c32[8];
    float K32, disc32;
    const DevTables *tabs;    // piecewise-linear and cubic tables
    const MlpWeights *mlp;    // network (ICDF_MLP only)
    double2 *partials;        // (sum D, sum D^2) per warp chunk, or per block
    int chunk_partials;       // 1: one partial per chunk of 32 pairs (result independent of the grid)
    unsigned long long *counter;  // chunk counter of the persistent schedule (chunk_partials)
    float *paths_out;         // optional per-sample output (3 or 5 floats per sample)
};

template <int P, bool KAHAN, int SDE>
struct PathPair {
    Pair<P> X, c, drift, diff, mean, mil, mconst;

    // Constants from the launch arguments, already rounded on the host (no
    // FP64 conversion per sample): HAT selects the binary32 copies of the
    // exact-normal paths; mconst is 1 on a fine path, 2 on a coarse one.
    template <bool HAT>
    __device__ __forceinline__ void init(const LevelArgs &a, bool coarse_path) {
        auto k = [&](int i) {
            if constexpr (HAT) return Pair<P>::bits(__float_as_uint(a.c32[i]));
            else return Pair<P>::bits(a.cw[i]);
        };
        drift = k(coarse_path ? CI_DRIFT_C : CI_DRIFT_F);
        diff = k(CI_DIFF);
        mean = k(CI_MEAN);
        X = k(CI_X0);
        c = Pair<P>::of2(0.0f, 0.0f);
        if (SDE == SDE_GBM_MIL) {
            mil = k(CI_MIL);
            mconst = k(coarse_path ? CI_TWO : CI_ONE);
        }
    }
    // X <- X (+) (A (+) B): A = a delta, B = (b sqrt(delta)) (x) z  (Sec. 2.2);
    // Milstein (GBM): X <- X (+) ((A (+) B) (+) M), M = (mil (x) X) (x)
    // ((z (x) z) (-) mconst); with Kahan compensation of the outer addition
    // (Sec. 2.3, Algorithm 1).
    __device__ __forceinline__ void step(Pair<P> z) {
        Pair<P> A, B;
        if (SDE == SDE_GBM || SDE == SDE_GBM_MIL) {
            A = mul(drift, X);
            B = mul(mul(diff, X), z);
        } else {
            A = mul(drift, sub(mean, X));
            B = mul(diff, z);
        }
        Pair<P> inc = add(A, B);
        if (SDE == SDE_GBM_MIL) inc = add(inc, mul(mul(mil, X), sub(mul(z, z), mconst)));
        if (KAHAN) {
            const Pair<P> y = sub(inc, c);
            const Pair<P> t = add(X, y);
            c = sub(sub(t, X), y);
            X = t;
        } else {
            X = add(X, inc);
        }
    }
};

// Table normals of two samples from their mirrored uniforms v0, v1 and the
// words carrying their signs (bit 31, or bit 15 with SIGN15).
template <int P, bool SIGN15>
__device__ __forceinline__ Pair<P> table_pair(const SmemTable &s, uint32_t w0, uint32_t w1, float v0, float v1) {
    if constexpr (P == P_F32) {
        return Pair<P>::of2(table_z32<false, SIGN15>(s, w0, v0), table_z32<false, SIGN15>(s, w1, v1));
    } else if constexpr (P == P_F16) {
        return Pair<P>{table_z16<false, SIGN15>(s, w0, w1, v0, v1)};
    } else {
        return Pair<P>{table_zbf16<false, SIGN15>(s, w0, w1, v0, v1)};
    }
}

// Approximate (or exact) normals of two samples from their Philox words.
// TABLE16 (four-way bar paths): the table at the centre of the 2^-16 cell
// that holds each word's 24-bit uniform, i.e. at the 16-bit uniform of the
// word's top half (u24 = (2 (w >> 9) + 1) 2^-24 lies in cell w >> 16).
template <int P, int ICDF>
__device__ __forceinline__ Pair<P> icdf_pair(const SmemTable &s, const float *mlp, uint32_t w0, uint32_t w1) {
    if constexpr (ICDF == ICDF_EXACT) {
        return Pair<P>::of2(exact_z(s, w0), exact_z(s, w1));
    } else if constexpr (ICDF == ICDF_TABLE) {
        return table_pair<P, false>(s, w0, w1, mirrored_v(w0), mirrored_v(w1));
    } else if constexpr (ICDF == ICDF_CUBIC) {
        const float v0 = mirrored_v(w0), v1 = mirrored_v(w1);
        if constexpr (P == P_F32) {
            return Pair<P>::of2(cubic_z32<false>(s, w0, v0), cubic_z32<false>(s, w1, v1));
        } else if constexpr (P == P_F16) {
            return Pair<P>{cubic_z16<false>(s, w0, w1, v0, v1)};
        } else {
            return Pair<P>{cubic_zbf16<false>(s, w0, w1, v0, v1)};
        }
    } else if constexpr (ICDF == ICDF_TABLE16) {
        const uint32_t f0 = half16_bits<true>(w0), f1 = half16_bits<true>(w1);
        return table_pair<P, true>(s, f0, f1, mirrored_v16(f0), mirrored_v16(f1));
    } else {
        // the network on the 24-bit grid, tabulated (mlp = MlpWeights::ygrid)
        return Pair<P>::of2(mlp_grid_z(mlp, w0), mlp_grid_z(mlp, w1));
    }
}

// Payoff in binary32: X, or disc (x) max(X (-) K, 0).
__device__ __forceinline__ float payoff_of(float X, int payoff, float K, float disc) {
    if (payoff == PAYOFF_X) return X;
    const float t = __fsub_rn(X, K);
    return __fmul_rn(disc, t > 0.0f ? t : 0.0f);
}

// Payoffs and differences of a simulated pair: D = P_f - P_c (two-way) or
// (P^_f - P^_c) - (P-_f - P-_c) (four-way), in binary32; out0/out1 receive
// the per-sample outputs (P_f, P_c, D) or (P^_f, P^_c, P-_f, P-_c, D).
template <int MODE, class PP, class HP>
__device__ __forceinline__ void pair_result(const LevelArgs &a, const PP &fine, const PP &coarse, const HP &hfine,
                                            const HP &hcoarse, float &d0, float &d1, float *out0, float *out1) {
    const float K = a.K32, disc = a.disc32;
    const float2 xf = fine.X.f32(), xc = coarse.X.f32();
    if (MODE == MODE_TWO) {
        const float pf0 = payoff_of(xf.x, a.payoff, K, disc), pf1 = payoff_of(xf.y, a.payoff, K, disc);
        float pc0 = 0.0f, pc1 = 0.0f;
        if (a.l > 0) {
            pc0 = payoff_of(xc.x, a.payoff, K, disc);
            pc1 = payoff_of(xc.y, a.payoff, K, disc);
            d0 = __fsub_rn(pf0, pc0);
            d1 = __fsub_rn(pf1, pc1);
        } else {
            d0 = pf0;
            d1 = pf1;
        }
        out0[0] = pf0; out0[1] = pc0; out0[2] = d0;
        out1[0] = pf1; out1[1] = pc1; out1[2] = d1;
    } else {
        const float2 hf = hfine.X.f32(), hc = hcoarse.X.f32();
        const float phf0 = payoff_of(hf.x, a.payoff, K, disc), phf1 = payoff_of(hf.y, a.payoff, K, disc);
        const float pbf0 = payoff_of(xf.x, a.payoff, K, disc), pbf1 = payoff_of(xf.y, a.payoff, K, disc);
        float phc0 = 0.0f, phc1 = 0.0f, pbc0 = 0.0f, pbc1 = 0.0f;
        if (a.l > 0) {
            phc0 = payoff_of(hc.x, a.payoff, K, disc);
            phc1 = payoff_of(hc.y, a.payoff, K, disc);
            pbc0 = payoff_of(xc.x, a.payoff, K, disc);
            pbc1 = payoff_of(xc.y, a.payoff, K, disc);
        }
        d0 = __fsub_rn(__fsub_rn(phf0, phc0), __fsub_rn(pbf0, pbc0));
        d1 = __fsub_rn(__fsub_rn(phf1, phc1), __fsub_rn(pbf1, pbc1));
        out0[0] = phf0; out0[1] = phc0; out0[2] = pbf0; out0[3] = pbc0; out0[4] = d0;
        out1[0] = phf1; out1[1] = phc1; out1[2] = pbf1; out1[3] = pbc1; out1[4] = d1;
    }
}

// Simulates samples 2g and 2g+1 of the level described by `a` and returns
// their differences D (d0, d1); out0/out1 receive the per-sample outputs
// (P_f, P_c, D) or (P^_f, P^_c, P-_f, P-_c, D).
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__device__ __forceinline__ void simulate_pair(const LevelArgs &a, const PhiloxKeys &K, const SmemTable &tab,
                                              const float *mlp, uint64_t g, float &d0, float &d1, float *out0,
                                              float *out1) {
    const uint32_t nf = 1u << a.l;
    const uint64_t p0 = a.path_offset + 2 * g, p1 = p0 + 1;
    PathPair<P, KAHAN, SDE> fine, coarse;
    fine.template init<false>(a, false);
    coarse.template init<false>(a, true);
    PathPair<P_F32, true, SDE> hfine, hcoarse;       // exact-normal pair (four-way only)
    if (MODE == MODE_FOUR) {
        hfine.template init<true>(a, false);
        hcoarse.template init<true>(a, true);
    }
    Pair<P> zprev;
    Pair<P_F32> zhprev;

    auto body = [&](uint32_t w0, uint32_t w1, int q) {
        const Pair<P> z = icdf_pair<P, ICDF>(tab, mlp, w0, w1);
        fine.step(z);
        if (q & 1) coarse.step(add(zprev, z));
        else zprev = z;
        if (MODE == MODE_FOUR) {
            const Pair<P_F32> zh = Pair<P_F32>::of2(exact_z(tab, w0), exact_z(tab, w1));
            hfine.step(zh);
            if (q & 1) hcoarse.step(add(zhprev, zh));
            else zhprev = zh;
        }
    };

    auto call_of = [&](uint64_t cp, uint32_t j) {
        return philox4x32_10(make_uint4((uint32_t)cp, (uint32_t)(cp >> 32), j, a.tag), K);
    };
    // Coarsest levels (a path needs at most half a call; level 1, and level
    // 2 with 16-bit uniforms -- level 0 runs in lane slots of several pairs,
    // run_slot): paths 2k and 2k+1 share call 0 of counter path field k,
    // path p starting at word (or half) (p mod 2) 2^l.  p0 = path_offset + 2g
    // has the launch's parity, so whether the pair's two paths share one call
    // is uniform.
    const uint64_t c0 = p0 >> 1, c1 = p1 >> 1;
    const uint32_t o0 = (uint32_t)(p0 & 1) << a.l, o1 = (uint32_t)(p1 & 1) << a.l;

    if constexpr (ICDF == ICDF_TABLE16 && MODE == MODE_TWO) {
        // two 16-bit uniforms per word: fine step n takes half n mod 2 (low
        // half first) of word (n / 2) mod 4 of call n / 8
        auto body16 = [&](uint32_t f0, uint32_t f1, int q) {
            const Pair<P> z = table_pair<P, true>(tab, f0, f1, mirrored_v16(f0), mirrored_v16(f1));
            fine.step(z);
            if (q & 1) coarse.step(add(zprev, z));
            else zprev = z;
        };
        auto halves = [&](uint32_t x0, uint32_t x1, int q) {
            body16(half16_bits<false>(x0), half16_bits<false>(x1), q);
            body16(half16_bits<true>(x0), half16_bits<true>(x1), q + 1);
        };
        auto half_of = [](const uint4 &r, uint32_t h) {
            const uint32_t w = word(r, (int)(h >> 1));
            return (h & 1) ? half16_bits<true>(w) : half16_bits<false>(w);
        };
        if (nf <= 4) {
            const uint4 ra = call_of(c0, 0);
            const uint4 rb = c1 == c0 ? ra : call_of(c1, 0);
            for (uint32_t n = 0; n < nf; ++n) body16(half_of(ra, o0 + n), half_of(rb, o1 + n), (int)n);
        }
        const uint32_t ncalls16 = nf <= 4 ? 0u : (nf + 7u) >> 3;
        for (uint32_t j = 0; j < ncalls16; ++j) {
            const uint4 r0 = philox4x32_10(make_uint4((uint32_t)p0, (uint32_t)(p0 >> 32), j, a.tag), K);
            const uint4 r1 = philox4x32_10(make_uint4((uint32_t)p1, (uint32_t)(p1 >> 32), j, a.tag), K);
            halves(r0.x, r1.x, 0);
            halves(r0.y, r1.y, 2);
            halves(r0.z, r1.z, 4);
            halves(r0.w, r1.w, 6);
        }
    } else if (nf <= 2) {
        const uint4 ra = call_of(c0, 0);
        const uint4 rb = c1 == c0 ? ra : call_of(c1, 0);
        body(word(ra, (int)o0), word(rb, (int)o1), 0);
        if (nf == 2) body(word(ra, (int)o0 + 1), word(rb, (int)o1 + 1), 1);
    } else {
        // five uniforms per call (the four words, then the spare word): full
        // blocks of 10 fine steps from two calls, then the remaining 2, 4, 6
        // or 8 steps (2^l mod 10) from one or two more
        const uint32_t blocks = nf / 10u, rest = nf - 10u * blocks;
        for (uint32_t m = 0; m < blocks; ++m) {
            const uint4 a0 = call_of(p0, 2 * m), a1 = call_of(p1, 2 * m);
            body(a0.x, a1.x, 0);
            body(a0.y, a1.y, 1);
            body(a0.z, a1.z, 2);
            body(a0.w, a1.w, 3);
            body(spare_word(a0), spare_word(a1), 4);
            const uint4 b0 = call_of(p0, 2 * m + 1), b1 = call_of(p1, 2 * m + 1);
            body(b0.x, b1.x, 5);
            body(b0.y, b1.y, 6);
            body(b0.z, b1.z, 7);
            body(b0.w, b1.w, 8);
            body(spare_word(b0), spare_word(b1), 9);
        }
        if (rest) {
            const uint4 a0 = call_of(p0, 2 * blocks), a1 = call_of(p1, 2 * blocks);
            body(a0.x, a1.x, 0);
            body(a0.y, a1.y, 1);
            if (rest >= 4) {
                body(a0.z, a1.z, 2);
                body(a0.w, a1.w, 3);
            }
            if (rest >= 6) {
                body(spare_word(a0), spare_word(a1), 4);
                const uint4 b0 = call_of(p0, 2 * blocks + 1), b1 = call_of(p1, 2 * blocks + 1);
                body(b0.x, b1.x, 5);
                if (rest == 8) {
                    body(b0.y, b1.y, 6);
                    body(b0.z, b1.z, 7);
                }
            }
        }
    }

    pair_result<MODE>(a, fine, coarse, hfine, hcoarse, d0, d1, out0, out1);
}

// Pairs per lane slot.  On two-way paths at the coarsest levels a path
// needs fewer words than one Philox call holds (2^l < 4 words, or 2^l < 8
// halves with 16-bit uniforms), and the S = 4 / 2^l (8 / 2^l) consecutive
// paths S k .. S k + S - 1 share call 0 of counter path field k, path p
// taking the words (halves) from (p mod S) 2^l on; four-way paths at level
// 0 share a call in fours too (S = 4, both paths of a sample reading its
// word).  Where S > 2 one lane simulates all S paths of a call (S / 2
// pairs); elsewhere a slot is one pair (at S = 2 the pair shares its call,
// as simulate_pair does).
__host__ __device__ __forceinline__ int unit_pairs(int mode, int icdf, int l) {
    if (mode != MODE_TWO) return l == 0 ? 2 : 1;
    if (icdf == ICDF_TABLE16) return l == 0 ? 4 : (l == 1 ? 2 : 1);
    return l == 0 ? 2 : 1;
}

// The 2B paths of unit u, paths base .. base + 2B - 1 with base =
// path_offset + 2B u: position q = (base mod S) + i of path i runs over the
// S positions of call base / S, then of the next call (ALIGNED: base mod S
// = 0, one call).  Level L = 0 (one fine step) or 1 (two fine steps, one
// coarse; 16-bit uniforms only).  emit(i, P_f, P_c, D) receives every path
// in order.
template <int MODE, int B, int L, bool ALIGNED, int P, bool KAHAN, int ICDF, int SDE, class Emit>
__device__ __forceinline__ void simulate_unit(const LevelArgs &a, const PhiloxKeys &K, const SmemTable &tab,
                                              const float *mlp, uint64_t u, Emit &&emit) {
    constexpr uint32_t S = 2 * B;
    constexpr bool U16 = ICDF == ICDF_TABLE16 && MODE == MODE_TWO;     // four-way paths read 24-bit words
    static_assert(L == 0 || U16, "level-1 units use 16-bit uniforms");
    const uint64_t base = a.path_offset + S * u;
    const uint32_t m = ALIGNED ? 0u : (uint32_t)(base % S);
    const uint64_t cp = base / S;
    auto call_of = [&](uint64_t c) {
        return philox4x32_10(make_uint4((uint32_t)c, (uint32_t)(c >> 32), 0u, a.tag), K);
    };
    const uint4 r0 = call_of(cp);
    uint4 r1 = r0;
    if (!ALIGNED) r1 = call_of(cp + 1);
    // the word holding position q (positions are words, or halves when
    // U16 and L = 0)
    auto word_at = [&](uint32_t q) -> uint32_t {
        const uint32_t p = q % S;
        const int wi = (int)(U16 && L == 0 ? p >> 1 : p);
        return q < S ? word(r0, wi) : word(r1, wi);
    };
    auto half_at = [](uint32_t w, uint32_t hi) { return hi ? half16_bits<true>(w) : half16_bits<false>(w); };
#pragma unroll
    for (int k = 0; k < B; ++k) {
        const uint32_t q0 = m + 2 * k, q1 = q0 + 1;
        PathPair<P, KAHAN, SDE> fine, coarse;
        PathPair<P_F32, true, SDE> hfine, hcoarse;     // exact-normal pair (four-way, level 0)
        fine.template init<false>(a, false);
        if (L == 1) coarse.template init<false>(a, true);
        if constexpr (U16 && L == 0) {
            const uint32_t f0 = half_at(word_at(q0), q0 & 1), f1 = half_at(word_at(q1), q1 & 1);
            fine.step(table_pair<P, true>(tab, f0, f1, mirrored_v16(f0), mirrored_v16(f1)));
        } else if constexpr (U16) {
            const uint32_t w0 = word_at(q0), w1 = word_at(q1);
            const uint32_t a0 = half16_bits<false>(w0), a1 = half16_bits<false>(w1);
            const uint32_t b0 = half16_bits<true>(w0), b1 = half16_bits<true>(w1);
            const Pair<P> z1 = table_pair<P, true>(tab, a0, a1, mirrored_v16(a0), mirrored_v16(a1));
            const Pair<P> z2 = table_pair<P, true>(tab, b0, b1, mirrored_v16(b0), mirrored_v16(b1));
            fine.step(z1);
            fine.step(z2);
            coarse.step(add(z1, z2));
        } else {
            const uint32_t w0 = word_at(q0), w1 = word_at(q1);
            fine.step(icdf_pair<P, ICDF>(tab, mlp, w0, w1));
            if constexpr (MODE == MODE_FOUR) {
                hfine.template init<true>(a, false);
                hfine.step(Pair<P_F32>::of2(exact_z(tab, w0), exact_z(tab, w1)));
            }
        }
        float d0, d1, o0[5], o1[5];
        pair_result<MODE>(a, fine, coarse, hfine, hcoarse, d0, d1, o0, o1);
        emit(2 * k, o0, d0);
        emit(2 * k + 1, o1, d1);
    }
}

// One lane slot of the level described by a (slot g; inactive lanes
// simulate the last slot and discard it): its samples' D and D^2 go to
// k1, k2 in sample order, and with a.paths_out their outputs (3 or 5
// floats per sample).  Shared by the level and the batched kernels, so both
// accumulate identically.
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__device__ __forceinline__ void run_slot(const LevelArgs &a, const PhiloxKeys &K, const SmemTable &tab,
                                         const float *mlp, uint64_t g, bool active, KahanF32 &k1, KahanF32 &k2) {
    if (a.unit > 1) {
        const uint64_t first = (uint64_t)(2 * a.unit) * g;        // sample index of the unit's first path
        auto emit = [&](int i, const float *out, float d) {
            if (!active || first + i >= a.N) return;
            k1.add(d);
            k2.add(d * d);
            if (a.paths_out != nullptr) {
                constexpr int W = MODE == MODE_TWO ? 3 : 5;
                float *o = a.paths_out + (first + i) * W;
#pragma unroll
                for (int k = 0; k < W; ++k) o[k] = out[k];
            }
        };
        const bool aligned = a.path_offset % (uint64_t)(2 * a.unit) == 0;
        if constexpr (ICDF == ICDF_TABLE16 && MODE == MODE_TWO) {
            if (a.l == 0) {
                if (aligned) simulate_unit<MODE, 4, 0, true, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
                else simulate_unit<MODE, 4, 0, false, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
            } else {
                if (aligned) simulate_unit<MODE, 2, 1, true, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
                else simulate_unit<MODE, 2, 1, false, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
            }
        } else {
            if (aligned) simulate_unit<MODE, 2, 0, true, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
            else simulate_unit<MODE, 2, 0, false, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, emit);
        }
        return;
    }
    float d0, d1, out0[5], out1[5];
    simulate_pair<MODE, P, KAHAN, ICDF, SDE>(a, K, tab, mlp, g, d0, d1, out0, out1);
    const bool valid1 = 2 * g + 1 < a.N;
    if (active) {
        k1.add(d0);
        k2.add(d0 * d0);
        if (valid1) {
            k1.add(d1);
            k2.add(d1 * d1);
        }
    }
    if (active && a.paths_out != nullptr) {
        constexpr int W = MODE == MODE_TWO ? 3 : 5;
        float *o = a.paths_out + (2 * g) * W;
#pragma unroll
        for (int k = 0; k < W; ++k) o[k] = out0[k];
        if (valid1) {
#pragma unroll
            for (int k = 0; k < W; ++k) o[W + k] = out1[k];
        }
    }
}

__device__ __forceinline__ void stage_table(SmemTable &tab, const DevTables *t) {
    static_assert(sizeof(SmemTable) % 4 == 0, "table size");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&t->e);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&tab);
    for (int i = threadIdx.x; i < (int)(sizeof(SmemTable) / 4); i += blockDim.x) dst[i] = src[i];
}

// Warp sum in FP32.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Chunks of 32 consecutive pairs (one per lane), in groups of
// chunk_group(l, chunks) chunks.  With chunk_partials the grid is persistent:
// each warp takes the next group from an atomic counter (a.counter, zeroed
// before the launch) until none is left; its lanes accumulate the group's
// samples in FP32
// (Kahan) and the warp sum goes, in FP64, to the group's own slot, so the
// finalize kernel adds the same values in the same order whatever the grid
// or the schedule.  Otherwise warp w takes chunks w, w + W, ... and one slot
// per block holds the block's sum (warps added in FP64).
//
// Group size: up to 64 >> l chunks at coarse levels (where a chunk is
// short), but at least GROUP_TARGET groups when there are enough chunks, so
// that every resident warp gets several groups.  It depends on (l, N) only,
// never on the device or the launch shape.
constexpr uint64_t GROUP_TARGET = 16384;
__host__ __device__ __forceinline__ uint32_t chunk_group(int l, uint64_t chunks) {
    if (l >= 6) return 1u;
    const uint64_t by_count = chunks / GROUP_TARGET;
    const uint64_t g = by_count < (64u >> l) ? by_count : (64u >> l);
    return g > 1 ? (uint32_t)g : 1u;
}

// Register budget: two-way kernels fit 64 registers (4 blocks of 256 per
// SM); four-way kernels carry four paths per sample and get 80 (3 blocks),
// which removes their spills (measured 8 % faster on GB300 than 64 registers
// with spills).  The network's normals come from its tabulated grid values,
// so the MLP kernels have the same budgets.
template <int MODE, int P, bool KAHAN, int ICDF, int SDE>
__global__ void __launch_bounds__(256, MODE == MODE_FOUR ? 3 : 4) level_kernel(const LevelArgs a) {
    __shared__ SmemTable tab;
    __shared__ double red[2][32];
    if (ICDF != ICDF_MLP || MODE == MODE_FOUR) {
        stage_table(tab, a.tabs);
        __syncthreads();
    }
    const float *mlp = ICDF == ICDF_MLP ? a.mlp->ygrid : nullptr;
    KahanF32 k1, k2;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t warp_id = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nchunks = (a.npairs + 31) >> 5;
    const uint64_t G = a.chunk_partials ? chunk_group(a.l, nchunks) : 1;
    for (uint64_t grp = warp_id;; grp += warps) {
        if (a.chunk_partials) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(a.counter, 1ull);
            grp = __shfl_sync(0xffffffffu, t, 0);
        }
        const uint64_t c0 = grp * G;
        if (c0 >= nchunks) break;
        const uint64_t c1 = c0 + G < nchunks ? c0 + G : nchunks;
        for (uint64_t c = c0; c < c1; ++c) {
            const uint64_t g = c * 32 + lane;
            const bool active = g < a.npairs;
            run_slot<MODE, P, KAHAN, ICDF, SDE>(a, a.rk, tab, mlp, active ? g : a.npairs - 1, active, k1, k2);
        }
        if (a.chunk_partials) {
            const float w1 = warp_sum(k1.value()), w2 = warp_sum(k2.value());
            if (lane == 0) a.partials[grp] = make_double2((double)w1, (double)w2);
            k1 = KahanF32();
            k2 = KahanF32();
        }
    }
    if (a.chunk_partials) return;
    // warp reduction in FP32, then FP64 across warps
    const float s1 = warp_sum(k1.value());
    const float s2 = warp_sum(k2.value());
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = (double)s1;
        red[1][warp] = (double)s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        a.partials[blockIdx.x] = make_double2(t1, t2);
    }
}

using LevelKernelFn = void (*)(LevelArgs);

}  // namespace mlmc
