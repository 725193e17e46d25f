// Device building blocks of the level kernels (sm_103a).
//
// Philox4x32-10, the 24-bit uniform map, rounding-exact arithmetic on path
// pairs (binary32 pairs and packed binary16x2), and the inverse CDFs:
// exact Phi^-1 in FP32 and the 16-interval piecewise-linear approximation
// (Sec. 2.1) staged in shared memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace mlmc {

// ---------------------------------------------------------------- RNG
// Philox4x32-10 (Salmon et al. 2011): ten rounds of two 32x32->64 products
// with a Weyl key schedule.  The key is the same for every thread (the
// seed), so the schedule stays in uniform registers.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The ten round keys of one key (seed): (k0 + r W0, k1 + r W1) for r = 0..9,
// computed once on the host.  Kernels read them from their parameter space,
// so each round takes its key as an operand instead of advancing the
// schedule in registers.
struct PhiloxKeys {
    uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_round_keys(uint32_t k0, uint32_t k1) {
    PhiloxKeys K;
    for (int r = 0; r < 10; ++r) {
        K.k[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        K.k[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
    return K;
}

// Philox4x32-10 with the precomputed round keys (the same function as
// philox4x32_10(c, k0, k1)).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ K.k[2 * r], lo1, hi0 ^ c.w ^ K.k[2 * r + 1], lo0);
    }
    return c;
}

__device__ __forceinline__ uint32_t word(const uint4 &w, int q) {
    return q == 0 ? w.x : q == 1 ? w.y : q == 2 ? w.z : w.w;
}

// The fifth uniform of a Philox call (x, y, z, w): a uniform reads a word's
// top 23 bits, so the low bytes of x, y and z, placed as bits 8..15, 16..23
// and 24..31 of a spare word (two byte permutes; its bits 0..7 are not
// read), give one more from bits no other uniform of the call reads.
__device__ __forceinline__ uint32_t spare_word(const uint4 &r) {
    return __byte_perm(__byte_perm(r.x, r.y, 0x0400u), r.z, 0x4210u);
}

// u = (2 (w >> 9) + 1) 2^-24, exact in binary32.
__device__ __forceinline__ float uniform_of(uint32_t w) {
    return __fsub_rn(__uint_as_float((w >> 9) | 0x3F800000u), 0x1.fffffep-1f);
}

// v = min(u, 1 - u) for the same u, exact: f = 1 + (w >> 9) 2^-23 (one
// funnel shift), s = (f - 3/2) + 2^-24 = u - 1/2 and v = 1/2 - |s| are exact
// binary32 operations on the grid (at most 23 significant bits), and keep
// the work on the FP32 pipe rather than the integer ALU.
__device__ __forceinline__ float mirrored_v(uint32_t w) {
    const float f = __uint_as_float(__funnelshift_r(w, 0x7Fu, 9));
    const float s = __fadd_rn(__fsub_rn(f, 1.5f), 0x1p-24f);
    return __fsub_rn(0.5f, fabsf(s));
}

// 16-bit uniforms u = (h + 1/2) 2^-16.  half16_bits<HI>(w) places half h of
// w (low or high 16 bits) under the binary32 exponent of 128 with one byte
// permute: f = 128 + h 2^-16, so bit 15 of the result is the top bit of h
// (set exactly when u > 1/2).
template <bool HI>
__device__ __forceinline__ uint32_t half16_bits(uint32_t w) {
    return __byte_perm(w, 0x43000000u, HI ? 0x7432u : 0x7410u);
}

// v = min(u, 1 - u) of such a 16-bit uniform, exact:
// s = (f - 128.5) + 2^-17 = u - 1/2, v = 1/2 - |s|.
__device__ __forceinline__ float mirrored_v16(uint32_t fbits) {
    const float s = __fadd_rn(__fsub_rn(__uint_as_float(fbits), 128.5f), 0x1p-17f);
    return __fsub_rn(0.5f, fabsf(s));
}


// ---------------------------------------------------------------- arithmetic
// Every operation is a single IEEE operation rounded to nearest even; none
// is ever fused into an FMA (Sec. 2.2 models exactly this operation order).
__device__ __forceinline__ __half2 h2add(__half2 a, __half2 b) {
    __half2 r;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(*reinterpret_cast<uint32_t *>(&r))
        : "r"(*reinterpret_cast<uint32_t *>(&a)), "r"(*reinterpret_cast<uint32_t *>(&b)));
    return r;
}
__device__ __forceinline__ __half2 h2sub(__half2 a, __half2 b) {
    __half2 r;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(*reinterpret_cast<uint32_t *>(&r))
        : "r"(*reinterpret_cast<uint32_t *>(&a)), "r"(*reinterpret_cast<uint32_t *>(&b)));
    return r;
}
__device__ __forceinline__ __half2 h2mul(__half2 a, __half2 b) {
    __half2 r;
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(*reinterpret_cast<uint32_t *>(&r))
        : "r"(*reinterpret_cast<uint32_t *>(&a)), "r"(*reinterpret_cast<uint32_t *>(&b)));
    return r;
}

// bfloat16x2 arithmetic, each operation rounded to nearest even, never fused.
__device__ __forceinline__ uint32_t b2add(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("add.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t b2sub(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("sub.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ uint32_t b2mul(uint32_t a, uint32_t b) {
    uint32_t r;
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
// binary64 -> bfloat16 with a single rounding to nearest even.
__device__ __forceinline__ uint16_t f64_to_bf16(double v) {
    unsigned short r;
    asm("cvt.rn.bf16.f64 %0, %1;" : "=h"(r) : "d"(v));
    return r;
}
// two binary32 -> bfloat16x2 (lo = a, hi = b), rounded to nearest even.
__device__ __forceinline__ uint32_t f32x2_to_bf16x2(float a, float b) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(b), "f"(a));
    return r;
}

// binary64 -> binary16 with a single rounding to nearest even.
__device__ __forceinline__ __half f64_to_f16(double v) {
    unsigned short r;
    asm("cvt.rn.f16.f64 %0, %1;" : "=h"(r) : "d"(v));
    return __ushort_as_half(r);
}

// A pair of paths in working precision P: two binary32 values or one
// packed binary16x2 / bfloat16x2 register.
enum { P_F32 = 0, P_F16 = 1, P_BF16 = 2 };

template <int P> struct Pair;

template <> struct Pair<P_F32> {
    float x, y;
    static __device__ __forceinline__ Pair of(double v) { float f = __double2float_rn(v); return {f, f}; }
    static __device__ __forceinline__ Pair of2(float a, float b) { return {a, b}; }
    // a constant from its binary32 bits
    static __device__ __forceinline__ Pair bits(uint32_t b) { return {__uint_as_float(b), __uint_as_float(b)}; }
    __device__ __forceinline__ float2 f32() const { return make_float2(x, y); }
};
template <> struct Pair<P_F16> {
    __half2 h;
    static __device__ __forceinline__ Pair of(double v) { __half t = f64_to_f16(v); return {__halves2half2(t, t)}; }
    static __device__ __forceinline__ Pair of2(float a, float b) { return {__floats2half2_rn(a, b)}; }
    // a constant from its packed binary16x2 bits
    static __device__ __forceinline__ Pair bits(uint32_t b) { return {*reinterpret_cast<const __half2 *>(&b)}; }
    __device__ __forceinline__ float2 f32() const { return __half22float2(h); }
};

template <> struct Pair<P_BF16> {
    uint32_t b;      // lo = path 0, hi = path 1
    static __device__ __forceinline__ Pair of(double v) {
        const uint32_t h = f64_to_bf16(v);
        return {h | (h << 16)};
    }
    static __device__ __forceinline__ Pair of2(float a, float c) { return {f32x2_to_bf16x2(a, c)}; }
    static __device__ __forceinline__ Pair bits(uint32_t b) { return {b}; }
    __device__ __forceinline__ float2 f32() const {
        return make_float2(__uint_as_float(b << 16), __uint_as_float(b & 0xFFFF0000u));
    }
};

__device__ __forceinline__ Pair<P_F32> add(Pair<P_F32> a, Pair<P_F32> b) { return {__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y)}; }
__device__ __forceinline__ Pair<P_F32> sub(Pair<P_F32> a, Pair<P_F32> b) { return {__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y)}; }
__device__ __forceinline__ Pair<P_F32> mul(Pair<P_F32> a, Pair<P_F32> b) { return {__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y)}; }
__device__ __forceinline__ Pair<P_F16> add(Pair<P_F16> a, Pair<P_F16> b) { return {h2add(a.h, b.h)}; }
__device__ __forceinline__ Pair<P_F16> sub(Pair<P_F16> a, Pair<P_F16> b) { return {h2sub(a.h, b.h)}; }
__device__ __forceinline__ Pair<P_F16> mul(Pair<P_F16> a, Pair<P_F16> b) { return {h2mul(a.h, b.h)}; }
__device__ __forceinline__ Pair<P_BF16> add(Pair<P_BF16> a, Pair<P_BF16> b) { return {b2add(a.b, b.b)}; }
__device__ __forceinline__ Pair<P_BF16> sub(Pair<P_BF16> a, Pair<P_BF16> b) { return {b2sub(a.b, b.b)}; }
__device__ __forceinline__ Pair<P_BF16> mul(Pair<P_BF16> a, Pair<P_BF16> b) { return {b2mul(a.b, b.b)}; }

// Kahan-compensated FP32 accumulator (Algorithm 1) for the per-thread sums
// of D and D^2; value() is the compensated sum s - c.
struct KahanF32 {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ float value() const { return __fsub_rn(s, c); }
};

// ---------------------------------------------------------------- inverse CDFs
// TABLE16: the table at a 16-bit uniform (two per Philox word on two-way
// paths; the cell centre of the 24-bit uniform on four-way bar paths).
// CUBIC: the piecewise cubic.
enum { ICDF_EXACT = 0, ICDF_TABLE = 1, ICDF_MLP = 2, ICDF_TABLE16 = 3, ICDF_CUBIC = 4 };

// Shared-memory copy of the piecewise-linear table, indexed by the biased
// binary32 exponent E of v: v in [2^(E-127), 2^(E-126)) lies in interval
// k = 126 - E (k = 1..15) or in interval 16 for E <= 110.  Entry E - 103
// for E = 103..125 (v >= 2^-24 on the uniform grid).
constexpr int TAB_ENTRIES = 23;
struct SmemTable {
    float2 c32[TAB_ENTRIES];     // linear (c0, c1) in binary32
    __half2 c16[TAB_ENTRIES];    // linear (c0, c1) in binary16
    uint32_t cb16[TAB_ENTRIES];  // linear (c0, c1) in bfloat16 (c0 in the low half)
    float4 q32[TAB_ENTRIES];     // cubic (d0, d1, d2, d3) in binary32
    uint2 q16[TAB_ENTRIES];      // cubic in binary16: (d0 | d1 << 16, d2 | d3 << 16)
    uint2 qbf[TAB_ENTRIES];      // cubic in bfloat16, same packing
    float2 qab[TAB_ENTRIES];     // cubic local variable s = A v - B as (A, -B)
    float4 ex[TAB_ENTRIES][2];   // exact normal: q0..q7 of Phi^-1(v) = (v - 1/2) q(s), one binade each
};

// The per-device tables: the entries staged by the kernels, and the FP64
// coefficients in interval order (intervals 1..16) for export.
struct DevTables {
    SmemTable e;
    double lin64[32];            // linear (c0, c1)
    double cub64[64];            // cubic (d0, d1, d2, d3)
};

// Entry index of v; CLAMP widens it to any v in (0, 1/2] (bulk API).
template <bool CLAMP>
__device__ __forceinline__ int tab_index(float v) {
    int e = (int)(__float_as_uint(v) >> 23);
    if (CLAMP) e = min(max(e, 103), 125);
    return e - 103;
}

// Exact normal in binary32 on the uniform grid (v >= 2^-24): on the binade
// [2^(E-127), 2^(E-126)) of v, Phi^-1(v) = (v - 1/2) q(s) with s = v 2^(128-E)
// - 3 in [-1, 1) (exact: v's significand under the exponent of 2, minus 3)
// and q of degree 7 interpolating Phi^-1(v)/(v - 1/2) at the Chebyshev
// points (built on the device from FP64 Phi^-1); FMA Horner.  Measured
// against FP64 over the whole grid: at most 2.5 ulp.  The sign is the
// word's half.
__device__ __forceinline__ float exact_zv(const SmemTable &t, uint32_t w, float v) {
    const uint32_t vb = __float_as_uint(v);
    const int i = (int)(vb >> 23) - 103;
    const float s = __fsub_rn(__uint_as_float((vb & 0x007FFFFFu) | 0x40000000u), 3.0f);
    const float4 a = t.ex[i][0], b = t.ex[i][1];
    float q = __fmaf_rn(b.w, s, b.z);
    q = __fmaf_rn(q, s, b.y);
    q = __fmaf_rn(q, s, b.x);
    q = __fmaf_rn(q, s, a.w);
    q = __fmaf_rn(q, s, a.z);
    q = __fmaf_rn(q, s, a.y);
    q = __fmaf_rn(q, s, a.x);
    const float z = __fmul_rn(__fsub_rn(v, 0.5f), q);
    return __uint_as_float(__float_as_uint(z) ^ (w & 0x80000000u));
}

__device__ __forceinline__ float exact_z(const SmemTable &t, uint32_t w) { return exact_zv(t, w, mirrored_v(w)); }

// Piecewise-linear Z~ in binary32: z = R(c0 + R(c1 v)), negated for u > 1/2.
// The sign is bit 31 of w (SIGN15: bit 15, for half16_bits words).
template <bool CLAMP, bool SIGN15 = false>
__device__ __forceinline__ float table_z32(const SmemTable &s, uint32_t w, float v) {
    const float2 c = s.c32[tab_index<CLAMP>(v)];
    const float z = __fadd_rn(c.x, __fmul_rn(c.y, v));
    return __uint_as_float(__float_as_uint(z) ^ ((SIGN15 ? w << 16 : w) & 0x80000000u));
}

// Piecewise-linear Z~ for two paths in binary16x2:
// z = R16(R16(c0) + R16(R16(c1) R16(v))), negated for u > 1/2.
template <bool CLAMP, bool SIGN15 = false>
__device__ __forceinline__ __half2 table_z16(const SmemTable &s, uint32_t w0, uint32_t w1, float v0, float v1) {
    const __half2 t0 = s.c16[tab_index<CLAMP>(v0)];
    const __half2 t1 = s.c16[tab_index<CLAMP>(v1)];
    const __half2 c0 = __lows2half2(t0, t1);
    const __half2 c1 = __highs2half2(t0, t1);
    const __half2 v = __floats2half2_rn(v0, v1);
    __half2 z = h2add(c0, h2mul(c1, v));
    // sign bits of the two words into bits 15 and 31 (top bytes of w0, w1;
    // SIGN15: second bytes)
    const uint32_t top = __byte_perm(w0, w1, SIGN15 ? 0x5010u : 0x7030u);
    uint32_t zb = *reinterpret_cast<uint32_t *>(&z) ^ (top & 0x80008000u);
    return *reinterpret_cast<__half2 *>(&zb);
}

// Piecewise-linear Z~ for two paths in bfloat16x2, same operation order.
template <bool CLAMP, bool SIGN15 = false>
__device__ __forceinline__ uint32_t table_zbf16(const SmemTable &s, uint32_t w0, uint32_t w1, float v0, float v1) {
    const uint32_t t0 = s.cb16[tab_index<CLAMP>(v0)];
    const uint32_t t1 = s.cb16[tab_index<CLAMP>(v1)];
    const uint32_t c0 = __byte_perm(t0, t1, 0x5410u);     // lo halves
    const uint32_t c1 = __byte_perm(t0, t1, 0x7632u);     // hi halves
    const uint32_t z = b2add(c0, b2mul(c1, f32x2_to_bf16x2(v0, v1)));
    const uint32_t top = __byte_perm(w0, w1, SIGN15 ? 0x5010u : 0x7030u);
    return z ^ (top & 0x80008000u);
}

}  // namespace mlmc

namespace mlmc {

// Piecewise-cubic Z~ (the high-fidelity approximation of Sec. 2.2): on the
// interval of v the local variable s = A v - B lies in [-1, 1]; it is formed
// with one rounding of the exact value (exact on the uniform grid), then
// Horner with every operation rounded:
//   z = R(d0 + R(s R(d1 + R(s R(d2 + R(s d3)))))),  negated for u > 1/2.
template <bool CLAMP>
__device__ __forceinline__ float cubic_z32(const SmemTable &t, uint32_t w, float v) {
    const int i = tab_index<CLAMP>(v);
    const float2 ab = t.qab[i];
    const float4 d = t.q32[i];
    const float s = __fmaf_rn(v, ab.x, ab.y);
    float z = __fmul_rn(s, d.w);
    z = __fadd_rn(d.z, z);
    z = __fmul_rn(s, z);
    z = __fadd_rn(d.y, z);
    z = __fmul_rn(s, z);
    z = __fadd_rn(d.x, z);
    return __uint_as_float(__float_as_uint(z) ^ (w & 0x80000000u));
}

// Two samples in binary16x2 (lo = sample of w0/v0, hi = w1/v1).
template <bool CLAMP>
__device__ __forceinline__ __half2 cubic_z16(const SmemTable &t, uint32_t w0, uint32_t w1, float v0, float v1) {
    const int i0 = tab_index<CLAMP>(v0), i1 = tab_index<CLAMP>(v1);
    const float2 ab0 = t.qab[i0], ab1 = t.qab[i1];
    const uint2 q0 = t.q16[i0], q1 = t.q16[i1];
    const __half2 s = __floats2half2_rn(__fmaf_rn(v0, ab0.x, ab0.y), __fmaf_rn(v1, ab1.x, ab1.y));
    uint32_t d[4] = {__byte_perm(q0.x, q1.x, 0x5410u), __byte_perm(q0.x, q1.x, 0x7632u),
                     __byte_perm(q0.y, q1.y, 0x5410u), __byte_perm(q0.y, q1.y, 0x7632u)};
    const __half2 *dh = reinterpret_cast<const __half2 *>(d);
    __half2 z = h2mul(s, dh[3]);
    z = h2add(dh[2], z);
    z = h2mul(s, z);
    z = h2add(dh[1], z);
    z = h2mul(s, z);
    z = h2add(dh[0], z);
    const uint32_t top = __byte_perm(w0, w1, 0x7030u);
    uint32_t zb = *reinterpret_cast<uint32_t *>(&z) ^ (top & 0x80008000u);
    return *reinterpret_cast<__half2 *>(&zb);
}

// Two samples in bfloat16x2, same operation order.
template <bool CLAMP>
__device__ __forceinline__ uint32_t cubic_zbf16(const SmemTable &t, uint32_t w0, uint32_t w1, float v0, float v1) {
    const int i0 = tab_index<CLAMP>(v0), i1 = tab_index<CLAMP>(v1);
    const float2 ab0 = t.qab[i0], ab1 = t.qab[i1];
    const uint2 q0 = t.qbf[i0], q1 = t.qbf[i1];
    const uint32_t s = f32x2_to_bf16x2(__fmaf_rn(v0, ab0.x, ab0.y), __fmaf_rn(v1, ab1.x, ab1.y));
    uint32_t z = b2mul(s, __byte_perm(q0.y, q1.y, 0x7632u));
    z = b2add(__byte_perm(q0.y, q1.y, 0x5410u), z);
    z = b2mul(s, z);
    z = b2add(__byte_perm(q0.x, q1.x, 0x7632u), z);
    z = b2mul(s, z);
    z = b2add(__byte_perm(q0.x, q1.x, 0x5410u), z);
    const uint32_t top = __byte_perm(w0, w1, 0x7030u);
    return z ^ (top & 0x80008000u);
}

}  // namespace mlmc
