// Small kernels: table construction, finalize reduction, and the bulk RNG /
// inverse-CDF entry points.
#include <math.h>

#include "internal.h"
#include "level_kernels.cuh"
#include "reduce.cuh"

namespace mlmc {

// ---------------------------------------------------------------- tables
// Piecewise-linear table: L2 (uniform-measure) linear fit of Phi^-1 on each
// interval [a, b) of v = min(u, 1-u): I_k = [2^-(k+1), 2^-k) for k = 1..15,
// I_16 = (0, 2^-16) (Sec. 2.1; the construction is deferred by the paper to
// its cited work, this is the least-squares reading).  The moments have
// closed forms in z = Phi^-1(v):
//   int_a^b Phi^-1(v) dv   = phi(z_a) - phi(z_b)
//   int_a^b v Phi^-1(v) dv = [ -phi(z) Phi(z) + Phi(sqrt(2) z) / (2 sqrt(pi)) ]_{z_a}^{z_b}
// and the normal equations are solved in centred form.
//
// Piecewise-cubic table (the high-fidelity approximation of Sec. 2.2): the
// L2 cubic fit on the same intervals in the local variable s = A v - B in
// [-1, 1] (A = 2^(k+2), B = 3 for k <= 15; A = 2^17, B = 1 for k = 16),
// computed as the projection on the Legendre polynomials P0..P3 of s by
// Gauss-Legendre quadrature (24 nodes per piece; I_16 is split into dyadic
// pieces down to 2^-76, below which the moments change by < 1e-17), then
// expanded in powers of s.
constexpr int GL_N = 24;
constexpr int CUBIC_TAIL_PIECES = 60;

// Gauss-Legendre nodes and weights on [-1, 1]: node i is the root of P_n
// found by Newton's method from cos(pi (i + 3/4) / (n + 1/2)), with the
// three-term recurrence for P_n and P_n' = n (x P_n - P_{n-1}) / (x^2 - 1);
// weight 2 / ((1 - x^2) P_n'(x)^2).  At most 100 iterations.
__device__ void gauss_legendre_node(int i, double &x, double &w) {
    x = cos(3.14159265358979323846 * (i + 0.75) / (GL_N + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = x;
        for (int n = 2; n <= GL_N; ++n) {
            const double p2 = ((2 * n - 1) * x * p1 - (n - 1) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        dp = GL_N * (x * p1 - p0) / (x * x - 1.0);
        const double dx = p1 / dp;
        x -= dx;
        if (fabs(dx) < 1e-16) break;
    }
    w = 2.0 / ((1.0 - x * x) * dp * dp);
}

// Exact-normal polynomial of table entry i (binade E = 103 + i of v):
// Phi^-1(v) / (v - 1/2) interpolated at the 8 Chebyshev points of
// s = v 2^(128-E) - 3 in [-1, 1], returned as monomial coefficients in s.
__device__ void exact_poly(int i, double q[8]) {
    constexpr int n = 8;
    const double A = ldexp(1.0, 128 - (103 + i));
    double y[n], x[n];
    for (int k = 0; k < n; ++k) {
        x[k] = cos(3.14159265358979323846 * (k + 0.5) / n);
        const double v = (x[k] + 3.0) / A;
        y[k] = normcdfinv(v) / (v - 0.5);
    }
    // Chebyshev coefficients c_j = (2/n) sum_k y_k T_j(x_k), c_0 halved
    double c[n];
    for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += y[k] * cos(j * acos(x[k]));
        c[j] = acc * 2.0 / n;
    }
    c[0] *= 0.5;
    // sum_j c_j T_j(s) in powers of s (T_{j+1} = 2 s T_j - T_{j-1})
    double tm[n], t0[n], t1[n];
    for (int m = 0; m < n; ++m) q[m] = t0[m] = t1[m] = 0.0;
    t0[0] = 1.0;
    t1[1] = 1.0;
    for (int m = 0; m < n; ++m) q[m] += c[0] * t0[m] + c[1] * t1[m];
    for (int j = 2; j < n; ++j) {
        for (int m = 0; m < n; ++m) tm[m] = (m > 0 ? 2.0 * t1[m - 1] : 0.0) - t0[m];
        for (int m = 0; m < n; ++m) {
            q[m] += c[j] * tm[m];
            t0[m] = t1[m];
            t1[m] = tm[m];
        }
    }
}

__device__ __forceinline__ int entry_interval(int entry) {     // 0-based interval of table entry E - 103
    return min(126 - (103 + entry), 16) - 1;
}

// One block of BUILD_THREADS threads: thread k-1 fits linear interval k; for the cubic,
// thread j < 75 integrates one piece (pieces 0..14: intervals 1..15; pieces
// 15..74: the dyadic pieces of interval 16), and the pieces of interval 16
// are added in a fixed order.
constexpr int BUILD_THREADS = 96;
__global__ void __launch_bounds__(BUILD_THREADS) build_table_kernel(DevTables *out) {
    __shared__ double lin[32], cub[64], glx[GL_N], glw[GL_N], piece[15 + CUBIC_TAIL_PIECES][4];
    const int i = threadIdx.x;
    if (i < GL_N) gauss_legendre_node(i, glx[i], glw[i]);
    if (i < 16) {
        const int k = i + 1;
        const double b = ldexp(1.0, -k);
        const double a = k < 16 ? ldexp(1.0, -(k + 1)) : 0.0;
        const double inv_sqrt2pi = 0.39894228040143267794;
        const double inv_2sqrtpi = 0.28209479177387814347;
        const double zb = normcdfinv(b);
        const double phib = inv_sqrt2pi * exp(-0.5 * zb * zb);
        double F0 = -phib;
        double F1 = -phib * b + inv_2sqrtpi * normcdf(1.41421356237309504880 * zb);
        if (a > 0.0) {
            const double za = normcdfinv(a);
            const double phia = inv_sqrt2pi * exp(-0.5 * za * za);
            F0 += phia;
            F1 -= -phia * a + inv_2sqrtpi * normcdf(1.41421356237309504880 * za);
        }
        const double M0 = b - a;
        const double vbar = 0.5 * (a + b);
        const double Svv = M0 * M0 * M0 / 12.0;
        const double c1 = (F1 - vbar * F0) / Svv;
        const double c0 = F0 / M0 - c1 * vbar;
        lin[2 * i] = c0;
        lin[2 * i + 1] = c1;
    }
    __syncthreads();
    if (i < 15 + CUBIC_TAIL_PIECES) {
        const int k = i < 15 ? i + 1 : 16;
        const int j = i - 15;                                     // tail piece index
        const double A = k < 16 ? ldexp(1.0, k + 2) : ldexp(1.0, 17);
        const double B = k < 16 ? 3.0 : 1.0;
        const double hi = k < 16 ? ldexp(1.0, -k) : ldexp(1.0, -16 - j);
        const double lo = k < 16 ? ldexp(1.0, -k - 1) : ldexp(1.0, -17 - j);
        const double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
        double pr[4] = {0.0, 0.0, 0.0, 0.0};
        for (int q = 0; q < GL_N; ++q) {
            const double v = mid + half * glx[q];
            const double s = A * v - B;
            const double wf = half * glw[q] * A * normcdfinv(v);     // ds = A dv
            pr[0] += wf;
            pr[1] += wf * s;
            pr[2] += wf * 0.5 * (3.0 * s * s - 1.0);
            pr[3] += wf * 0.5 * (5.0 * s * s * s - 3.0 * s);
        }
        for (int m = 0; m < 4; ++m) piece[i][m] = pr[m];
    }
    __syncthreads();
    if (i < 16) {
        double pr[4];
        for (int m = 0; m < 4; ++m) pr[m] = i < 15 ? piece[i][m] : 0.0;
        if (i == 15)
            for (int j = 0; j < CUBIC_TAIL_PIECES; ++j)
                for (int m = 0; m < 4; ++m) pr[m] += piece[15 + j][m];
        const double a0 = 0.5 * pr[0], a1 = 1.5 * pr[1], a2 = 2.5 * pr[2], a3 = 3.5 * pr[3];
        cub[4 * i] = a0 - 0.5 * a2;
        cub[4 * i + 1] = a1 - 1.5 * a3;
        cub[4 * i + 2] = 1.5 * a2;
        cub[4 * i + 3] = 2.5 * a3;
    }
    __syncthreads();
    if (i < 32) out->lin64[i] = lin[i];
    for (int j = i; j < 64; j += blockDim.x) out->cub64[j] = cub[j];
    if (i < TAB_ENTRIES) {
        const int iv = entry_interval(i);
        const double c0 = lin[2 * iv], c1 = lin[2 * iv + 1];
        out->e.c32[i] = make_float2(__double2float_rn(c0), __double2float_rn(c1));
        out->e.c16[i] = __halves2half2(f64_to_f16(c0), f64_to_f16(c1));
        out->e.cb16[i] = (uint32_t)f64_to_bf16(c0) | ((uint32_t)f64_to_bf16(c1) << 16);
        const double *d = cub + 4 * iv;
        out->e.q32[i] = make_float4(__double2float_rn(d[0]), __double2float_rn(d[1]), __double2float_rn(d[2]),
                                    __double2float_rn(d[3]));
        auto h16 = [](double x) { return (uint32_t)__half_as_ushort(f64_to_f16(x)); };
        out->e.q16[i] = make_uint2(h16(d[0]) | (h16(d[1]) << 16), h16(d[2]) | (h16(d[3]) << 16));
        out->e.qbf[i] = make_uint2((uint32_t)f64_to_bf16(d[0]) | ((uint32_t)f64_to_bf16(d[1]) << 16),
                                   (uint32_t)f64_to_bf16(d[2]) | ((uint32_t)f64_to_bf16(d[3]) << 16));
        const int k = iv + 1;
        out->e.qab[i] = make_float2(k < 16 ? ldexpf(1.0f, k + 2) : 131072.0f, k < 16 ? -3.0f : -1.0f);
        double q[8];
        exact_poly(i, q);
        out->e.ex[i][0] = make_float4(__double2float_rn(q[0]), __double2float_rn(q[1]), __double2float_rn(q[2]),
                                      __double2float_rn(q[3]));
        out->e.ex[i][1] = make_float4(__double2float_rn(q[4]), __double2float_rn(q[5]), __double2float_rn(q[6]),
                                      __double2float_rn(q[7]));
    }
}

cudaError_t launch_build_table(DevTables *out, cudaStream_t s) {
    build_table_kernel<<<1, BUILD_THREADS, 0, s>>>(out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- finalize
// Deterministic FP64 sum of the partials (block_sum_fixed): one block when
// the partials fit one span; otherwise a first pass, one block per span,
// writes the span sums and one block adds those.
__global__ void __launch_bounds__(SUM_THREADS) finalize_kernel(const double2 *partials, uint64_t count,
                                                               uint64_t spans, double2 *out) {
    __shared__ double r1[SUM_THREADS], r2[SUM_THREADS];
    const uint64_t lo = (uint64_t)blockIdx.x * FINALIZE_SPAN;
    const uint64_t n = spans == 0 ? count : (lo + FINALIZE_SPAN < count ? FINALIZE_SPAN : count - lo);
    const double2 s = block_sum_fixed(partials + lo, n, r1, r2);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

uint64_t finalize_scratch(uint64_t count) { return count <= FINALIZE_SPAN ? 0 : (count + FINALIZE_SPAN - 1) / FINALIZE_SPAN; }

cudaError_t launch_finalize(const double2 *partials, uint64_t count, double *out, double2 *scratch, cudaStream_t s) {
    const uint64_t spans = finalize_scratch(count);
    if (spans == 0) {
        finalize_kernel<<<1, SUM_THREADS, 0, s>>>(partials, count, 0, reinterpret_cast<double2 *>(out));
    } else {
        finalize_kernel<<<(unsigned)spans, SUM_THREADS, 0, s>>>(partials, count, spans, scratch);
        finalize_kernel<<<1, SUM_THREADS, 0, s>>>(scratch, spans, 0, reinterpret_cast<double2 *>(out));
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bulk RNG
__global__ void philox_bulk_kernel(const uint4 *ctr, const uint2 *key, uint4 *out, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = philox4x32_10(ctr[i], key[i].x, key[i].y);
}

__global__ void uniform_bulk_kernel(const uint32_t *w, float *u, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        u[i] = uniform_of(w[i]);
}

static int bulk_grid(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_philox_bulk(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t n, cudaStream_t s) {
    philox_bulk_kernel<<<bulk_grid(n), 256, 0, s>>>(reinterpret_cast<const uint4 *>(ctr),
                                                     reinterpret_cast<const uint2 *>(key),
                                                     reinterpret_cast<uint4 *>(out), n);
    return cudaGetLastError();
}

cudaError_t launch_uniform_bulk(const uint32_t *w, float *u, size_t n, cudaStream_t s) {
    uniform_bulk_kernel<<<bulk_grid(n), 256, 0, s>>>(w, u, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- bulk inverse CDF
// Any u in (0, 1): v = min(u, 1-u) is exact in binary32 (1 - u is exact for
// u >= 1/2), the sign comes from u > 1/2.  Each warp takes 64 consecutive
// values per round (two per lane).
template <int P, int ICDF>
__global__ void icdf_bulk_kernel(const float *u, void *z, size_t n, const DevTables *tabs, const MlpWeights *mlpw) {
    __shared__ SmemTable tab;
    __shared__ MlpShared mlp;
    stage_table(tab, tabs);
    if (ICDF == ICDF_MLP) mlp_stage(mlp, mlpw);
    __syncthreads();
    const size_t lane = threadIdx.x & 31;
    const size_t warps = (size_t)gridDim.x * (blockDim.x >> 5);
    for (size_t base = ((size_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 64; base < n;
         base += warps * 64) {
        float r[2];
        float v[2], tt[2];
        uint32_t sg[2];
        size_t idx[2];
        for (int h = 0; h < 2; ++h) {
            idx[h] = base + 2 * lane + h;
            float ui = u[idx[h] < n ? idx[h] : n - 1];
            // TABLE16: centre of the 2^-16 cell that holds u (exact steps)
            if (ICDF == ICDF_TABLE16) ui = __fmul_rn(__fadd_rn(floorf(__fmul_rn(ui, 65536.0f)), 0.5f), 0x1p-16f);
            const bool upper = ui > 0.5f;
            v[h] = upper ? __fsub_rn(1.0f, ui) : ui;
            sg[h] = upper ? 0x80000000u : 0u;
            tt[h] = mlp_feature(v[h]);
        }
        if (ICDF == ICDF_MLP) {
            for (int h = 0; h < 2; ++h) {
                const float y = mlp_eval16(mlp, mlpw->tanh16, tt[h]);
                r[h] = sg[h] ? y : -y;
            }
        }
        for (int h = 0; h < 2; ++h) {
            if (idx[h] >= n) continue;
            if (ICDF == ICDF_EXACT) {
                // the kernels' polynomial on the grid's range, CUDA's normcdfinvf below it
                r[h] = v[h] >= 0x1p-24f ? exact_zv(tab, sg[h], v[h])
                                        : __uint_as_float(__float_as_uint(normcdfinvf(v[h])) ^ sg[h]);
            } else if (ICDF == ICDF_CUBIC) {
                if (P == P_F16) {
                    static_cast<__half *>(z)[idx[h]] = __low2half(cubic_z16<true>(tab, sg[h], sg[h], v[h], v[h]));
                    continue;
                }
                if (P == P_BF16) {
                    static_cast<uint16_t *>(z)[idx[h]] = (uint16_t)cubic_zbf16<true>(tab, sg[h], sg[h], v[h], v[h]);
                    continue;
                }
                r[h] = cubic_z32<true>(tab, sg[h], v[h]);
            } else if (ICDF == ICDF_TABLE || ICDF == ICDF_TABLE16) {
                if (P == P_F16) {
                    const __half2 hz = table_z16<true>(tab, sg[h], sg[h], v[h], v[h]);
                    static_cast<__half *>(z)[idx[h]] = __low2half(hz);
                    continue;
                }
                if (P == P_BF16) {
                    static_cast<uint16_t *>(z)[idx[h]] = (uint16_t)table_zbf16<true>(tab, sg[h], sg[h], v[h], v[h]);
                    continue;
                }
                r[h] = table_z32<true>(tab, sg[h], v[h]);
            }
            if (P == P_F32) static_cast<float *>(z)[idx[h]] = r[h];
            else if (P == P_F16) static_cast<__half *>(z)[idx[h]] = __float2half_rn(r[h]);
            else static_cast<uint16_t *>(z)[idx[h]] = (uint16_t)f32x2_to_bf16x2(r[h], 0.0f);
        }
    }
}

cudaError_t launch_icdf_bulk(const float *u, void *z, size_t n, int icdf, int prec, const DevTables *tabs,
                             const MlpWeights *mlp, cudaStream_t s) {
    const int g = bulk_grid(n);
#define MLMC_ICDF_CASE(PP, II) icdf_bulk_kernel<PP, II><<<g, 256, 0, s>>>(u, z, n, tabs, mlp)
#define MLMC_ICDF_PREC(PP)                                  \
    if (icdf == ICDF_EXACT) MLMC_ICDF_CASE(PP, ICDF_EXACT); \
    else if (icdf == ICDF_TABLE) MLMC_ICDF_CASE(PP, ICDF_TABLE); \
    else if (icdf == ICDF_TABLE16) MLMC_ICDF_CASE(PP, ICDF_TABLE16); \
    else if (icdf == ICDF_CUBIC) MLMC_ICDF_CASE(PP, ICDF_CUBIC); \
    else MLMC_ICDF_CASE(PP, ICDF_MLP)
    if (prec == P_F32) {
        MLMC_ICDF_PREC(P_F32);
    } else if (prec == P_F16) {
        MLMC_ICDF_PREC(P_F16);
    } else {
        MLMC_ICDF_PREC(P_BF16);
    }
#undef MLMC_ICDF_PREC
#undef MLMC_ICDF_CASE
    return cudaGetLastError();
}

}  // namespace mlmc
