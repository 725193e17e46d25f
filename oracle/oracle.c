/*
 * Oracle for nested multilevel Monte Carlo with low-precision approximate
 * random variables (Giles & Sheridan-Methven, "Rounding error using low
 * precision approximate random variables").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * restatement of the method in FP64.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it.  It shares
 * no code with the CUDA library and includes none of its headers.
 *
 * Contents, each following the paper (or, where the paper is silent, the
 * reading stated beside it):
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     SC'11; the paper names no generator).
 *   - 24-bit uniform map u = (2*(w>>9)+1) * 2^-24 (reading: the paper only
 *     says U_n is uniform, Sec. 3).
 *   - Exact inverse Gaussian CDF in FP64 (Sec. 2.1, inverse transform
 *     sampling; Sec. 3 Z_n = Phi^-1(U_n)).
 *   - Piecewise-linear approximate inverse CDF on 16 dyadic intervals,
 *     mirrored (Sec. 2.1, Fig. 1).  The coefficients are an input (built by
 *     oracle/table.py).
 *   - Rounding of every operation to binary16 / binary32 / p-bit mantissa
 *     with round-to-nearest-even (Sec. 2.2 assumes RNE; Sec. 2.2 Fig. 2
 *     varies the mantissa width).
 *   - Euler-Maruyama with the finite-precision operation order
 *     X <- X (+) (A (+) B), A = a (x) delta, B = (b (x) sqrt(delta)) (x) Z
 *     (Sec. 2.2), optionally with Kahan compensated summation (Sec. 2.3,
 *     Algorithm 1).
 *   - Fine/coarse coupling: delta_f = 2^-l T, coarse increments are the
 *     pairwise sums of the fine ones; exact and approximate normals share
 *     the same U_n (Sec. 3).
 *   - Two-way P_l - P_{l-1} and four-way P^_l - P^_{l-1} - P-_l + P-_{l-1}
 *     differences and their sums (Sec. 3, estimators theta^ and theta-).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011): 10 rounds of two 32x32->64      */
/* multiplications with a Weyl-sequence key schedule.                  */
/* ------------------------------------------------------------------ */
static void philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {           /* key schedule: add the Weyl constants */
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod_b;
        uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        philox(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

/* u = (2*(w >> 9) + 1) * 2^-24: 2^23 equiprobable values, symmetric about
 * 1/2, never 0 or 1, exact in binary32 and binary64. */
static double uniform_of(uint32_t w)
{
    return ldexp(2.0 * (double)(w >> 9) + 1.0, -24);
}

void orc_u32_to_uniform(const uint32_t *w, double *u, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) u[i] = uniform_of(w[i]);
}

/* 16-bit uniforms for the approximate normals (a reading, not the paper's:
 * the paper leaves the generator open).  A 16-bit value h gives
 * u = (h + 1/2) 2^-16, the centre of the h-th of 2^16 equal cells of (0, 1).
 * q16(u) maps any u in (0, 1) to the centre of the cell that contains it,
 * so q16 of a 24-bit uniform is distributed exactly like a 16-bit uniform
 * (each cell holds 2^7 of the 2^23 grid points); this keeps the two-way
 * approximate estimator and the four-way bar paths consistent (Sec. 3). */
static double uniform16_of(uint32_t h)
{
    return ldexp((double)h + 0.5, -16);
}

static double q16(double u)
{
    return ldexp(floor(ldexp(u, 16)) + 0.5, -16);
}

void orc_u16_to_uniform(const uint32_t *h, double *u, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) u[i] = uniform16_of(h[i] & 0xFFFFu);
}

void orc_q16(const double *u, double *q, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) q[i] = q16(u[i]);
}

/* ------------------------------------------------------------------ */
/* Exact inverse Gaussian CDF in FP64.                                 */
/* Initial guess: Abramowitz & Stegun 26.2.23 (|error| < 4.5e-4), then */
/* Halley iterations on F(x) = Phi(x) - p.  Near the centre the        */
/* residual is formed with erf (accurate for small x), in the tail     */
/* with erfc.                                                          */
/* ------------------------------------------------------------------ */
static double ndtri_lower(double p)     /* p in (0, 1/2] */
{
    if (p == 0.5) return 0.0;
    double t = sqrt(-2.0 * log(p));
    double x = -(t - (2.515517 + 0.802853 * t + 0.010328 * t * t) /
                     (1.0 + 1.432788 * t + 0.189269 * t * t + 0.001308 * t * t * t));
    const double inv_sqrt2 = 0.70710678118654752440;
    const double inv_sqrt2pi = 0.39894228040143267794;
    for (int it = 0; it < 10; ++it) {
        double r;                       /* r = Phi(x) - p */
        if (p >= 0.25) r = 0.5 * erf(x * inv_sqrt2) - (p - 0.5);
        else r = 0.5 * erfc(-x * inv_sqrt2) - p;
        double dens = inv_sqrt2pi * exp(-0.5 * x * x);
        double e = r / dens;
        double dx = e / (1.0 + 0.5 * x * e);
        x -= dx;
        if (fabs(dx) <= 1e-17 * fabs(x)) break;
    }
    return x;
}

double orc_ndtri1(double p)
{
    if (!(p > 0.0 && p < 1.0)) {
        if (p == 0.0) return -INFINITY;
        if (p == 1.0) return INFINITY;
        return NAN;
    }
    if (p > 0.5) return -ndtri_lower(1.0 - p);
    return ndtri_lower(p);
}

void orc_ndtri(const double *p, double *x, int64_t n)
{
    for (int64_t i = 0; i < n; ++i) x[i] = orc_ndtri1(p[i]);
}

/* ------------------------------------------------------------------ */
/* Rounding to a p-bit significand with minimum normal exponent emin   */
/* (gradual underflow) and overflow to infinity above maxv, round to   */
/* nearest even.  binary16: p=11, emin=-14, maxv=65504.  binary32:      */
/* p=24, emin=-126.  Applied to the exact-or-FP64 result of each +,-,x. */
/* For these operations FP64 has 53 >= 2p+2 bits, so computing in FP64 */
/* and then rounding equals a single correct rounding.                 */
/* ------------------------------------------------------------------ */
typedef struct { int p; int emin; double maxv; int active; } rmode;

static double round_p(double x, const rmode *m)
{
    if (!m->active || x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                       /* |x| in [2^(e-1), 2^e) */
    int q = e - m->p;                   /* exponent of one unit in the last place */
    if (e - 1 < m->emin) q = m->emin - m->p + 1;
    double r = ldexp(nearbyint(ldexp(x, -q)), q);
    if (fabs(r) > m->maxv) r = copysign(INFINITY, x);
    return r;
}

void orc_round_bits(const double *x, double *y, int64_t n, int p, int emin, double maxv)
{
    rmode m = {p, emin, maxv, 1};
    for (int64_t i = 0; i < n; ++i) y[i] = round_p(x[i], &m);
}

/* precision codes shared with oracle/__init__.py */
enum { ORC_F64 = 0, ORC_F32 = 1, ORC_F16 = 2, ORC_BF16 = 3, ORC_PBITS = 4 };

static rmode mode_of(int prec, int pbits)
{
    rmode m = {53, -1022, 1.0e308, 0};
    switch (prec) {
    case ORC_F32: m.p = 24; m.emin = -126; m.maxv = 3.4028234663852886e38; m.active = 1; break;
    case ORC_F16: m.p = 11; m.emin = -14; m.maxv = 65504.0; m.active = 1; break;
    case ORC_BF16: m.p = 8; m.emin = -126; m.maxv = 3.3895313892515355e38; m.active = 1; break;
    case ORC_PBITS: m.p = pbits; m.emin = -1022; m.maxv = 1.0e308; m.active = 1; break;
    default: break;
    }
    return m;
}

/* ------------------------------------------------------------------ */
/* Approximate inverse CDF.                                            */
/* Piecewise linear (Sec. 2.1): on v = min(u, 1-u) in (0, 1/2], interval */
/* k = 1..15 is [2^-(k+1), 2^-k), interval 16 is (0, 2^-16); g(v) =     */
/* c0 + c1 v on each; Phi~^-1(u) = g(v) for u <= 1/2 and -g(v) above.   */
/* table[2i], table[2i+1] = c0, c1 of interval i+1.  Evaluation in      */
/* working precision: z = R(R(c0) + R(R(c1) * R(v))).                   */
/* ------------------------------------------------------------------ */
static int interval_of(double v)
{
    int e;
    frexp(v, &e);                       /* v in [2^(e-1), 2^e) */
    int k = -e;                         /* v in [2^-(k+1), 2^-k) */
    if (k > 16) k = 16;
    if (k < 1) k = 1;                   /* v = 1/2 joins the first interval */
    return k - 1;
}

static double table_icdf(double u, const double *table, const rmode *m)
{
    int upper = u > 0.5;
    double v = upper ? 1.0 - u : u;
    int i = interval_of(v);
    double c0 = round_p(table[2 * i], m);
    double c1 = round_p(table[2 * i + 1], m);
    double z = round_p(c0 + round_p(c1 * round_p(v, m), m), m);
    return upper ? -z : z;
}

/* Piecewise cubic (the high-fidelity approximation of the Sec. 2.2
 * experiments): same intervals and mirroring; on interval k the local
 * variable s = A v - B lies in [-1, 1] (A = 2^(k+2), B = 3 for k <= 15;
 * A = 2^17, B = 1 for k = 16) and g = d0 + d1 s + d2 s^2 + d3 s^3.
 * cubic[4i + j] = d_j of interval i+1.  Working precision: s = R(A v - B)
 * (exact on the uniform grid), then Horner with a rounding after every
 * operation: z = R(d0 + R(s R(d1 + R(s R(d2 + R(s d3)))))). */
static double cubic_icdf(double u, const double *cubic, const rmode *m)
{
    int upper = u > 0.5;
    double v = upper ? 1.0 - u : u;
    int i = interval_of(v);
    double A = i < 15 ? ldexp(1.0, i + 3) : ldexp(1.0, 17);
    double B = i < 15 ? 3.0 : 1.0;
    double s = round_p(v * A - B, m);
    const double *d = cubic + 4 * i;
    double z = round_p(s * round_p(d[3], m), m);
    z = round_p(round_p(d[2], m) + z, m);
    z = round_p(s * z, m);
    z = round_p(round_p(d[1], m) + z, m);
    z = round_p(s * z, m);
    z = round_p(round_p(d[0], m) + z, m);
    return upper ? -z : z;
}

/* MLP surrogate: t = sqrt(-2 ln v), y = W3 tanh(W2 tanh(W1 t + b1) + b2)
 * + b3 approximates |Phi^-1(v)|; Phi~^-1(u) = -y for u <= 1/2, +y above.
 * Weight layout (1153 values): W1[32], b1[32], W2[32][32] (row = output
 * unit), b2[32], W3[32], b3. */
#define MLP_H 32
static double mlp_forward(double t, const double *w)
{
    const double *W1 = w, *b1 = w + 32, *W2 = w + 64, *b2 = w + 64 + 1024;
    const double *W3 = w + 64 + 1024 + 32, *b3 = w + 64 + 1024 + 64;
    double h1[MLP_H], y = b3[0];
    for (int j = 0; j < MLP_H; ++j) h1[j] = tanh(W1[j] * t + b1[j]);
    for (int o = 0; o < MLP_H; ++o) {
        double a = b2[o];
        for (int j = 0; j < MLP_H; ++j) a += W2[o * MLP_H + j] * h1[j];
        y += W3[o] * tanh(a);
    }
    return y;
}

static double mlp_icdf(double u, const double *w)
{
    int upper = u > 0.5;
    double v = upper ? 1.0 - u : u;
    double y = mlp_forward(sqrt(-2.0 * log(v)), w);
    return upper ? y : -y;
}

/* The same network as evaluated in binary16 inference arithmetic (the
 * reading of "FP16 MLP" used by the learned part; every step rounds where
 * the reading says, to nearest even):
 *   t = sqrt(-2 ln v) from binary32 operations: v = m 2^e with m in
 *     [1/sqrt2, sqrt2] (m > R32(sqrt 2) halves m), z = R32((m - 1) / R32(m + 1)),
 *     w = R32(z z), q = 1/9 then q = fma32(q, w, c) for c = 1/7, 1/5, 1/3, 1
 *     (constants R32 of the fractions), ln m = R32(2 z q) -- the atanh series
 *     ln m = 2 atanh z -- and t = R32(sqrt(fma32(-2 e, R32(ln 2), -2 ln m)));
 *   activations: tanh16(x) = R16(tanh(R16(x))), the hyperbolic tangent of
 *     the binary16 value, correctly rounded to binary16;
 *   layer 1: h1_j = tanh16(fma32(W1_j, t, b1_j));
 *   layer 2: c_j = b2_j, then c_j = fma32(R16(W2_ji), h1_i, c_j) for
 *     i = 0, 1, ..., 31 in turn; h2_j = tanh16(c_j);
 *   layer 3: y = b3, then y = fma32(R16(W3_j), h2_j, y) for j = 0, ..., 31.
 * The weights are binary32 values; fma32 is C's fmaf (the exact a b + c
 * rounded once).  tanh16 takes the binary64 tanh (within an ulp of binary64)
 * and rounds it to binary16: correct unless tanh(x) lay within 2^-52 of a
 * binary16 rounding boundary, which no binary16 input comes near (checked
 * against high-precision values for all of them). */
static double r32(double x) { return (double)(float)x; }

static double r16(double x)
{
    rmode m = mode_of(ORC_F16, 0);
    return round_p(x, &m);
}

double orc_tanh16(double x) { return r16(tanh(r16(x))); }

double orc_mlp_feature32(double v)
{
    int e;
    double m = frexp(v, &e);           /* v = m 2^e, m in [1/2, 1) */
    m *= 2.0;
    e -= 1;                            /* m in [1, 2) */
    if (m > (double)(float)1.41421354f) {
        m *= 0.5;
        e += 1;
    }
    double z = r32((m - 1.0) / r32(m + 1.0));
    double w = r32(z * z);
    double q = (double)fmaf((float)(1.0 / 9.0), (float)w, (float)(1.0 / 7.0));
    q = (double)fmaf((float)q, (float)w, (float)(1.0 / 5.0));
    q = (double)fmaf((float)q, (float)w, (float)(1.0 / 3.0));
    q = (double)fmaf((float)q, (float)w, 1.0f);
    double lnm = r32((2.0 * z) * q);
    double t2 = (double)fmaf((float)(-2 * e), (float)log(2.0), (float)(-2.0 * lnm));
    return r32(sqrt(t2));
}

/* The network as the entry points hold it: the weights as given (the FP64
 * network reads them) and a copy with W2 and W3 rounded to binary16 (the
 * binary16 reading), made once per entry-point call. */
#define ORC_MLP_N 1153
typedef struct {
    const double *w;
    double w16[ORC_MLP_N];
} orc_net;

static void net_init(orc_net *n, const double *mlp)
{
    n->w = mlp;
    if (!mlp) return;
    for (int i = 0; i < ORC_MLP_N; ++i) n->w16[i] = mlp[i];
    for (int i = 64; i < 64 + 1024; ++i) n->w16[i] = r16(mlp[i]);                   /* W2 */
    for (int i = 64 + 1024 + 32; i < 64 + 1024 + 64; ++i) n->w16[i] = r16(mlp[i]);  /* W3 */
}

/* w: the network with W2 and W3 already rounded to binary16 (orc_net.w16). */
static double mlp_forward16(double t, const double *w)
{
    const double *W1 = w, *b1 = w + 32, *W2 = w + 64, *b2 = w + 64 + 1024;
    const double *W3 = w + 64 + 1024 + 32, *b3 = w + 64 + 1024 + 64;
    float h1[MLP_H], h2[MLP_H];
    for (int j = 0; j < MLP_H; ++j) h1[j] = (float)orc_tanh16((double)fmaf((float)W1[j], (float)t, (float)b1[j]));
    for (int o = 0; o < MLP_H; ++o) {
        float c = (float)b2[o];
        for (int i = 0; i < MLP_H; ++i) c = fmaf((float)W2[o * MLP_H + i], h1[i], c);
        h2[o] = (float)orc_tanh16((double)c);
    }
    float y = (float)b3[0];
    for (int j = 0; j < MLP_H; ++j) y = fmaf((float)W3[j], h2[j], y);
    return (double)y;
}

static double mlp_icdf16(double u, const double *w)
{
    int upper = u > 0.5;
    double v = upper ? 1.0 - u : u;
    double y = mlp_forward16(orc_mlp_feature32(v), w);
    return upper ? y : -y;
}

/* RV kinds.  TABLE16: the piecewise-linear table at the 16-bit uniform
 * q16(u) (see uniform16_of).  CUBIC: the piecewise cubic.  MLP: the FP64
 * network; MLP16: the network in binary16 inference arithmetic (above).  The
 * `table` argument of the entry points holds the linear table (32 values)
 * followed by the cubic one (64 values). */
enum { ORC_RV_EXACT = 0, ORC_RV_TABLE = 1, ORC_RV_MLP = 2, ORC_RV_TABLE16 = 3, ORC_RV_CUBIC = 4, ORC_RV_MLP16 = 5 };

static double rv_of(double u, int rv, const double *table, const orc_net *net, const rmode *m)
{
    switch (rv) {
    case ORC_RV_TABLE: return table_icdf(u, table, m);
    case ORC_RV_TABLE16: return table_icdf(q16(u), table, m);
    case ORC_RV_CUBIC: return cubic_icdf(u, table + 32, m);
    case ORC_RV_MLP: return round_p(mlp_icdf(u, net->w), m);
    case ORC_RV_MLP16: return round_p(mlp_icdf16(u, net->w16), m);
    default: return round_p(orc_ndtri1(u), m);
    }
}

/* Element by element (OpenMP threads take independent elements). */
void orc_approx_icdf(const double *u, double *z, int64_t n, int rv, int prec, int pbits,
                     const double *table, const double *mlp)
{
    rmode m = mode_of(prec, pbits);
    orc_net net;
    net_init(&net, mlp);
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < n; ++i) z[i] = rv_of(u[i], rv, table, &net, &m);
}

/* ------------------------------------------------------------------ */
/* SDEs and Euler-Maruyama in working precision.                       */
/* ------------------------------------------------------------------ */
enum { ORC_GBM = 0, ORC_OU = 1 };
enum { ORC_PAYOFF_X = 0, ORC_PAYOFF_CALL = 1 };

typedef struct {
    int sde, payoff;
    double p0, p1, p2;      /* GBM: mu, sigma, -;  OU: theta, m, s */
    double x0, T, K, disc;  /* call payoff: disc * max(X_T - K, 0) */
    int scheme;             /* 0: Euler-Maruyama; 1: Milstein (GBM; OU's b' = 0 makes it Euler) */
} orc_sde;

/* Per-level constants of one path, each rounded once to the working
 * precision.  GBM: a(X) delta = (mu delta) X, b(X) sqrt(delta) = (sigma
 * sqrt(delta)) X.  OU: a(X) delta = (theta delta)(m - X), b sqrt(delta) =
 * s sqrt(delta). */
typedef struct {
    rmode m;
    int kahan, sde, milstein;
    double drift, diff, mean;   /* drift: mu*delta or theta*delta; diff: sigma*sqrt(delta_f) or s*sqrt(delta_f) */
    double mil, mconst;         /* Milstein: R(sigma^2 delta_f / 2), and 1 (fine) or 2 (coarse) */
    double X, c;                /* state and Kahan compensation */
} path_state;

/* delta = delta_f (fine path) or 2 delta_f (coarse path, coarse = 1). */
static void path_init(path_state *s, const orc_sde *p, int prec, int pbits, int kahan, double delta, double sqrt_delta_f,
                      int coarse)
{
    s->m = mode_of(prec, pbits);
    s->kahan = kahan;
    s->sde = p->sde;
    s->milstein = p->sde == ORC_GBM && p->scheme == 1;
    s->drift = round_p(p->p0 * delta, &s->m);
    s->diff = round_p(p->p1 * sqrt_delta_f, &s->m);
    s->mean = 0.0;
    if (p->sde == ORC_OU) {
        s->diff = round_p(p->p2 * sqrt_delta_f, &s->m);
        s->mean = round_p(p->p1, &s->m);
    }
    /* the coarse step (delta = 2 delta_f) uses Z1 + Z2 with the fine
     * sqrt(delta_f): (dW_c)^2 - delta_c = delta_f ((Z1 + Z2)^2 - 2) */
    s->mil = round_p(0.5 * p->p1 * p->p1 * (coarse ? 0.5 * delta : delta), &s->m);
    s->mconst = coarse ? 2.0 : 1.0;
    s->X = round_p(p->x0, &s->m);
    s->c = 0.0;
}

/* One step X <- X (+) (A (+) B), or with the Milstein term of GBM
 * X <- X (+) ((A (+) B) (+) M), M = (mil (x) X) (x) ((z (x) z) (-) mconst),
 * i.e. 1/2 b b' ((dW)^2 - delta) with b = sigma X (the scheme the paper
 * names in its conclusions; order of operations a reading).  Kahan
 * (Algorithm 1) on the outer addition if on.  dW is the normal increment
 * multiplier: Z for a fine step, Z1 (+) Z2 for a coarse step (the coarse
 * Wiener increment is the pairwise sum of the two fine ones, Sec. 3). */
static void path_step(path_state *s, double z)
{
    const rmode *m = &s->m;
    double A, B;
    if (s->sde == ORC_GBM) {
        A = round_p(s->drift * s->X, m);
        B = round_p(round_p(s->diff * s->X, m) * z, m);
    } else {
        A = round_p(s->drift * round_p(s->mean - s->X, m), m);
        B = round_p(s->diff * z, m);
    }
    double inc = round_p(A + B, m);
    if (s->milstein) {
        double w = round_p(round_p(z * z, m) - s->mconst, m);
        inc = round_p(inc + round_p(round_p(s->mil * s->X, m) * w, m), m);
    }
    if (s->kahan) {
        double y = round_p(inc - s->c, m);
        double t = round_p(s->X + y, m);
        s->c = round_p(round_p(t - s->X, m) - y, m);
        s->X = t;
    } else {
        s->X = round_p(s->X + inc, m);
    }
}

/* Payoff in FP64 for an FP64 path, in binary32 otherwise. */
static double payoff_of(double X, const orc_sde *p, int prec)
{
    if (p->payoff == ORC_PAYOFF_X) return X;
    if (prec == ORC_F64) {
        double t = X - p->K;
        return p->disc * (t > 0.0 ? t : 0.0);
    }
    rmode f = mode_of(ORC_F32, 0);
    double t = round_p(X - round_p(p->K, &f), &f);
    if (!(t > 0.0)) t = 0.0;
    return round_p(round_p(p->disc, &f) * t, &f);
}

/* Random-number counter layout.  ctr = (path lo32, path hi32, j, tag),
 * key = (seed lo32, seed hi32).  A uniform takes the top 23 bits of a word
 * (uniform_of), so one call (x, y, z, w) carries five: its four words and
 * a fifth word assembled from the low bytes of x, y and z as bits 8..15,
 * 16..23, 24..31 (spare_word: the uniform reads bits 9..31, disjoint from
 * the bits the four words' uniforms read).  Fine step n of a path of
 * 2^l >= 4 steps uses uniform n mod 5 of call j = n / 5 (0..3: the words,
 * 4: the spare).  tag = kind | level << 8 | set << 16 with kind 0: standard
 * two-way with exact normals, 1: two-way with approximate normals, 2:
 * four-way.  (Reading: the paper is silent on the generator.)
 * With 16-bit uniforms (RV TABLE16 on a two-way path) fine step n uses half
 * n mod 2 (low half first) of word (n / 2) mod 4 of call j = n / 8.
 * Coarsest levels, two-way paths: while a path needs fewer words than one
 * call holds (2^l < 4 words, or 2^l < 8 halves with 16-bit uniforms), the
 * S = 4 / 2^l (8 / 2^l) consecutive paths S k .. S k + S - 1 share call 0 of
 * counter path field k, path p taking the words (halves) from
 * (p mod S) 2^l on.  Four-way paths share call 0 of counter path field k
 * in the same way at l = 0 (S = 4: paths 4k .. 4k+3, word p mod 4) and at
 * l = 1 (S = 2: paths 2k, 2k+1, words 2 (p mod 2) and the next). */
static void draw4w(uint64_t path, uint32_t j, uint32_t tag, uint64_t seed, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)path, (uint32_t)(path >> 32), j, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    philox(ctr, key, w);
}

static void draw4(uint64_t path, uint32_t j, uint32_t tag, uint64_t seed, double u[4])
{
    uint32_t w[4];
    draw4w(path, j, tag, seed, w);
    for (int i = 0; i < 4; ++i) u[i] = uniform_of(w[i]);
}

static uint32_t spare_word(const uint32_t w[4])
{
    return ((w[0] & 0xFFu) << 8) | ((w[1] & 0xFFu) << 16) | ((w[2] & 0xFFu) << 24);
}

/* The five uniforms of a call: its four words, then the spare word. */
static void draw5(uint64_t path, uint32_t j, uint32_t tag, uint64_t seed, double u[5])
{
    uint32_t w[4];
    draw4w(path, j, tag, seed, w);
    for (int i = 0; i < 4; ++i) u[i] = uniform_of(w[i]);
    u[4] = uniform_of(spare_word(w));
}

/* The uniform of fine step n of a path of at least 4 steps (calls of its
 * own counter path field, five uniforms each); u holds the current call's. */
static double uniform_at(uint64_t path, int64_t n, uint32_t tag, uint64_t seed, double u[5])
{
    if (n % 5 == 0) draw5(path, (uint32_t)(n / 5), tag, seed, u);
    return u[n % 5];
}

typedef struct { int prec, pbits, kahan, rv; } orc_variant;

/* Two-way sample of level l: out = (P_fine, P_coarse, D); P_coarse = 0 at l = 0. */
static void twoway_one(int l, uint64_t path, const orc_variant *v, const orc_sde *p, uint64_t seed,
                       uint32_t tag, const double *table, const orc_net *net, double out[3])
{
    int64_t nf = (int64_t)1 << l;
    double delta_f = ldexp(p->T, -l);
    double sq = sqrt(delta_f);
    path_state fine, coarse;
    path_init(&fine, p, v->prec, v->pbits, v->kahan, delta_f, sq, 0);
    path_init(&coarse, p, v->prec, v->pbits, v->kahan, 2.0 * delta_f, sq, 1);
    double zprev = 0.0, u[5];
    uint32_t w[4];
    const int u16 = v->rv == ORC_RV_TABLE16;
    const int64_t per_call = u16 ? 8 : 4;                       /* halves or words of one call */
    const uint64_t S = nf < per_call ? (uint64_t)(per_call / nf) : 1;   /* paths sharing a call */
    const uint64_t cpath = path / S;
    const int64_t off = (int64_t)(path % S) * nf;               /* first word (half) of this path */
    for (int64_t n = 0; n < nf; ++n) {
        double z;
        const int64_t q = off + n;
        if (u16) {
            if (n == 0 || (q & 7) == 0) draw4w(cpath, (uint32_t)(q >> 3), tag, seed, w);
            uint32_t word = w[(q >> 1) & 3];
            uint32_t h = (q & 1) ? word >> 16 : word & 0xFFFFu;
            z = table_icdf(uniform16_of(h), table, &fine.m);
        } else if (S > 1) {
            if (n == 0 || (q & 3) == 0) draw4(cpath, (uint32_t)(q >> 2), tag, seed, u);
            z = rv_of(u[q & 3], v->rv, table, net, &fine.m);
        } else {
            z = rv_of(uniform_at(path, n, tag, seed, u), v->rv, table, net, &fine.m);
        }
        path_step(&fine, z);
        if (l > 0 && (n & 1)) path_step(&coarse, round_p(zprev + z, &coarse.m));
        zprev = z;
    }
    double pf = payoff_of(fine.X, p, v->prec);
    double pc = l > 0 ? payoff_of(coarse.X, p, v->prec) : 0.0;
    double d;
    if (l == 0) d = pf;
    else if (v->prec == ORC_F64) d = pf - pc;
    else { rmode f = mode_of(ORC_F32, 0); d = round_p(pf - pc, &f); }
    out[0] = pf; out[1] = pc; out[2] = d;
}

/* Four-way sample: out = (P^_f, P^_c, P-_f, P-_c, D) with
 * D = (P^_f - P^_c) - (P-_f - P-_c); all four paths share U_n (Sec. 3). */
static void fourway_one(int l, uint64_t path, const orc_variant *hat, const orc_variant *bar, const orc_sde *p,
                        uint64_t seed, uint32_t tag, const double *table, const orc_net *net, double out[5])
{
    int64_t nf = (int64_t)1 << l;
    double delta_f = ldexp(p->T, -l);
    double sq = sqrt(delta_f);
    path_state hf, hc, bf, bc;
    path_init(&hf, p, hat->prec, hat->pbits, hat->kahan, delta_f, sq, 0);
    path_init(&hc, p, hat->prec, hat->pbits, hat->kahan, 2.0 * delta_f, sq, 1);
    path_init(&bf, p, bar->prec, bar->pbits, bar->kahan, delta_f, sq, 0);
    path_init(&bc, p, bar->prec, bar->pbits, bar->kahan, 2.0 * delta_f, sq, 1);
    double zh_prev = 0.0, zb_prev = 0.0, u[5];
    const int shared = l <= 1;
    const uint64_t S4 = l == 0 ? 4 : 2;                           /* paths sharing a call, see draw4w */
    const uint64_t cpath = shared ? path / S4 : path;
    const int64_t off = shared ? (int64_t)(path % S4) << l : 0;
    for (int64_t n = 0; n < nf; ++n) {
        const int64_t q = off + n;
        double un;
        if (shared) {
            if (n == 0 || (q & 3) == 0) draw4(cpath, (uint32_t)(q >> 2), tag, seed, u);
            un = u[q & 3];
        } else {
            un = uniform_at(path, n, tag, seed, u);
        }
        double zh = rv_of(un, hat->rv, table, net, &hf.m);
        double zb = rv_of(un, bar->rv, table, net, &bf.m);
        path_step(&hf, zh);
        path_step(&bf, zb);
        if (l > 0 && (n & 1)) {
            path_step(&hc, round_p(zh_prev + zh, &hc.m));
            path_step(&bc, round_p(zb_prev + zb, &bc.m));
        }
        zh_prev = zh; zb_prev = zb;
    }
    double phf = payoff_of(hf.X, p, hat->prec);
    double phc = l > 0 ? payoff_of(hc.X, p, hat->prec) : 0.0;
    double pbf = payoff_of(bf.X, p, bar->prec);
    double pbc = l > 0 ? payoff_of(bc.X, p, bar->prec) : 0.0;
    double d;
    if (hat->prec == ORC_F64 || bar->prec == ORC_F64) {
        d = (phf - phc) - (pbf - pbc);
    } else {
        rmode f = mode_of(ORC_F32, 0);
        d = round_p(round_p(phf - phc, &f) - round_p(pbf - pbc, &f), &f);
    }
    out[0] = phf; out[1] = phc; out[2] = pbf; out[3] = pbc; out[4] = d;
}

static orc_variant variant_of(const int *v) { orc_variant r = {v[0], v[1], v[2], v[3]}; return r; }

/* Per-path outputs for an explicit list of path indices (sampled parity). */
void orc_twoway_paths(int l, const uint64_t *idx, int64_t n, const int *var, const orc_sde *p, uint64_t seed,
                      uint32_t tag, const double *table, const double *mlp, double *out)
{
    orc_variant v = variant_of(var);
    orc_net net;
    net_init(&net, mlp);
    for (int64_t i = 0; i < n; ++i) twoway_one(l, idx[i], &v, p, seed, tag, table, &net, out + 3 * i);
}

void orc_fourway_paths(int l, const uint64_t *idx, int64_t n, const int *hat, const int *bar, const orc_sde *p,
                       uint64_t seed, uint32_t tag, const double *table, const double *mlp, double *out)
{
    orc_variant h = variant_of(hat), b = variant_of(bar);
    orc_net net;
    net_init(&net, mlp);
    for (int64_t i = 0; i < n; ++i) fourway_one(l, idx[i], &h, &b, p, seed, tag, table, &net, out + 5 * i);
}

/* Level sums over paths path_offset .. path_offset + N - 1:
 * sums = (sum D, sum D^2).  four = 0: two-way with variant var; four = 1:
 * four-way with hat var and bar var2.  nthreads > 1 splits the paths
 * across OpenMP threads. */
void orc_level_sums(int l, uint64_t N, uint64_t path_offset, int four, const int *var, const int *var2,
                    const orc_sde *p, uint64_t seed, uint32_t tag, const double *table, const double *mlp,
                    int nthreads, double *sums)
{
    orc_variant v = variant_of(var), v2 = variant_of(four ? var2 : var);
    orc_net net;
    net_init(&net, mlp);
    double s1 = 0.0, s2 = 0.0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for reduction(+ : s1, s2) num_threads(nthreads) schedule(static)
#endif
    for (int64_t i = 0; i < (int64_t)N; ++i) {
        double out[5];
        double d;
        if (four) { fourway_one(l, path_offset + (uint64_t)i, &v, &v2, p, seed, tag, table, &net, out); d = out[4]; }
        else { twoway_one(l, path_offset + (uint64_t)i, &v, p, seed, tag, table, &net, out); d = out[2]; }
        s1 += d;
        s2 += d * d;
    }
    sums[0] = s1;
    sums[1] = s2;
    (void)nthreads;
}

/* Terminal values of the exact (FP64, exact normals) and low-precision
 * paths driven by the same normals Z~ (the same approximate variable in
 * both), for the rounding-error experiments of Sec. 2.2-2.3 (Fig. 2):
 * out[2i] = X in FP64, out[2i+1] = X in the working precision. */
void orc_rounding_pairs(int l, uint64_t N, uint64_t path_offset, const int *var, const orc_sde *p, uint64_t seed,
                        uint32_t tag, const double *table, const double *mlp, double *out)
{
    orc_variant v = variant_of(var);
    orc_net net;
    net_init(&net, mlp);
    int64_t nf = (int64_t)1 << l;
    double delta_f = ldexp(p->T, -l);
    double sq = sqrt(delta_f);
    for (int64_t i = 0; i < (int64_t)N; ++i) {
        path_state hi, lo;
        path_init(&hi, p, ORC_F64, 53, 0, delta_f, sq, 0);
        path_init(&lo, p, v.prec, v.pbits, v.kahan, delta_f, sq, 0);
        double u[5];
        rmode exact = mode_of(ORC_F64, 0);
        const uint64_t path = path_offset + (uint64_t)i;
        const uint64_t S = nf < 4 ? (uint64_t)(4 / nf) : 1;          /* two-way layout, see draw4w */
        const uint64_t cpath = path / S;
        const int64_t off = (int64_t)(path % S) * nf;
        for (int64_t n = 0; n < nf; ++n) {
            const int64_t q = off + n;
            double un;
            if (S > 1) {
                if (n == 0 || (q & 3) == 0) draw4(cpath, (uint32_t)(q >> 2), tag, seed, u);
                un = u[q & 3];
            } else {
                un = uniform_at(path, n, tag, seed, u);
            }
            double z64 = rv_of(un, v.rv, table, &net, &exact);
            path_step(&hi, z64);
            path_step(&lo, round_p(z64, &lo.m));
        }
        out[2 * i] = hi.X;
        out[2 * i + 1] = lo.X;
    }
}

/* Kahan compensated summation of a sequence in working precision
 * (Algorithm 1).  Returns the accumulator a. */
double orc_kahan_sum(const double *x, int64_t n, int prec, int pbits)
{
    rmode m = mode_of(prec, pbits);
    double a = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double y = round_p(round_p(x[i], &m) - c, &m);
        double t = round_p(a + y, &m);
        c = round_p(round_p(t - a, &m) - y, &m);
        a = t;
    }
    return a;
}

int orc_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
