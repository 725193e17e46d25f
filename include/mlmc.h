/*
 * mlmc.h -- C ABI of the GB300 (sm_103a) library for nested multilevel Monte
 * Carlo with low-precision approximate random variables, after Giles &
 * Sheridan-Methven, "Rounding error using low precision approximate random
 * variables" (arXiv 2012.09739).
 *
 * Conventions shared by every entry point
 *   - Pointers named *_dev are CUDA device pointers on the current device;
 *     pointers named *_host are ordinary host memory.  All memory passed in
 *     belongs to the caller; the library never frees it.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that return results in host memory synchronise with `stream` before
 *     returning; calls with device outputs only enqueue work.
 *   - Every call returns an mlmc_status and never aborts.  Invalid arguments
 *     give MLMC_EINVAL before anything is launched.  A CUDA error gives
 *     MLMC_ECUDA; mlmc_last_error() describes it.
 *   - Results are a deterministic function of (seed, path_offset, N, level,
 *     estimator kind, variant, set id): the sums are accumulated per chunk
 *     group of 32-pair chunks, a split that depends on (l, N) only, and the
 *     level and batch entry points give the same sums for the same item.
 *     Only a level call of more than 2^22 chunk groups keeps one partial per
 *     block instead, and then depends on the grid as well.
 *
 * Random numbers.  Philox4x32-10 (Salmon et al., SC'11; the paper names no
 * generator).  Counter (path lo32, path hi32, j, tag), key (seed lo32, seed
 * hi32); tag = kind | level << 8 | set << 16 with kind 0 = standard two-way
 * with exact normals, 1 = two-way with approximate normals, 2 = four-way.  A
 * word w becomes the uniform u = (2 (w >> 9) + 1) 2^-24 (Sec. 3: Z_n =
 * Phi^-1(U_n) and Z~_n = Phi~^-1(U_n) share U_n).  As a uniform reads only a
 * word's top 23 bits, a call (x, y, z, w) gives five: its four words, then
 * the spare word whose bits 8..15, 16..23, 24..31 are the low bytes of x, y
 * and z.  Fine step n of a path of 2^l >= 4 steps uses uniform n mod 5 of
 * call j = n / 5 (0..3 the words, 4 the spare).  Coarsest levels: a two-way path of
 * level l needs 2^l words (halves with TABLE16); while that is fewer than a
 * call holds (4 words, 8 halves), the S = 4 / 2^l (8 / 2^l) paths S k ..
 * S k + S - 1 share call 0 of counter path field k, path p taking the words
 * (halves) from (p mod S) 2^l on; four-way paths share a call in fours at
 * l = 0 (S = 4) and in pairs at l = 1 (S = 2), both paths of a sample
 * reading its words.  A launch whose path_offset is a multiple of S computes
 * one call per S paths, otherwise two.
 */
#ifndef MLMC_H
#define MLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MLMC_OK = 0,
    MLMC_EINVAL = 1,      /* invalid argument; nothing launched */
    MLMC_ECUDA = 2,       /* CUDA runtime error (see mlmc_last_error) */
    MLMC_ETIMEOUT = 3,    /* wait exceeded the library's wall-clock limit */
    MLMC_ENOMEM = 4,      /* device or host allocation failed */
    MLMC_ENOTCONV = 5,    /* mlmc_run reached max_level without meeting eps */
    MLMC_ENOTREADY = 6    /* MLP weights requested but never set or trained */
} mlmc_status;

typedef enum { MLMC_GBM = 0, MLMC_OU = 1 } mlmc_sde_kind;
typedef enum { MLMC_PAYOFF_X = 0, MLMC_PAYOFF_CALL = 1 } mlmc_payoff;
/* working precision of the approximate ("bar") paths and of Z~: IEEE
 * binary32, IEEE binary16 (10 stored significand bits), or bfloat16 (7
 * stored significand bits, binary32's exponent range; Sec. 4.1 and 5.1
 * compare it with binary16 through the rounding model).  All arithmetic on
 * the bar paths rounds to nearest-even in that format after every
 * operation. */
typedef enum { MLMC_F32 = 0, MLMC_F16 = 1, MLMC_BF16 = 2 } mlmc_prec;
/* How the normals of the approximate paths are formed from the Philox words
 * (counter (path lo32, path hi32, j, tag), key = seed; 24-bit uniform
 * u = (2 (w >> 9) + 1) 2^-24 from a word w; five uniforms per call, as
 * above):
 *   EXACT    Phi^-1(u) in FP32 (no approximation beyond binary32: on each
 *            binade of v = min(u, 1-u) a degree-7 polynomial of the
 *            binade's local variable times (v - 1/2), built on the device
 *            from FP64 values; within 2.5 ulp of Phi^-1 on the 24-bit grid);
 *   TABLE    the 16-interval piecewise-linear Phi~^-1 of Sec. 2.1 at u;
 *   MLP      the network of mlmc_mlp_set_weights / mlmc_mlp_train at u;
 *   TABLE16  the same table at a 16-bit uniform u16 = (h + 1/2) 2^-16, a
 *            design choice of this library (the paper leaves the generator
 *            open).  On two-way paths each word gives two: fine step n uses
 *            half n mod 2 (low half first) of word (n / 2) mod 4 of call
 *            j = n / 8, halving the generator's work.  On four-way bar paths
 *            h = w >> 16, the 2^-16 cell of the hat path's 24-bit u, so both
 *            estimators see the same law of Z~ and the telescoping sum of
 *            Sec. 3 keeps its expectation.
 *   CUBIC    the piecewise cubic at u: the L2 cubic fit of Phi^-1 on the
 *            same 16 intervals (the high-fidelity approximation of the
 *            Sec. 2.2 experiments), g = d0 + d1 s + d2 s^2 + d3 s^3 in the
 *            interval's variable s = A v - B in [-1, 1] (A = 2^(k+2), B = 3
 *            on interval k <= 15; A = 2^17, B = 1 on interval 16), evaluated
 *            by Horner in the working precision with every operation
 *            rounded. */
typedef enum {
    MLMC_ICDF_EXACT = 0,
    MLMC_ICDF_TABLE = 1,
    MLMC_ICDF_MLP = 2,
    MLMC_ICDF_TABLE16 = 3,
    MLMC_ICDF_CUBIC = 4
} mlmc_icdf;

/* Time-stepping scheme.  EULER: Euler-Maruyama.  MILSTEIN: adds the term
 * b b' ((dW)^2 - delta) / 2 (the scheme of order 1 strong convergence the
 * paper's conclusions name); for GBM each fine step adds
 * (mil (x) X) (x) ((Z (x) Z) (-) 1) with mil = R(sigma^2 delta_f / 2), the
 * coarse step (mil (x) X) (x) ((Zc (x) Zc) (-) 2) with Zc = Z1 (+) Z2, added
 * after A (+) B: X <- X (+) ((A (+) B) (+) M).  For OU b' = 0 and the two
 * schemes coincide. */
typedef enum { MLMC_EULER = 0, MLMC_MILSTEIN = 1 } mlmc_scheme;

/* SDE dX = a(X) dt + b(X) dW on [0, T], X_0 = x0.
 *   GBM: a = p0 X, b = p1 X            (mu = p0, sigma = p1)
 *   OU:  a = p0 (p1 - X), b = p2       (theta = p0, m = p1, s = p2)
 * Payoff P = X_T, or disc * max(X_T - K, 0) for the call. */
typedef struct {
    int32_t sde;      /* mlmc_sde_kind */
    int32_t payoff;   /* mlmc_payoff */
    double p0, p1, p2;
    double x0, T, K, disc;
    int32_t scheme;   /* mlmc_scheme */
    int32_t reserved; /* must be 0 */
} mlmc_sde_params;

/* Sums of one level estimator: s1 = sum D, s2 = sum D^2 over n samples
 * (accumulated in FP32 per thread and warp, in FP64 across warps and
 * blocks); cost_ns = device time of the level kernel in nanoseconds; mean
 * and var = the sample mean and the unbiased sample variance of D, combined
 * from (s1, s2, n) by mlmc_moments (FP64). */
typedef struct {
    double s1, s2;
    uint64_t n;
    double cost_ns;
    double mean, var;
} mlmc_sums;

/* Level mean and variance from the sums of n samples (Sec. 3: the estimator
 * of a level is the sample mean of its differences, and its variance enters
 * the sample split through V_l / N_l):
 *   mean = s1 / n,   var = (s2 - s1 * mean) / (n - 1)   (var = 0 for n = 1),
 * in FP64, clamped below at 0 (s2 - s1^2 / n cancels when the mean dominates
 * the spread; the FP64 sums keep the relative error near 1e-16 * s2 / var).
 * sums_host = {s1, s2} as two doubles (the layout the *_async calls write).
 * n = 0 or a NULL pointer gives MLMC_EINVAL.  Host-only; no GPU needed.  Every
 * entry point that fills an mlmc_sums, and the adaptive driver, combine with
 * this routine. */
mlmc_status mlmc_moments(const double *sums_host, uint64_t n, double *mean_host, double *var_host);

/* Two-way level difference D = P_l - P_{l-1} (P_{-1} = 0) over N samples,
 * paths path_offset .. path_offset + N - 1 (Sec. 3, estimator theta^ with
 * icdf = EXACT, first sum of theta- otherwise).
 *   fine: 2^l Euler steps of delta = T 2^-l; coarse: 2^(l-1) steps of 2 delta
 *   driven by the pairwise sums of the fine normals (Sec. 3).
 *   Each Euler step is X <- X (+) (A (+) B), A = (a delta) X-term,
 *   B = ((b sqrt(delta)) X-term) (x) Z in working precision `prec`, every
 *   operation rounded to nearest even and never fused (Sec. 2.2); with
 *   kahan != 0 the addition is Kahan-compensated (Sec. 2.3, Algorithm 1).
 *   The normals are Phi^-1 (icdf EXACT, computed in FP32) or the
 *   approximate inverse CDF (TABLE: 16-interval piecewise linear, Sec. 2.1;
 *   MLP: the network set by mlmc_mlp_set_weights / mlmc_mlp_train).
 * 0 <= l <= 18, N >= 1, T > 0; GBM sigma > 0; OU s > 0.
 * out_host receives the sums; the call synchronises with `stream`. */
mlmc_status mlmc_level(int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *params,
                       uint64_t seed, uint64_t path_offset, mlmc_sums *out_host, void *stream);

/* Four-way nested difference D = P^_l - P^_{l-1} - P-_l + P-_{l-1} (Sec. 3,
 * second sum of theta-).  The "hat" pair uses exact normals Phi^-1(U_n) in
 * FP32 with Kahan compensation; the "bar" pair uses the approximate normals
 * Phi~^-1(U_n) of kind `icdf` (TABLE or MLP) in precision `prec`, with Kahan
 * if kahan != 0.  All four paths share U_n.  Same arguments and errors as
 * mlmc_level; icdf = EXACT is invalid. */
mlmc_status mlmc_nested_level(int l, uint64_t N, int prec, int kahan, int icdf, const mlmc_sde_params *params,
                              uint64_t seed, uint64_t path_offset, mlmc_sums *out_host, void *stream);

/* As mlmc_level / mlmc_nested_level (four = 0 / 1) but asynchronous: writes
 * {s1, s2} as two doubles to sums_dev and nothing to the host.  Launches
 * two kernels (level, finalize) on `stream`. */
mlmc_status mlmc_level_async(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                             const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset,
                             double *sums_dev, void *stream);

/* Allocation-free variant of mlmc_level_async (no counterpart in the paper:
 * it exists for callers that cannot allocate device memory when they ask for
 * an estimate -- e.g. a service that hands all of HBM to its own allocator at
 * start-up, or a latency-critical loop where an allocation could synchronise
 * the device or fail).  It calls no cudaMalloc, cudaFree or other allocating
 * routine: its scratch (one FP64 pair per block of 256 threads, one sample
 * pair per thread) is a fixed 64 KiB file-scope device array, held by every
 * GPU that loads the library until the process exits, and it uses a private
 * copy of the table in the same way.
 *   - N <= 2,097,152 (the scratch holds 4096 blocks); larger N, or
 *     icdf = MLP, gives MLMC_EINVAL with a message.
 *   - The first call on a device does the set-up (builds the private table
 *     on `stream` and waits for it); make that first call before any stream
 *     capture.  Every call looks the arrays' device addresses up again and
 *     repeats the set-up if they moved (the module was loaded anew, e.g.
 *     after a reset of the device's primary context).
 *   - All calls share the one scratch array, which keeps the last call's
 *     contents: calls that overlap on the GPU (e.g. on different streams
 *     without ordering) race and give wrong sums.
 * Writes {sum D, sum D^2} to sums_dev; same arguments as mlmc_level_async. */
mlmc_status mlmc_level_noalloc(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                               const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset,
                               double *sums_dev, void *stream);

/* Per-path diagnostics of the same computation: writes, for sample i,
 * out_dev[i*3 + {0,1,2}] = (P_fine, P_coarse, D) for the two-way difference
 * (four = 0) or out_dev[i*5 + {0..4}] = (P^_f, P^_c, P-_f, P-_c, D) for the
 * four-way difference (four = 1), as float.  Enqueued on `stream`. */
mlmc_status mlmc_level_paths(int four, int l, uint64_t N, int prec, int kahan, int icdf,
                             const mlmc_sde_params *params, uint64_t seed, uint64_t path_offset,
                             float *out_dev, void *stream);

/* Bulk approximate inverse CDF (Sec. 2.1): z_dev[i] = Phi~^-1(u_dev[i]) for
 * 0 < u < 1 (values outside give unspecified finite results); TABLE16
 * evaluates the table at the centre of the 2^-16 cell that holds u.  For
 * CUBIC in binary16 / bfloat16 the local variable s is rounded to binary32
 * first (exact for u on the 24-bit grid).  z_dev is
 * float for prec = F32, IEEE binary16 (uint16_t storage) for F16 and
 * bfloat16 (uint16_t storage, the upper half of a binary32) for BF16.
 * icdf = EXACT evaluates Phi^-1 in FP32 (the kernels' polynomial for
 * v >= 2^-24, CUDA's normcdfinvf below). */
mlmc_status approx_icdf(const float *u_dev, void *z_dev, size_t n, int icdf, int prec, void *stream);

/* Philox4x32-10 of n counters: ctr_dev (n x 4 uint32), key_dev (n x 2),
 * out_dev (n x 4).  And the uniform map u = (2 (w >> 9) + 1) 2^-24. */
mlmc_status mlmc_philox4x32_10(const uint32_t *ctr_dev, const uint32_t *key_dev, uint32_t *out_dev, size_t n,
                               void *stream);
mlmc_status mlmc_uniforms(const uint32_t *w_dev, float *u_dev, size_t n, void *stream);

/* The piecewise-linear table as built on the device (FP64 closed-form L2
 * fit of Phi^-1 on the 16 dyadic intervals of v = min(u, 1-u), Sec. 2.1):
 * c_host[2i], c_host[2i+1] = (c0, c1) of interval i+1.  Any pointer may be
 * NULL.  c32_host / c16_host / cbf16_host receive the binary32 / binary16 /
 * bfloat16 roundings (round to nearest-even from the FP64 value), in the
 * same (c0, c1) order. */
mlmc_status mlmc_icdf_table(double *c_host, float *c32_host, uint16_t *c16_host, uint16_t *cbf16_host);

/* The piecewise cubic as built on the device (FP64 Legendre projection by
 * Gauss-Legendre quadrature): d_host[4i + j] = d_j of interval i+1, and its
 * binary32 / binary16 / bfloat16 roundings in the same order.  Any pointer
 * may be NULL. */
mlmc_status mlmc_icdf_cubic(double *d_host, float *d32_host, uint16_t *d16_host, uint16_t *dbf16_host);

/* ---- MLP surrogate inverse CDF: 1 -> 32 -> 32 -> 1 tanh network on
 * t = sqrt(-2 ln v), v = min(u, 1-u); Z~ = -y for u <= 1/2, +y above.
 * 1153 parameters, layout W1[32], b1[32], W2[32][32] (row = output unit),
 * b2[32], W3[32], b3.  The library keeps one FP32 master copy per device.
 * Inference (approx_icdf with MLMC_ICDF_MLP, and the level kernels through
 * the grid table below) is in binary16 inference arithmetic, every
 * operation rounded once to nearest even: t from binary32 operations (the
 * input map of mlmc_mlp_grad); each activation tanh16(x) = the tanh of x
 * rounded to binary16, correctly rounded to binary16; h1_j =
 * tanh16(fma(W1_j, t, b1_j)); W2 and W3 rounded to binary16; c_o = b2_o,
 * then c_o = fma(W2_oi, h1_i, c_o) for i = 0 .. 31 in turn (binary32),
 * h2_o = tanh16(c_o); y = b3, then y = fma(W3_o, h2_o, y) for o = 0 .. 31.
 * The result is defined bit for bit by these steps. */
#define MLMC_MLP_PARAMS 1153
mlmc_status mlmc_mlp_set_weights(const float *w_host, size_t n);
mlmc_status mlmc_mlp_get_weights(float *w_host, size_t n);

/* The network tabulated on the 24-bit uniform grid (a design of this
 * library; the network itself is not the paper's): the input v = min(u, 1-u)
 * takes the 2^22 values v_k = (2k + 1) 2^-24, and whenever the weights are
 * set or trained the library evaluates the network on all of them (the
 * inference above) into a 16 MiB device table.  The level and batch kernels
 * take Z~ = -y_k for u <= 1/2, +y_k above from that table: the same value
 * the inference gives for the sample.  y_host receives the 2^22 values y_k
 * in k order (n must be 2^22); MLMC_ENOTREADY before weights are set.
 * approx_icdf with MLP evaluates the network directly (any u). */
#define MLMC_MLP_GRID (1u << 22)
mlmc_status mlmc_mlp_grid_table(float *y_host, size_t n);

typedef struct {
    uint64_t steps;       /* Adam steps */
    uint32_t batch;       /* samples per step (multiple of 128) */
    float lr0, lr_min;    /* cosine schedule from lr0 to lr_min */
    float beta1, beta2, eps;
    uint64_t seed;        /* minibatch sampling */
} mlmc_train_opts;

/* Loss and gradient of the mean squared error over n pairs (t = features of
 * u_dev, target z_dev = |Phi^-1(v)|) with the current weights: grad_dev
 * receives 1153 floats, *loss_host the loss.  FP16 tensor-core forward and
 * backward with FP32 accumulation. */
mlmc_status mlmc_mlp_grad(const float *u_dev, const float *z_dev, size_t n, float *grad_dev, float *loss_host,
                          void *stream);
/* Adam training on n (u, |Phi^-1(min(u,1-u))|) pairs.  If z_dev is NULL the
 * targets are computed on the device with FP64 Phi^-1.  The final loss
 * (over the last minibatch) goes to *loss_host if non-NULL. */
mlmc_status mlmc_mlp_train(const float *u_dev, const float *z_dev, size_t n, const mlmc_train_opts *opts,
                           float *loss_host, void *stream);

/* ---- Batched levels: many (parameter set, level, estimator) items in one
 * persistent launch.  kind: 0 two-way, 1 four-way. */
typedef struct {
    mlmc_sde_params params;
    int32_t l, kind, prec, kahan, icdf, set_id;
    uint64_t N, path_offset;
} mlmc_work;

/* Runs all items, tiles by length (longest first or interleaved long and
 * short, tuned with the tile size): one persistent kernel per group of items
 * that share estimator, working precision, Kahan flag, inverse CDF and SDE
 * scheme (the same per-sample code as the level kernels), then one finalize
 * kernel, all captured in a CUDA graph.  out_host[i] receives the sums of
 * items[i]; the call waits for them.  The library keeps the graphs of up to 8
 * item-list shapes (the level, kind, prec, kahan, icdf, N, SDE type and
 * scheme of every item, and the seed), least recently used evicted; the first
 * call with a shape tunes the tile size, block shape and tile order, captures
 * and instantiates (hundreds of ms).  A call with a known shape and seed but
 * other parameter values, payoffs, set ids or path offsets uploads n_items *
 * mlmc_batch_descriptor_bytes() bytes of descriptors and replays the graph; a
 * new seed captures a new graph (the tuned choice is kept).  An item's sums
 * are accumulated as the level kernels do (FP32 Kahan per lane over each
 * chunk group of 32-pair chunks, a warp sum, FP64 partials, the same
 * fixed-order finalize): they equal those of mlmc_level / mlmc_nested_level /
 * mlmc_level_async for the same item, seed and offset bit for bit whenever
 * that call keeps one partial per chunk group (at most 2^22 groups), whatever
 * tile size and order the tuner picks.  Errors: MLMC_EINVAL for an invalid
 * item or a batch beyond 2^32 - 1 tiles or partials (before any launch),
 * MLMC_ENOTREADY for MLP items without weights, MLMC_ECUDA, MLMC_ETIMEOUT. */
mlmc_status mlmc_batch(const mlmc_work *items, int n_items, uint64_t seed, mlmc_sums *out_host, void *stream);

/* mlmc_batch without the wait: enqueues the batch on `stream` and returns.
 * sums_dev (caller-owned device or pinned host memory, 2 * n_items doubles)
 * receives (sum D, sum D^2) of every item when the stream reaches that
 * point.  Launches of the same shape on different streams are ordered by the
 * library (each waits for the previous one on the device).  Same errors as
 * mlmc_batch, plus MLMC_EINVAL for a NULL sums_dev. */
mlmc_status mlmc_batch_async(const mlmc_work *items, int n_items, uint64_t seed, double *sums_dev, void *stream);

/* Bytes of device descriptors uploaded per item when a batch of a known
 * shape is re-staged. */
size_t mlmc_batch_descriptor_bytes(void);

/* ---- Adaptive MLMC to a target RMSE (Sec. 3 cost model). */

/* One draw of mlmc_run: dn new samples (paths path_offset .. path_offset +
 * dn - 1) of one estimator term, with their sums.  kind 0: two-way, 1:
 * four-way; kept = 0 for a per-level candidate that was measured and then
 * discarded (prec = -1), 1 for a term of the estimate; cost_ns = the cost
 * model's device time per sample of the term (the C_t of Sec. 3). */
typedef struct {
    int32_t round, l, kind, prec, kahan, icdf, kept, reserved;
    uint64_t dn, path_offset;
    double s1, s2, cost_ns;
} mlmc_round_record;

typedef struct {
    int32_t estimator;    /* 0: standard theta^ (FP32, exact normals, plain Euler);
                             1: nested theta- (two-way approximate + four-way) */
    int32_t prec, kahan, icdf;   /* variant of the approximate paths (estimator 1); prec = -1:
                                    choose per level, by the smallest sqrt(v c) + sqrt(V C) measured
                                    on n0 warm-up samples of each (Sec. 3), among the nested pairs in
                                    FP16 + Kahan, FP16 and FP32 (kahan ignored) and the standard FP32
                                    exact-normal two-way difference alone (FP32 + Kahan, the hat
                                    paths' arithmetic, so the level differences still telescope) */
    int32_t max_level;    /* <= 18 */
    int32_t min_levels;   /* levels 0 .. min_levels-1 always present (>= 3) */
    uint64_t n0;          /* warm-up samples per level and estimator */
    uint64_t seed;
    double alpha;         /* weak order used in the bias test (Euler: 1) */
    double timeout_s;     /* wall-clock limit; MLMC_ETIMEOUT beyond it */
    /* prec = -1: 0 = measure the candidates on each new level until two
     * consecutive levels have chosen the same FP32 variant (nested FP32 or
     * the standard term), then give finer levels that variant without
     * candidate samples; 1 = measure every candidate on every level (the
     * full per-level efficiency map, at the cost of the discarded samples).
     * The candidates of the min_levels initial levels share one round. */
    int32_t trial_all;
    int32_t trace_cap;    /* capacity of trace (records); 0: no trace */
    mlmc_round_record *trace;   /* optional caller-owned host array: every draw of the run, in order */
} mlmc_run_opts;

#define MLMC_MAX_LEVELS 19
typedef struct {
    double estimate;              /* sum over levels and estimators of the means */
    double variance;              /* sum of V_l / N_l (estimated MSE minus bias^2) */
    int32_t levels;               /* L + 1 */
    int32_t rounds;
    double wall_s;                /* wall-clock time of mlmc_run */
    double path_steps;            /* fine path-steps simulated */
    uint64_t n[2][MLMC_MAX_LEVELS];       /* samples per estimator (0: two-way, 1: four-way) and level */
    double mean[2][MLMC_MAX_LEVELS];
    double var[2][MLMC_MAX_LEVELS];
    double cost[2][MLMC_MAX_LEVELS];      /* device ns per sample */
    int32_t prec[MLMC_MAX_LEVELS];        /* variant used per level (nested estimator) */
    int32_t kahan[MLMC_MAX_LEVELS];
    /* Sec. 3 per-level efficiency of the nested estimator against the standard
     * one: (v c / v^ c^) (1 + sqrt(V C / (v c)))^2 with v^, c^ of the FP32
     * exact-normal two-way difference measured on n0 samples (< 1: saving);
     * 0 when not measured (estimator 0, or levels added without warm-up). */
    double efficiency[MLMC_MAX_LEVELS];
    /* 1: the level uses the nested pair (two-way approximate + four-way);
     * 0: the standard FP32 exact-normal two-way difference alone (estimator
     * 0, or prec = -1 when that is cheaper for the level). */
    int32_t nested[MLMC_MAX_LEVELS];
    int32_t trace_len;            /* draws of the run (records written: min(trace_len, trace_cap)) */
    int32_t reserved;
    double model_s;               /* the cost model's device time of every sample drawn, sum of dn C_t */
    double device_s;              /* measured device time of the rounds (CUDA events around each round) */
    double discarded_path_steps;  /* path-steps of discarded per-level candidates */
} mlmc_run_result;

mlmc_status mlmc_run(double eps, const mlmc_sde_params *params, const mlmc_run_opts *opts, mlmc_run_result *out);

/* Optimal sample counts (Sec. 3): N_i = ceil(2 eps^-2 sqrt(V_i / C_i)
 * sum_j sqrt(V_j C_j)) over n estimator terms.  Host-only; no GPU needed. */
mlmc_status mlmc_optimal_samples(const double *V, const double *C, int n, double eps, uint64_t *N_out);

/* ---- Measurement: peak issue-rate probes of the non-tensor pipes.
 * kind 0: FP32 FFMA, 1: FP16x2 HFMA2, 2: 32-bit IMAD, 3: LOP3.  Writes
 * the measured thread-operations per second (one FMA = one operation, one
 * HFMA2 = two). */
mlmc_status mlmc_peak_probe(int kind, double *ops_per_s, void *stream);

/* Library info and lifetime. */
const char *mlmc_strerror(mlmc_status s);
const char *mlmc_last_error(void);
const char *mlmc_version(void);
/* Frees the library's per-device state (tables, weights, captured batch
 * graphs and their buffers, the adaptive driver's round buffers), after
 * waiting for the batch launches still in flight.  No other call may run
 * concurrently; a later call re-creates the state (tables rebuilt, MLP
 * weights to be set again). */
mlmc_status mlmc_shutdown(void);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_H */
