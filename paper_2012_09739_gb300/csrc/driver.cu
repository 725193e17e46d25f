// Adaptive multilevel Monte Carlo to a target RMSE (mlmc_run).
//
// Sec. 3: with V_t and C_t the variance and cost per sample of each estimator
// term t, the cost of reaching mean-square error eps^2 (half of it sampling
// variance) is T = 2 eps^-2 (sum_t sqrt(V_t C_t))^2, reached with
// N_t = ceil(2 eps^-2 sqrt(V_t / C_t) sum_s sqrt(V_s C_s)).  The terms are,
// per level l, the two-way difference (standard estimator theta^), or the
// two-way approximate difference plus the four-way difference (nested
// estimator theta-).  The level count grows until the weak-error estimate
// from the last level means meets eps / sqrt(2) (the standard algorithm the
// paper cites; alpha = weak order).
//
// Each round enqueues every term's new samples on one stream (fresh counter
// ranges: path_offset = samples already taken), then copies all sums to the
// host once.
#include <math.h>
#include <string.h>

#include <chrono>
#include <vector>

#include "api_internal.h"

namespace mlmc {

namespace {

struct Term {
    int l, four, prec, kahan, icdf;
    uint64_t n = 0;              // samples taken
    uint64_t dn = 0;             // samples to add this round
    double s1 = 0.0, s2 = 0.0;
    double cost = 0.0;           // ns per sample (model)
    double var() const { return n > 1 ? fmax((s2 - s1 * s1 / n) / (n - 1), 0.0) : 0.0; }
    double mean() const { return n ? s1 / n : 0.0; }
};

// Device ns per fine path-step of each variant, measured from launches big
// enough to fill the GPU; a launch-size-independent cost model C = 2^l nu.
struct CostModel {
    double ns[2][2][2][3] = {};        // [four][prec][kahan][icdf]
    double ps[2][2][2][3] = {};
    double nu(const Term &t) const {
        const double n = ns[t.four][t.prec][t.kahan][t.icdf], p = ps[t.four][t.prec][t.kahan][t.icdf];
        if (p > 0.0) return n / p;
        // before any large launch: relative weights from the operation counts
        return t.four ? 2.2e-3 : (t.icdf == MLMC_ICDF_EXACT ? 1.7e-3 : 1.2e-3);
    }
    void add(const Term &t, double kernel_ns, double path_steps) {
        if (path_steps < 4194304.0) return;
        ns[t.four][t.prec][t.kahan][t.icdf] += kernel_ns;
        ps[t.four][t.prec][t.kahan][t.icdf] += path_steps;
    }
};

}  // namespace

static mlmc_status run_impl(double eps, const mlmc_sde_params *p, const mlmc_run_opts *o, mlmc_run_result *out) {
    const auto t_start = std::chrono::steady_clock::now();
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    const bool nested = o->estimator == 1;
    if (nested && o->icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");

    cudaStream_t s;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
    const int max_terms = 2 * MLMC_MAX_LEVELS;
    double *sums_dev = nullptr, *sums_host = nullptr;
    std::vector<cudaEvent_t> ev(2 * max_terms, nullptr);
    if ((e = cudaMalloc(&sums_dev, 2 * max_terms * sizeof(double))) != cudaSuccess) st = cuda_fail(e, "cudaMalloc");
    if (!st && (e = cudaMallocHost(&sums_host, 2 * max_terms * sizeof(double))) != cudaSuccess)
        st = cuda_fail(e, "cudaMallocHost");
    for (auto &x : ev)
        if (!st && (e = cudaEventCreate(&x)) != cudaSuccess) st = cuda_fail(e, "cudaEventCreate");
    cudaEvent_t done = nullptr;
    if (!st && (e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess)
        st = cuda_fail(e, "cudaEventCreate");

    std::vector<Term> terms;
    CostModel model;
    auto add_level = [&](int l) {
        if (nested) {
            terms.push_back(Term{l, 0, o->prec, o->kahan ? 1 : 0, o->icdf});
            terms.push_back(Term{l, 1, o->prec, o->kahan ? 1 : 0, o->icdf});
        } else {
            terms.push_back(Term{l, 0, MLMC_F32, o->kahan ? 1 : 0, MLMC_ICDF_EXACT});
        }
        for (size_t i = terms.size() - (nested ? 2 : 1); i < terms.size(); ++i) terms[i].dn = o->n0;
    };
    int L = o->min_levels - 1;
    for (int l = 0; l <= L; ++l) add_level(l);
    const double limit = o->timeout_s > 0 ? o->timeout_s : wait_limit_s();
    const int per_level = nested ? 2 : 1;
    int rounds = 0;
    double path_steps = 0.0;
    bool converged = false;

    while (!st) {
        // ---- enqueue this round's samples, one launch per term with new samples
        bool any = false;
        for (size_t i = 0; i < terms.size() && !st; ++i) {
            Term &t = terms[i];
            if (t.dn == 0) continue;
            any = true;
            st = enqueue_level(*d, t.four, t.l, t.dn, t.prec, t.kahan, t.icdf, p, o->seed, t.n, 0, sums_dev + 2 * i,
                               nullptr, s, ev[2 * i], ev[2 * i + 1]);
        }
        if (st) break;
        if (any) {
            ++rounds;
            if ((e = cudaMemcpyAsync(sums_host, sums_dev, 2 * terms.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                     s)) != cudaSuccess) {
                st = cuda_fail(e, "cudaMemcpyAsync");
                break;
            }
            cudaEventRecord(done, s);
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if ((st = wait_event(done, fmax(limit - el, 0.001)))) break;
            for (size_t i = 0; i < terms.size(); ++i) {
                Term &t = terms[i];
                if (t.dn == 0) continue;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
                const double ps = (double)t.dn * ldexp(1.0, t.l);
                model.add(t, (double)ms * 1e6, ps);
                path_steps += ps;
                t.s1 += sums_host[2 * i];
                t.s2 += sums_host[2 * i + 1];
                t.n += t.dn;
                t.dn = 0;
            }
        }
        // ---- variance and cost estimates; optimal sample counts
        std::vector<double> V(terms.size()), C(terms.size());
        for (size_t i = 0; i < terms.size(); ++i) {
            V[i] = terms[i].var();
            // a level's variance is at least half its predecessor's, decayed
            // at strong rate beta = 1 (guards new levels with few samples)
            if (terms[i].l >= 2) V[i] = fmax(V[i], 0.5 * V[i - per_level] * 0.5);
            C[i] = ldexp(1.0, terms[i].l) * model.nu(terms[i]);
            terms[i].cost = C[i];
        }
        double total = 0.0;
        for (size_t i = 0; i < terms.size(); ++i) total += sqrt(V[i] * C[i]);
        bool need = false;
        for (size_t i = 0; i < terms.size(); ++i) {
            const double Nopt = ceil(2.0 / (eps * eps) * sqrt(V[i] / C[i]) * total);
            const double dn = Nopt - (double)terms[i].n;
            if (dn > 0.01 * (double)terms[i].n) {
                terms[i].dn = (uint64_t)dn;
                need = true;
            }
        }
        if (need) continue;
        // ---- weak-error test on the last three level means
        std::vector<double> Y(L + 1, 0.0);
        for (const Term &t : terms) Y[t.l] += t.mean();
        const double r = pow(2.0, o->alpha);
        double bias = fabs(Y[L]);
        if (L >= 1) bias = fmax(bias, fabs(Y[L - 1]) / r);
        if (L >= 2) bias = fmax(bias, fabs(Y[L - 2]) / (r * r));
        bias /= (r - 1.0);
        if (bias <= eps / sqrt(2.0)) {
            converged = true;
            break;
        }
        if (L >= o->max_level) break;
        ++L;
        add_level(L);
    }

    if (!st) {
        memset(out, 0, sizeof *out);
        double est = 0.0, var = 0.0;
        for (const Term &t : terms) {
            const int k = nested ? t.four : 0;
            out->n[k][t.l] = t.n;
            out->mean[k][t.l] = t.mean();
            out->var[k][t.l] = t.var();
            out->cost[k][t.l] = t.cost;
            est += t.mean();
            if (t.n) var += t.var() / t.n;
        }
        out->estimate = est;
        out->variance = var;
        out->levels = L + 1;
        out->rounds = rounds;
        out->path_steps = path_steps;
        out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (!converged) st = fail(MLMC_ENOTCONV, "bias test not met at max_level %d", o->max_level);
    }
    for (auto &x : ev)
        if (x) cudaEventDestroy(x);
    if (done) cudaEventDestroy(done);
    if (sums_dev) cudaFree(sums_dev);
    if (sums_host) cudaFreeHost(sums_host);
    cudaStreamDestroy(s);
    return st;
}

}  // namespace mlmc

using namespace mlmc;

extern "C" mlmc_status mlmc_run(double eps, const mlmc_sde_params *params, const mlmc_run_opts *opts,
                                mlmc_run_result *out) {
    if (!(eps > 0.0) || !isfinite(eps)) return fail(MLMC_EINVAL, "eps must be > 0");
    if (!opts || !out) return fail(MLMC_EINVAL, "NULL argument");
    mlmc_status st = check_params(params);
    if (st) return st;
    if (opts->estimator != 0 && opts->estimator != 1) return fail(MLMC_EINVAL, "estimator must be 0 or 1");
    if (opts->max_level < 2 || opts->max_level > 18) return fail(MLMC_EINVAL, "max_level must be in 2..18");
    if (opts->min_levels < 3 || opts->min_levels > opts->max_level + 1)
        return fail(MLMC_EINVAL, "min_levels must be in 3..max_level+1");
    if (opts->n0 < 2) return fail(MLMC_EINVAL, "n0 must be >= 2");
    if (!(opts->alpha > 0.0)) return fail(MLMC_EINVAL, "alpha must be > 0");
    if (opts->estimator == 1) {
        if (opts->prec != MLMC_F32 && opts->prec != MLMC_F16) return fail(MLMC_EINVAL, "unknown precision");
        if (opts->icdf != MLMC_ICDF_TABLE && opts->icdf != MLMC_ICDF_MLP)
            return fail(MLMC_EINVAL, "nested estimator needs approximate normals");
    }
    return run_impl(eps, params, opts, out);
}
