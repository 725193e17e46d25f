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
// Each round runs every term's new samples (fresh counter ranges:
// path_offset = samples already taken) as the items of one persistent batched
// launch, then copies all sums to the host once.  The allocation uses a cost
// model of measured device time per sample of each term (kCost below); only
// the ratios between terms matter to the split.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <vector>

#include "api_internal.h"

namespace mlmc {

namespace {

struct Term {
    int l, four, prec, kahan, icdf;
    bool off = false;            // placeholder four-way slot of a level run by the standard estimator
    uint64_t n = 0;              // samples taken
    uint64_t dn = 0;             // samples to add this round
    double s1 = 0.0, s2 = 0.0;
    double cost = 0.0;           // ns per sample (model)
    double var() const {
        double m = 0.0, v = 0.0;
        if (n) level_moments(s1, s2, n, &m, &v);
        return v;
    }
    double mean() const {
        double m = 0.0, v = 0.0;
        if (n) level_moments(s1, s2, n, &m, &v);
        return m;
    }
};

// Per-level choice of the nested estimator with prec = -1 (Sec. 3, Fig. 4).
enum Choice { CH_F16K = 0, CH_F16 = 1, CH_F32 = 2, CH_STANDARD = 3, CH_NONE = 4 };

// Sample counts are drawn in multiples of 8, so that every term's path
// offset is a multiple of the 4 or 8 paths that share one Philox call at the
// coarsest two-way levels.
uint64_t round8(uint64_t n) { return (n + 7) / 8 * 8; }

// Cost model C_t of Sec. 3: device time per sample of each estimator term,
// measured on GB300 as single-item batched launches at full occupancy
// (GBM call, N = max(2^27 >> (l - 1), 2^21) samples, best of three, L2
// warm), in picoseconds per sample for levels 0..10; finer levels scale the
// level-10 cost by 2^(l - 10).  Only the ratios between terms enter the
// sample split and the per-level choice.
struct CostRow {
    int four, prec, kahan, icdf, milstein;
    float ps[11];
};
const CostRow kCost[] = {
    {0, MLMC_F32, 0, MLMC_ICDF_EXACT, 0, {2.9, 4.893, 7.367, 13.34, 25.47, 47.57, 91.66, 176.8, 332.8, 642.6, 1264}},
    {0, MLMC_F32, 1, MLMC_ICDF_EXACT, 0, {2.867, 5.058, 7.856, 14.16, 27.76, 51.63, 97.19, 192.7, 365.7, 709.4, 1401}},
    {0, MLMC_F16, 1, MLMC_ICDF_TABLE, 0, {2.522, 4.044, 5.871, 10.6, 20.31, 36.63, 68.36, 134.2, 250.9, 479.5, 935.8}},
    {0, MLMC_F16, 0, MLMC_ICDF_TABLE, 0, {2.475, 4.071, 5.61, 9.742, 18.39, 32.73, 62.36, 124.1, 227.1, 432, 836.9}},
    {0, MLMC_F32, 0, MLMC_ICDF_TABLE, 0, {2.539, 4.349, 6.062, 10.65, 20.18, 36, 68.91, 132.8, 249.4, 476.5, 930.2}},
    {0, MLMC_F16, 1, MLMC_ICDF_TABLE16, 0, {1.867, 3.099, 6.302, 8.54, 15.53, 29.52, 57.62, 116.8, 209.5, 398.6, 776.9}},
    {0, MLMC_F16, 0, MLMC_ICDF_TABLE16, 0, {1.863, 2.99, 6.059, 7.798, 14.03, 26.69, 50.99, 99.76, 182.3, 344.7, 670.2}},
    {0, MLMC_F32, 0, MLMC_ICDF_TABLE16, 0, {1.863, 3.106, 7.181, 8.778, 15.97, 29.75, 60.51, 113.1, 208.8, 401, 781}},
    {0, MLMC_F16, 1, MLMC_ICDF_CUBIC, 0, {2.695, 4.385, 6.697, 12.09, 22.94, 42.71, 80.51, 158.3, 298.3, 575.5, 1131}},
    {0, MLMC_F32, 0, MLMC_ICDF_CUBIC, 0, {2.672, 4.57, 6.747, 12.03, 23.28, 42.47, 79.8, 156.6, 293.5, 565.1, 1109}},
    {1, MLMC_F16, 1, MLMC_ICDF_TABLE, 0, {3.459, 5.811, 9.566, 17.46, 37.08, 64.19, 125.3, 248.3, 472.8, 926.7, 1830}},
    {1, MLMC_F16, 0, MLMC_ICDF_TABLE, 0, {3.417, 5.731, 9.109, 16.66, 34.97, 61.45, 117.8, 231.3, 442.8, 860.1, 1699}},
    {1, MLMC_F32, 0, MLMC_ICDF_TABLE, 0, {3.409, 6.081, 9.894, 17.69, 36.7, 62.91, 121.6, 240.1, 458.7, 891.4, 1761}},
    {1, MLMC_F16, 1, MLMC_ICDF_TABLE16, 0, {3.626, 6.069, 9.991, 18.25, 38.92, 67.65, 132.1, 265.1, 506.3, 981.5, 1943}},
    {1, MLMC_F16, 0, MLMC_ICDF_TABLE16, 0, {3.553, 6.01, 9.688, 17.69, 37.69, 65.53, 125.6, 248, 470.3, 914.6, 1808}},
    {1, MLMC_F32, 0, MLMC_ICDF_TABLE16, 0, {3.537, 6.444, 10.39, 18.67, 38.28, 67.02, 130.7, 258.9, 496.6, 967.3, 1914}},
    {1, MLMC_F16, 1, MLMC_ICDF_CUBIC, 0, {3.554, 6.036, 10.27, 18.72, 39.86, 69.48, 139.7, 273, 519, 1024, 2020}},
    {1, MLMC_F32, 0, MLMC_ICDF_CUBIC, 0, {3.592, 6.483, 10.56, 19.1, 38.85, 68.38, 133.6, 264.9, 506.2, 983.2, 1942}},
    {0, MLMC_F32, 0, MLMC_ICDF_EXACT, 1, {3, 5.264, 7.974, 14.72, 29.1, 53.41, 104, 202.5, 383.3, 748.9, 1472}},
    {0, MLMC_F32, 1, MLMC_ICDF_EXACT, 1, {2.982, 5.391, 8.641, 15.73, 30.92, 56.03, 108.7, 215.7, 410.4, 799.7, 1577}},
    {0, MLMC_F16, 1, MLMC_ICDF_TABLE, 1, {2.548, 4.168, 6.65, 11.89, 23.16, 42.43, 80.51, 158.9, 301.6, 580.3, 1140}},
    {0, MLMC_F32, 0, MLMC_ICDF_TABLE, 1, {2.657, 4.562, 6.741, 12.08, 23.32, 42.36, 80.96, 154.3, 292, 563.6, 1104}},
    {0, MLMC_F16, 1, MLMC_ICDF_TABLE16, 1, {1.896, 3.284, 6.702, 9.871, 18.65, 35.68, 70.92, 137.6, 259.7, 497.3, 976.3}},
    {0, MLMC_F32, 0, MLMC_ICDF_TABLE16, 1, {1.983, 3.578, 8.87, 10.24, 19.02, 36.67, 71.91, 138.2, 258.4, 497.5, 975.6}},
    {1, MLMC_F16, 1, MLMC_ICDF_TABLE, 1, {3.396, 6.303, 10.89, 20.17, 45.3, 79.15, 153.9, 300.2, 579.6, 1130, 2239}},
    {1, MLMC_F32, 0, MLMC_ICDF_TABLE, 1, {3.608, 6.691, 11.16, 20.3, 46, 82.57, 155.5, 304.6, 578.9, 1087, 2151}},
    {1, MLMC_F16, 1, MLMC_ICDF_TABLE16, 1, {3.491, 6.613, 11.48, 21.38, 46.18, 83.45, 161.9, 318.5, 615, 1200, 2376}},
    {1, MLMC_F32, 0, MLMC_ICDF_TABLE16, 1, {3.748, 7.041, 11.93, 21.6, 48.4, 85.3, 170.1, 342.5, 608.3, 1170, 2320}},
};

// The row of a term, or the nearest measured one: bfloat16 as binary16 (the
// same packed arithmetic), the other Kahan setting, the Euler row for a
// Milstein term; the network (MLP, a gather from its tabulated grid values)
// as its table row times the measured ratio (binary16 + Kahan at l = 10 and
// 12: four-way 1.81, two-way 3.55).
double cost_ps(int four, int prec, int kahan, int icdf, int milstein, int l) {
    double factor = 1.0;
    if (prec == MLMC_BF16) prec = MLMC_F16;
    if (icdf == MLMC_ICDF_MLP) {
        icdf = MLMC_ICDF_TABLE;
        factor = four ? 1.81 : 3.55;
    }
    const CostRow *row = nullptr;
    for (int pass = 0; pass < 4 && !row; ++pass) {
        const int k = pass & 1 ? !kahan : kahan, m = pass & 2 ? 0 : milstein;
        for (const CostRow &r : kCost)
            if (r.four == four && r.prec == prec && r.kahan == k && r.icdf == icdf && r.milstein == m) row = &r;
        if (row && m != milstein) factor *= 1.2;
    }
    if (!row) row = &kCost[four ? 10 : 0];
    return factor * (l <= 10 ? (double)row->ps[l] : ldexp((double)row->ps[10], l - 10));
}

double cost_of(const Term &t, int milstein) {
    return 1e-3 * cost_ps(t.four, t.prec, t.kahan, t.icdf, milstein, t.l);
}

}  // namespace

static mlmc_status run_impl(double eps, const mlmc_sde_params *p, const mlmc_run_opts *o, mlmc_run_result *out) {
    const auto t_start = std::chrono::steady_clock::now();
    DeviceState *d;
    mlmc_status st = device_state(&d);
    if (st) return st;
    const bool nested = o->estimator == 1;
    const int mil = p->scheme == MLMC_MILSTEIN && p->sde == MLMC_GBM ? 1 : 0;
    if (nested && o->icdf == MLMC_ICDF_MLP && !d->mlp_ready) return fail(MLMC_ENOTREADY, "MLP weights not set");

    // one run at a time per process: the stream and round buffers persist
    // across runs so that a run allocates nothing once they are large enough
    static std::mutex run_mu;
    std::lock_guard<std::mutex> lock(run_mu);
    cudaError_t e;
    if (!d->run_stream && (e = cudaStreamCreateWithFlags(&d->run_stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    if (!d->run_cache) d->run_cache = batch_cache_create();
    cudaStream_t s = d->run_stream;
    BatchCache *cache = d->run_cache;
    // around each round's launches (created once per device); the wait is on ev_b
    for (cudaEvent_t &ev : d->run_events)
        if (!ev && (e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(e, "cudaEventCreate");
    cudaEvent_t ev_a = d->run_events[0], ev_b = d->run_events[1];
    // MLMC_RUN_LOG=1: one JSON line per round on stderr (items, path-steps,
    // the cost model's and the measured device time, wall time, host time to
    // plan and enqueue the round)
    const char *log_env = getenv("MLMC_RUN_LOG");
    const bool log = log_env && atoi(log_env) > 0;
    std::vector<mlmc_round_record> trace;
    double model_ns = 0.0, device_ms = 0.0, discarded_steps = 0.0;

    std::vector<Term> terms;
    std::vector<int> lvl_prec(MLMC_MAX_LEVELS, o->prec), lvl_kahan(MLMC_MAX_LEVELS, o->kahan ? 1 : 0);
    std::vector<double> lvl_eff(MLMC_MAX_LEVELS, 0.0);
    std::vector<int> lvl_nested(MLMC_MAX_LEVELS, nested ? 1 : 0);
    std::vector<int> lvl_choice(MLMC_MAX_LEVELS, CH_NONE);
    double path_steps = 0.0;
    const double limit = o->timeout_s > 0 ? o->timeout_s : wait_limit_s();
    int rounds = 0;

    // Adds dn samples to every term with dn > 0 in one batched launch;
    // kept = 0 marks the draws of candidate terms (their records are fixed
    // up once the level's choice is made).
    auto run_round = [&](std::vector<Term> &ts, int kept) -> mlmc_status {
        std::vector<mlmc_work> items;
        std::vector<size_t> which;
        for (size_t i = 0; i < ts.size(); ++i) {
            if (ts[i].dn == 0) continue;
            ts[i].cost = cost_of(ts[i], mil);
            mlmc_work w;
            memset(&w, 0, sizeof w);
            w.params = *p;
            w.l = ts[i].l;
            w.kind = ts[i].four;
            w.prec = ts[i].prec;
            w.kahan = ts[i].kahan;
            w.icdf = ts[i].icdf;
            w.set_id = 0;
            w.N = ts[i].dn;
            w.path_offset = ts[i].n;
            items.push_back(w);
            which.push_back(i);
        }
        if (items.empty()) return MLMC_OK;
        const auto t0 = std::chrono::steady_clock::now();
        cudaEventRecord(ev_a, s);
        mlmc_status r = batch_round(*d, *cache, items.data(), (int)items.size(), o->seed, s);
        if (r) return r;
        const auto t_enq = std::chrono::steady_clock::now();
        cudaEventRecord(ev_b, s);
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if ((r = wait_event(ev_b, fmax(limit - el, 0.001)))) return r;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, ev_a, ev_b);
        device_ms += ms;
        double round_model_ns = 0.0;
        for (size_t k = 0; k < which.size(); ++k) round_model_ns += (double)ts[which[k]].dn * ts[which[k]].cost;
        model_ns += round_model_ns;
        if (log) {
            double ps = 0.0;
            for (const auto &w : items) ps += ldexp((double)w.N, w.l);
            const double host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            const double enq_ms = std::chrono::duration<double, std::milli>(t_enq - t0).count();
            fprintf(stderr, "{\"mlmc_run_round\": %d, \"items\": %zu, \"path_steps\": %.0f, \"model_ms\": %.4f, "
                            "\"device_ms\": %.4f, \"wall_ms\": %.4f, \"enqueue_ms\": %.4f}\n",
                    rounds, items.size(), ps, round_model_ns * 1e-6, ms, host_ms, enq_ms);
        }
        const double2 *sums = batch_sums_host(*cache);
        for (size_t k = 0; k < which.size(); ++k) {
            Term &t = ts[which[k]];
            mlmc_round_record rec;
            memset(&rec, 0, sizeof rec);
            rec.round = rounds;
            rec.l = t.l;
            rec.kind = t.four;
            rec.prec = t.prec;
            rec.kahan = t.kahan;
            rec.icdf = t.icdf;
            rec.kept = kept;
            rec.dn = t.dn;
            rec.path_offset = t.n;
            rec.s1 = sums[k].x;
            rec.s2 = sums[k].y;
            rec.cost_ns = t.cost;
            trace.push_back(rec);
            path_steps += (double)t.dn * ldexp(1.0, t.l);
            t.s1 += sums[k].x;
            t.s2 += sums[k].y;
            t.n += t.dn;
            t.dn = 0;
        }
        ++rounds;
        return MLMC_OK;
    };
    // The records of the candidate terms of the last trial that the level
    // kept become kept = 1.
    auto keep_trial_records = [&](const std::vector<Term> &kept_terms) {
        for (auto it = trace.rbegin(); it != trace.rend() && it->kept == 0 && it->round == rounds - 1; ++it)
            for (const Term &t : kept_terms)
                if (!t.off && it->l == t.l && it->kind == t.four && it->prec == t.prec && it->kahan == t.kahan &&
                    it->icdf == t.icdf)
                    it->kept = 1;
    };
    const bool autoprec = nested && o->prec < 0;
    bool half_done = false;      // a coarser level already chose FP32 or the standard estimator
    // The standard FP32 exact-normal two-way term alone at level l, with an
    // empty four-way slot (both estimate E[P^_l - P^_{l-1}]).
    auto push_standard = [&](int l, const Term &std_term) {
        lvl_prec[l] = MLMC_F32;
        lvl_kahan[l] = 1;
        lvl_nested[l] = 0;
        terms.push_back(std_term);
        Term slot{l, 1, MLMC_F32, 0, o->icdf};
        slot.off = true;
        terms.push_back(slot);
    };
    // Candidates of level l (two-way, four-way) x {FP16 + Kahan, FP16, FP32},
    // plus the standard FP32 exact-normal two-way term (with Kahan, the
    // four-way hat paths' arithmetic): the efficiency reference and a
    // candidate.  Seven terms in that order; those from variant `first` on
    // and the standard term draw n0 samples.  Once a level has chosen FP32
    // (or the standard estimator) the binary16 candidates are not tried
    // again: their rounding variance does not decay with delta while the
    // level variance does (Sec. 3), so they only lose further on finer
    // levels.
    const int cp[3] = {MLMC_F16, MLMC_F16, MLMC_F32}, ck[3] = {1, 0, 0};
    auto candidates = [&](int l, int first) {
        std::vector<Term> cand;
        for (int c = 0; c < 3; ++c) {
            cand.push_back(Term{l, 0, cp[c], ck[c], o->icdf});
            cand.push_back(Term{l, 1, cp[c], ck[c], o->icdf});
        }
        cand.push_back(Term{l, 0, MLMC_F32, 1, MLMC_ICDF_EXACT});
        for (size_t i = 0; i < cand.size(); ++i)
            if (i >= (size_t)(2 * first)) cand[i].dn = round8(o->n0);
        return cand;
    };
    // The level's choice from its sampled candidates (coarser levels already
    // chosen): the carried FP32 choice where two coarser levels agree on it
    // (its candidate's samples are its warm-up), else the smallest score
    // sqrt(v c) + sqrt(V C) among the variants still allowed, or the
    // standard term if cheaper still.
    auto choose_level = [&](int l, std::vector<Term> cand) {
        auto vc = [&](const Term &t) { return t.var() * cost_of(t, mil); };
        auto steps = [&](const Term &t) { return (double)t.n * ldexp(1.0, l); };
        for (const Term &t : cand) discarded_steps += steps(t);
        if (!o->trial_all && l >= 2 && lvl_choice[l - 1] == lvl_choice[l - 2] &&
            (lvl_choice[l - 1] == CH_F32 || lvl_choice[l - 1] == CH_STANDARD)) {
            lvl_choice[l] = lvl_choice[l - 1];
            if (lvl_choice[l] == CH_STANDARD) {
                push_standard(l, cand[6]);
                keep_trial_records({cand[6]});
                discarded_steps -= steps(cand[6]);
            } else {
                lvl_prec[l] = MLMC_F32;
                lvl_kahan[l] = 0;
                terms.push_back(cand[4]);
                terms.push_back(cand[5]);
                keep_trial_records({cand[4], cand[5]});
                discarded_steps -= steps(cand[4]) + steps(cand[5]);
            }
            return;
        }
        int first = 0;
        while (first < 2 && cand[2 * first].n == 0) ++first;
        if (half_done) first = 2;
        int best = first;
        double best_score = 1e300;
        for (int c = first; c < 3; ++c) {
            const double score = sqrt(vc(cand[2 * c])) + sqrt(vc(cand[2 * c + 1]));
            if (score < best_score) {
                best_score = score;
                best = c;
            }
        }
        const double vc2 = vc(cand[2 * best]), vc4 = vc(cand[2 * best + 1]), vch = vc(cand[6]);
        if (vch > 0.0 && vc2 > 0.0) lvl_eff[l] = vc2 / vch * pow(1.0 + sqrt(vc4 / vc2), 2.0);
        if (vch > 0.0 && sqrt(vch) < best_score) {
            // the standard estimator alone is cheaper for this level
            lvl_choice[l] = CH_STANDARD;
            half_done = true;
            push_standard(l, cand[6]);
            keep_trial_records({cand[6]});
            discarded_steps -= steps(cand[6]);
            return;
        }
        lvl_choice[l] = best;
        lvl_prec[l] = cp[best];
        lvl_kahan[l] = ck[best];
        if (cp[best] == MLMC_F32) half_done = true;
        terms.push_back(cand[2 * best]);
        terms.push_back(cand[2 * best + 1]);
        keep_trial_records({cand[2 * best], cand[2 * best + 1]});
        discarded_steps -= steps(cand[2 * best]) + steps(cand[2 * best + 1]);
    };
    auto add_level = [&](int l) -> mlmc_status {
        if (!nested) {
            terms.push_back(Term{l, 0, MLMC_F32, o->kahan ? 1 : 0, MLMC_ICDF_EXACT});
            terms.back().dn = round8(o->n0);
            return MLMC_OK;
        }
        if (!autoprec) {
            terms.push_back(Term{l, 0, o->prec, o->kahan ? 1 : 0, o->icdf});
            terms.push_back(Term{l, 1, o->prec, o->kahan ? 1 : 0, o->icdf});
            terms[terms.size() - 2].dn = terms.back().dn = round8(o->n0);
            return MLMC_OK;
        }
        // Carried choice: once two consecutive levels have chosen the same
        // FP32 variant, finer levels take it without candidate samples (the
        // binary16 rounding floor only loses ground as delta shrinks, Sec. 3).
        if (!o->trial_all && l >= 2 && lvl_choice[l - 1] == lvl_choice[l - 2] &&
            (lvl_choice[l - 1] == CH_F32 || lvl_choice[l - 1] == CH_STANDARD)) {
            lvl_choice[l] = lvl_choice[l - 1];
            if (lvl_choice[l] == CH_STANDARD) {
                push_standard(l, Term{l, 0, MLMC_F32, 1, MLMC_ICDF_EXACT});
                terms[terms.size() - 2].dn = round8(o->n0);
            } else {
                lvl_prec[l] = MLMC_F32;
                lvl_kahan[l] = 0;
                terms.push_back(Term{l, 0, MLMC_F32, 0, o->icdf});
                terms.push_back(Term{l, 1, MLMC_F32, 0, o->icdf});
                terms[terms.size() - 2].dn = terms.back().dn = round8(o->n0);
            }
            return MLMC_OK;
        }
        std::vector<Term> cand = candidates(l, half_done ? 2 : 0);
        std::vector<Term> tried;
        for (const Term &t : cand)
            if (t.dn) tried.push_back(t);
        mlmc_status r = run_round(tried, 0);
        if (r) return r;
        for (Term &t : cand)
            for (const Term &u : tried)
                if (t.l == u.l && t.four == u.four && t.prec == u.prec && t.kahan == u.kahan && t.icdf == u.icdf) t = u;
        choose_level(l, cand);
        return MLMC_OK;
    };
    int L = o->min_levels - 1;
    if (autoprec) {
        // the initial levels' candidates in one round, then each level's
        // choice in order of l
        std::vector<Term> all;
        for (int l = 0; l <= L; ++l) {
            std::vector<Term> c = candidates(l, 0);
            all.insert(all.end(), c.begin(), c.end());
        }
        st = run_round(all, 0);
        for (int l = 0; l <= L && !st; ++l)
            choose_level(l, std::vector<Term>(all.begin() + 7 * l, all.begin() + 7 * (l + 1)));
    } else {
        for (int l = 0; l <= L && !st; ++l) st = add_level(l);
    }
    const int per_level = nested ? 2 : 1;
    bool converged = false;

    // Optimal sample counts from the current estimates (Sec. 3).  When the
    // estimated variance sum V_t / N_t of the terms already sampled exceeds
    // eps^2 / 2, each term's dn grows to its shortfall against the optimal
    // split; returns whether a round is needed (a shortfall, or a new level's
    // pending warm-up).  A term without samples yet (a new level) takes an
    // extrapolated variance, so the re-optimisation of all levels can share
    // the new level's warm-up round.
    auto plan_samples = [&]() -> bool {
        std::vector<double> V(terms.size()), C(terms.size());
        for (size_t i = 0; i < terms.size(); ++i) {
            V[i] = terms[i].off ? 0.0 : terms[i].var();
            const bool prev_on = terms[i].l >= 2 && !terms[i].off && !terms[i - per_level].off;
            if (prev_on && terms[i].n == 0 && terms[i].l >= 3 && !terms[i - 2 * per_level].off &&
                V[i - 2 * per_level] > 0.0) {
                // a level without samples yet: extrapolate the decay of the
                // two levels below it (between 1/4 and 1 per level)
                const double ratio = V[i - per_level] / V[i - 2 * per_level];
                V[i] = V[i - per_level] * fmin(fmax(ratio, 0.25), 1.0);
            } else if (prev_on) {
                // a level's variance is at least a quarter of its
                // predecessor's (guards levels with few samples)
                V[i] = fmax(V[i], 0.25 * V[i - per_level]);
            }
            C[i] = cost_of(terms[i], mil);
            terms[i].cost = C[i];
        }
        double total = 0.0, var_sum = 0.0;
        bool pending = false;
        for (size_t i = 0; i < terms.size(); ++i) {
            total += sqrt(V[i] * C[i]);
            if (terms[i].n) var_sum += V[i] / (double)terms[i].n;
            if (terms[i].dn) pending = true;
        }
        if (var_sum <= 0.5 * eps * eps && !pending) return false;
        bool need = pending;
        for (size_t i = 0; i < terms.size(); ++i) {
            if (terms[i].off) continue;
            const double Nopt = ceil(2.0 / (eps * eps) * sqrt(V[i] / C[i]) * total);
            const double dn = Nopt - (double)(terms[i].n + terms[i].dn);
            if (dn > 0.0) {
                terms[i].dn = round8(terms[i].dn + (uint64_t)dn);
                need = true;
            }
        }
        return need;
    };

    while (!st) {
        if ((st = run_round(terms, 1))) break;
        const bool need = plan_samples();
        // ---- weak-error test on the last three level means, after every
        // round (the loop of the MLMC review's algorithm): a failed test adds
        // level L + 1 at once, so that its warm-up shares the next round with
        // the top-ups plan_samples just asked for
        std::vector<double> Y(L + 1, 0.0);
        for (const Term &t : terms) Y[t.l] += t.mean();
        const double r = pow(2.0, o->alpha);
        double bias = fabs(Y[L]);
        if (L >= 1) bias = fmax(bias, fabs(Y[L - 1]) / r);
        if (L >= 2) bias = fmax(bias, fabs(Y[L - 2]) / (r * r));
        bias /= (r - 1.0);
        if (bias <= eps / sqrt(2.0)) {
            if (!need) {
                converged = true;
                break;
            }
            continue;
        }
        if (L >= o->max_level) {
            if (!need) break;
            continue;
        }
        ++L;
        st = add_level(L);
        // the new level's warm-up and the other levels' top-ups in one round
        if (!st) plan_samples();
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
        for (int l = 0; l <= L && l < MLMC_MAX_LEVELS; ++l) {
            out->prec[l] = nested ? lvl_prec[l] : MLMC_F32;
            out->kahan[l] = nested ? lvl_kahan[l] : (o->kahan ? 1 : 0);
            out->efficiency[l] = lvl_eff[l];
            out->nested[l] = lvl_nested[l];
        }
        out->path_steps = path_steps;
        out->trace_len = (int32_t)trace.size();
        if (o->trace && o->trace_cap > 0)
            memcpy(o->trace, trace.data(), std::min<size_t>(trace.size(), (size_t)o->trace_cap) * sizeof(mlmc_round_record));
        out->model_s = model_ns * 1e-9;
        out->device_s = device_ms * 1e-3;
        out->discarded_path_steps = discarded_steps;
        out->wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
        if (!converged) st = fail(MLMC_ENOTCONV, "bias test not met at max_level %d", o->max_level);
    }
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
        if (opts->prec != MLMC_F32 && opts->prec != MLMC_F16 && opts->prec != MLMC_BF16 && opts->prec != -1)
            return fail(MLMC_EINVAL, "unknown precision");
        if (opts->icdf != MLMC_ICDF_TABLE && opts->icdf != MLMC_ICDF_MLP && opts->icdf != MLMC_ICDF_TABLE16 &&
            opts->icdf != MLMC_ICDF_CUBIC)
            return fail(MLMC_EINVAL, "nested estimator needs approximate normals");
    }
    return run_impl(eps, params, opts, out);
}
