"""Closed forms and the adaptive multilevel Monte Carlo driver (Sec. 3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Closed forms used as pins (exact, not asymptotic):
  * GBM terminal law: E X_T = X0 e^{mu T}, Var X_T = X0^2 e^{2 mu T}(e^{sigma^2 T} - 1);
    Black-Scholes call with r = mu.
  * Euler-Maruyama GBM with P(X) = X (Sec. 3 takes P(X) = X): each step
    multiplies X by (1 + mu delta + sigma sqrt(delta) Z).  With i.i.d. pairs
    (Z, Z~), E Z = E Z~ = 0, E Z^2 = 1, E Z~^2 = m2, E Z Z~ = mc, every
    product of two of the four coupled paths (exact/approximate x
    fine/coarse) has an expectation that is a product over coarse steps of
    a polynomial in a = 1 + mu delta, b = 1 + 2 mu delta, s2 = sigma^2 delta.

The driver follows the cost model of Sec. 3 (T^ and T- with the optimal
sample split N_l proportional to sqrt(V_l / C_l)); the weak-error test and
warm-up follow the standard MLMC algorithm the paper cites (giles2008
multilevel); the constants are readings, stated in the function docstrings.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr


def gbm_terminal(mu=0.05, sigma=0.2, x0=1.0, T=1.0):
    m = x0 * math.exp(mu * T)
    return m, x0 * x0 * math.exp(2 * mu * T) * (math.exp(sigma * sigma * T) - 1.0)


def bs_call(mu=0.05, sigma=0.2, x0=1.0, T=1.0, K=1.0, discounted=True):
    """Black-Scholes price with r = mu (undiscounted: times e^{mu T})."""
    d1 = (math.log(x0 / K) + (mu + 0.5 * sigma * sigma) * T) / (sigma * math.sqrt(T))
    d2 = d1 - sigma * math.sqrt(T)
    price = x0 * ndtr(d1) - K * math.exp(-mu * T) * ndtr(d2)
    return float(price if discounted else price * math.exp(mu * T))


def _step_moments(mu, sigma, delta, m2=1.0, mc=1.0):
    a, b, s2 = 1.0 + mu * delta, 1.0 + 2.0 * mu * delta, sigma * sigma * delta
    # per coarse step (two fine steps); keys name the pair of paths
    return {
        "hf": a * a, "hc": b, "bf": a * a, "bc": b,
        "hf_hf": (a * a + s2) ** 2, "hc_hc": b * b + 2 * s2,
        "bf_bf": (a * a + s2 * m2) ** 2, "bc_bc": b * b + 2 * s2 * m2,
        "hf_hc": a * a * b + 2 * a * s2, "bf_bc": a * a * b + 2 * a * s2 * m2,
        "hf_bf": (a * a + s2 * mc) ** 2, "hc_bc": b * b + 2 * s2 * mc,
        "hf_bc": a * a * b + 2 * a * s2 * mc, "hc_bf": a * a * b + 2 * a * s2 * mc,
    }


def euler_twoway_moments(l, mu=0.05, sigma=0.2, x0=1.0, T=1.0, m2=1.0):
    """(E D, Var D) of D = X_f - X_c at level l (D = X_f at l = 0) for the
    Euler GBM with i.i.d. normals of second moment m2 (m2 = 1: exact)."""
    if l == 0:
        a = 1.0 + mu * T
        return x0 * a, x0 * x0 * sigma * sigma * T * m2
    delta = T * 2.0 ** -l
    n = 2 ** (l - 1)
    k = _step_moments(mu, sigma, delta, m2=m2, mc=m2)
    ef, ec = k["bf"] ** n, k["bc"] ** n
    eff, ecc, efc = k["bf_bf"] ** n, k["bc_bc"] ** n, k["bf_bc"] ** n
    mean = x0 * (ef - ec)
    second = x0 * x0 * (eff + ecc - 2 * efc)
    return mean, second - mean * mean


def euler_fourway_moments(l, m2, mc, mu=0.05, sigma=0.2, x0=1.0, T=1.0):
    """(E D, Var D) of the four-way D = X^_f - X^_c - X-_f + X-_c (FP64,
    exact vs approximate normals with E Z~^2 = m2, E Z Z~ = mc)."""
    if l == 0:
        # D = sigma sqrt(T) x0 (Z - Z~)
        return 0.0, x0 * x0 * sigma * sigma * T * (1.0 - 2 * mc + m2)
    delta = T * 2.0 ** -l
    n = 2 ** (l - 1)
    k = _step_moments(mu, sigma, delta, m2=m2, mc=mc)
    sign = {"hf": 1, "hc": -1, "bf": -1, "bc": 1}
    names = list(sign)
    second = 0.0
    for i, p in enumerate(names):
        for q in names[i:]:
            key = f"{p}_{q}" if f"{p}_{q}" in k else f"{q}_{p}"
            mult = 1 if p == q else 2
            second += mult * sign[p] * sign[q] * k[key] ** n
    mean = x0 * (k["hf"] ** n - k["hc"] ** n - k["bf"] ** n + k["bc"] ** n)
    return mean, x0 * x0 * second - mean * mean


def optimal_samples(V, C, eps):
    """N_l = ceil(2 eps^-2 sqrt(V_l / C_l) sum_j sqrt(V_j C_j)) (Sec. 3: the
    split that gives T = 2 eps^-2 (sum sqrt(V C))^2, half of eps^2 to the
    sampling variance)."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    total = np.sum(np.sqrt(V * C))
    return np.ceil(2.0 * eps ** -2 * np.sqrt(V / C) * total).astype(np.int64)


def predicted_cost(V, C, eps):
    """T = 2 eps^-2 (sum_l sqrt(V_l C_l))^2 (Sec. 3)."""
    return 2.0 * eps ** -2 * float(np.sum(np.sqrt(np.asarray(V) * np.asarray(C)))) ** 2


def weak_converged(Y, eps, alpha=1.0):
    """Weak-error test of the standard MLMC algorithm: the remaining bias
    max(|Y_L|, |Y_{L-1}| 2^-alpha, |Y_{L-2}| 2^-2alpha) / (2^alpha - 1) must
    be <= eps / sqrt(2) (reading: the paper defers the algorithm to
    giles2008multilevel; alpha = 1, the Euler weak order)."""
    if len(Y) < 3:
        return False
    r = 2.0 ** alpha
    bias = max(abs(Y[-1]), abs(Y[-2]) / r, abs(Y[-3]) / (r * r)) / (r - 1.0)
    return bias <= eps / math.sqrt(2.0)


# ---------------------------------------------------------------- GBM step polynomials
# Per coarse step (two fine steps), each of the four coupled paths multiplies
# X by a polynomial in the step's normals: variables (Z1, W1, Z2, W2), with
# Z the exact normal and W = Z~ the approximate one of the same uniform.
#   fine (Euler):     (1 + mu d + s Z1)(1 + mu d + s Z2),  s = sigma sqrt(d)
#   fine (Milstein):  each factor + m (Z^2 - 1),           m = sigma^2 d / 2
#   coarse (Euler):   1 + 2 mu d + s (Z1 + Z2)
#   coarse (Milstein): + m ((Z1 + Z2)^2 - 2)
# and the same with W for the approximate paths.  Expectations use the
# joint moments mom(a, b) = E[Z^a W^b] of one step, steps being independent.

def _pmul(p, q):
    out = {}
    for ep, cp in p.items():
        for eq, cq in q.items():
            e = tuple(x + y for x, y in zip(ep, eq))
            out[e] = out.get(e, 0.0) + cp * cq
    return out


def _unit(i, power=1):
    e = [0, 0, 0, 0]
    e[i] = power
    return tuple(e)


def _step_polys(mu, sigma, delta, milstein):
    s = sigma * math.sqrt(delta)
    m = 0.5 * sigma * sigma * delta if milstein else 0.0
    zero = (0, 0, 0, 0)

    def fine_factor(i):
        return {zero: 1.0 + mu * delta - m, _unit(i): s, _unit(i, 2): m}

    def coarse(i, j):
        ij = tuple(a + b for a, b in zip(_unit(i), _unit(j)))
        return {zero: 1.0 + 2.0 * mu * delta - 2.0 * m, _unit(i): s, _unit(j): s,
                _unit(i, 2): m, _unit(j, 2): m, ij: 2.0 * m}

    return {"hf": _pmul(fine_factor(0), fine_factor(2)), "hc": coarse(0, 2),
            "bf": _pmul(fine_factor(1), fine_factor(3)), "bc": coarse(1, 3)}


def _expect(p, mom):
    return sum(c * mom(e[0], e[1]) * mom(e[2], e[3]) for e, c in p.items())


def gaussian_moment(a, b=0):
    """E[Z^(a+b)] for W = Z (exact normals in both slots)."""
    k = a + b
    return 0.0 if k % 2 else float(np.prod(np.arange(k - 1, 0, -2))) if k else 1.0


def gbm_level_moments(l, mom=gaussian_moment, four=False, milstein=False, mu=0.05, sigma=0.2, x0=1.0, T=1.0):
    """(E D, Var D) of the level-l difference for GBM with P(X) = X in exact
    arithmetic: two-way D = X_f - X_c on the approximate normals W (W = Z by
    default), or four-way D = X^_f - X^_c - X-_f + X-_c (hat on Z, bar on
    W); Euler or Milstein.  mom(a, b) = E[Z^a W^b] for one step."""
    if l == 0:
        m = 0.5 * sigma * sigma * T if milstein else 0.0
        s = sigma * math.sqrt(T)
        zero = (0, 0, 0, 0)
        h = {zero: 1.0 + mu * T - m, _unit(0): s, _unit(0, 2): m}
        b = {zero: 1.0 + mu * T - m, _unit(1): s, _unit(1, 2): m}
        if four:
            d = dict(h)
            for e, c in b.items():
                d[e] = d.get(e, 0.0) - c
        else:
            d = b
        mean = x0 * _expect(d, mom)
        return mean, x0 * x0 * _expect(_pmul(d, d), mom) - mean * mean
    delta = T * 2.0 ** -l
    n = 2 ** (l - 1)
    P = _step_polys(mu, sigma, delta, milstein)
    sign = {"hf": 1, "hc": -1, "bf": -1, "bc": 1} if four else {"bf": 1, "bc": -1}
    names = list(sign)
    mean = x0 * sum(sign[p] * _expect(P[p], mom) ** n for p in names)
    second = 0.0
    for i, p in enumerate(names):
        for q in names[i:]:
            mult = 1 if p == q else 2
            second += mult * sign[p] * sign[q] * _expect(_pmul(P[p], P[q]), mom) ** n
    return mean, x0 * x0 * second - mean * mean


def grid_joint_moments(z, w, max_order=4):
    """mom(a, b) = mean of z^a w^b over a grid (the uniform's law)."""
    table = {}
    for a in range(max_order + 1):
        for b in range(max_order + 1 - a):
            table[(a, b)] = float(np.mean(z ** a * w ** b))
    return lambda a, b: table[(a, b)]


# ---------------------------------------------------------------- adaptive driver
# The standard adaptive MLMC algorithm that Sec. 3's T^ / T- cost comparison
# assumes (the paper defers its steps to giles2008multilevel), with the
# nested estimator's terms and the per-level variant choice, written as a
# plain loop.  Samples come from a callback, so the loop can be driven by
# exact synthetic level statistics (its pins) or replay the sums an
# implementation drew (to compare decisions).
#
# Readings (stated once, used by both the oracle and the library):
#   * terms per level l: standard estimator theta^: the FP32 exact-normal
#     two-way difference; nested theta-: the two-way difference with
#     approximate normals and the four-way difference;
#   * warm-up n0 samples per new term; every draw is rounded up to a
#     multiple of 8 samples;
#   * V_l of a term without samples at l >= 3 is extrapolated from the two
#     levels below it, V_{l-1} min(max(V_{l-1} / V_{l-2}, 1/4), 1); a sampled
#     term at l >= 2 keeps V_l >= V_{l-1} / 4;
#   * N_t = ceil(2 eps^-2 sqrt(V_t / C_t) sum_s sqrt(V_s C_s)) (Sec. 3),
#     drawn whenever sum_t V_t / N_t > eps^2 / 2;
#   * bias test max(|Y_L|, |Y_{L-1}| 2^-alpha, |Y_{L-2}| 2^-2alpha) /
#     (2^alpha - 1) <= eps / sqrt(2), else L + 1 (up to max_level), after
#     every round (the loop of the MLMC review's algorithm: evaluate the
#     extra samples, update V_l and N_l, test weak convergence, add a level
#     if it fails), so a new level's warm-up shares a round with the top-ups;
#     the run ends when the test holds and no term needs more samples;
#   * per-level choice (prec = -1): the candidates {binary16 + Kahan,
#     binary16, binary32} nested pairs and the standard term alone, n0
#     samples each in a round of their own (the initial levels' candidates
#     all in one round, each level then chosen in order of l, the rules
#     below applied at the choice); the level keeps the nested pair
#     with the smallest sqrt(v C) + sqrt(V C), or the standard term if its
#     sqrt(v^ c^) is smaller still; binary16 candidates stop once a level has
#     chosen binary32 or the standard term; without trial_all, once two
#     consecutive levels chose the same binary32 variant, finer levels take
#     it without candidates.

F32, F16 = 0, 1
EXACT = 0
CH_F16K, CH_F16, CH_F32, CH_STANDARD = 0, 1, 2, 3


def moments(s1, s2, n):
    """Sample mean and unbiased variance from the sums of n samples."""
    m = s1 / n
    return m, (max((s2 - s1 * m) / (n - 1), 0.0) if n > 1 else 0.0)


def _round8(n):
    return (n + 7) // 8 * 8


class _Term:
    def __init__(self, l, kind, prec, kahan, icdf, off=False):
        self.key = (l, kind, prec, kahan, icdf)
        self.l = l
        self.off = off
        self.n = 0
        self.dn = 0
        self.s1 = 0.0
        self.s2 = 0.0

    def V(self):
        return moments(self.s1, self.s2, self.n)[1] if self.n else 0.0

    def Y(self):
        return moments(self.s1, self.s2, self.n)[0] if self.n else 0.0


def adaptive_mlmc(eps, draw, cost, *, nested, prec=F16, kahan=1, icdf=1, n0=10000, min_levels=3,
                  max_level=18, alpha=1.0, trial_all=False):
    """Adaptive MLMC to RMSE eps.

    draw(requests) -> [(s1, s2), ...]: one round; requests are
    (key, dn, path_offset) with key = (l, kind, prec, kahan, icdf), kind 0
    two-way, 1 four-way.  cost(key) -> C_t, the device cost per sample.
    prec = -1 (nested only): the per-level choice.
    Returns a dict: estimate, levels (L + 1), rounds, choice per level,
    the terms' (key, n, mean, var)."""
    terms = []                    # two-way and four-way slot per level (nested), one term per level (standard)
    per = 2 if nested else 1
    rounds = [0]
    choice = {}
    half_done = [False]

    def run(ts):
        req = [t for t in ts if t.dn > 0]
        if not req:
            return
        sums = draw([(t.key, t.dn, t.n) for t in req])
        for t, (s1, s2) in zip(req, sums):
            t.s1 += s1
            t.s2 += s2
            t.n += t.dn
            t.dn = 0
        rounds[0] += 1

    def vc(t):
        return t.V() * cost(t.key)

    variants = [(F16, 1), (F16, 0), (F32, 0)]     # the nested pairs' candidates CH_F16K, CH_F16, CH_F32

    def add_level(l):
        if not nested:
            t = _Term(l, 0, F32, kahan, EXACT)
            t.dn = _round8(n0)
            terms.append(t)
            return
        if prec != -1:
            for kind in (0, 1):
                t = _Term(l, kind, prec, kahan, icdf)
                t.dn = _round8(n0)
                terms.append(t)
            return
        carried = choice.get(l - 1) if l >= 2 and choice.get(l - 1) == choice.get(l - 2) else None
        if not trial_all and carried in (CH_F32, CH_STANDARD):
            choice[l] = carried
            if carried == CH_STANDARD:
                pair = [_Term(l, 0, F32, 1, EXACT), _Term(l, 1, F32, 0, icdf, off=True)]
            else:
                pair = [_Term(l, 0, F32, 0, icdf), _Term(l, 1, F32, 0, icdf)]
            for t in pair:
                t.dn = 0 if t.off else _round8(n0)
            terms.extend(pair)
            return
        cands, standard = trial_terms(l, 2 if half_done[0] else 0)
        run([t for c in sorted(cands) for t in cands[c]] + [standard])
        choose(l, cands, standard)

    def trial_terms(l, first):
        """The candidates of level l (the nested pairs from variant `first`
        on, and the standard term), n0 samples each."""
        cands = {c: (_Term(l, 0, *variants[c], icdf), _Term(l, 1, *variants[c], icdf)) for c in range(first, 3)}
        standard = _Term(l, 0, F32, 1, EXACT)
        for c in cands:
            for t in cands[c]:
                t.dn = _round8(n0)
        standard.dn = _round8(n0)
        return cands, standard

    def choose(l, cands, standard):
        """The level's variant from its sampled candidates (levels coarser
        than l already chosen): the carried binary32 choice where two
        coarser levels agree on it (its candidate's samples are its
        warm-up), else the smallest score among the variants still allowed
        (binary32 only once a coarser level chose binary32 or the standard
        term), or the standard term if cheaper still."""
        carried = choice.get(l - 1) if l >= 2 and choice.get(l - 1) == choice.get(l - 2) else None
        if not trial_all and carried in (CH_F32, CH_STANDARD):
            choice[l] = carried
            if carried == CH_STANDARD:
                terms.extend([standard, _Term(l, 1, F32, 0, icdf, off=True)])
            else:
                terms.extend(cands[CH_F32])
            return
        first = 2 if half_done[0] else min(cands)
        best, best_score = first, 1e300
        for c in range(first, 3):
            score = math.sqrt(vc(cands[c][0])) + math.sqrt(vc(cands[c][1]))
            if score < best_score:
                best, best_score = c, score
        vch = vc(standard)
        if vch > 0.0 and math.sqrt(vch) < best_score:
            choice[l] = CH_STANDARD
            half_done[0] = True
            terms.extend([standard, _Term(l, 1, F32, 0, icdf, off=True)])
            return
        choice[l] = best
        if variants[best][0] == F32:
            half_done[0] = True
        terms.extend(cands[best])

    def plan():
        V = []
        for i, t in enumerate(terms):
            v = 0.0 if t.off else t.V()
            prev_on = t.l >= 2 and not t.off and not terms[i - per].off
            if prev_on and t.n == 0 and t.l >= 3 and not terms[i - 2 * per].off and V[i - 2 * per] > 0.0:
                v = V[i - per] * min(max(V[i - per] / V[i - 2 * per], 0.25), 1.0)
            elif prev_on:
                v = max(v, 0.25 * V[i - per])
            V.append(v)
        C = [cost(t.key) for t in terms]
        total = 0.0
        var_sum = 0.0
        for i, t in enumerate(terms):
            total += math.sqrt(V[i] * C[i])
            if t.n:
                var_sum += V[i] / t.n
        pending = any(t.dn for t in terms)
        if var_sum <= 0.5 * eps * eps and not pending:
            return False
        need = pending
        for i, t in enumerate(terms):
            if t.off:
                continue
            N_t = math.ceil(2.0 / (eps * eps) * math.sqrt(V[i] / C[i]) * total)
            short = N_t - (t.n + t.dn)
            if short > 0:
                t.dn = _round8(t.dn + short)
                need = True
        return need

    L = min_levels - 1
    if nested and prec == -1:
        # the initial levels' candidates in one round, then each level's
        # choice in order of l
        batch = [(l, *trial_terms(l, 0)) for l in range(L + 1)]
        run([t for _, cands, standard in batch for t in [x for c in sorted(cands) for x in cands[c]] + [standard]])
        for l, cands, standard in batch:
            choose(l, cands, standard)
    else:
        for l in range(L + 1):
            add_level(l)
    converged = False
    while True:
        run(terms)
        need = plan()
        # the weak-error test after every round, on the samples so far: a
        # failed test adds level L + 1 at once, so that its warm-up shares
        # the next round with the top-ups plan() just asked for
        Y = [0.0] * (L + 1)
        for t in terms:
            Y[t.l] += t.Y()
        r = 2.0 ** alpha
        bias = abs(Y[L])
        if L >= 1:
            bias = max(bias, abs(Y[L - 1]) / r)
        if L >= 2:
            bias = max(bias, abs(Y[L - 2]) / (r * r))
        bias /= (r - 1.0)
        if bias <= eps / math.sqrt(2.0):
            if not need:
                converged = True
                break
            continue
        if L >= max_level:
            if not need:
                break
            continue
        L += 1
        add_level(L)
        plan()
    est = var = 0.0
    for t in terms:                 # plain left-to-right sums (builtin sum() compensates)
        est += t.Y()
        if t.n:
            var += t.V() / t.n
    return {"estimate": est, "variance": var, "levels": L + 1, "rounds": rounds[0], "converged": converged,
            "choice": [choice.get(l) for l in range(L + 1)],
            "terms": [(t.key, t.n, t.Y(), t.V()) for t in terms if not t.off]}
