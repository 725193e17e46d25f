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
