"""Pins of the oracle's adaptive MLMC driver (the standard algorithm behind
Sec. 3's cost comparison) on synthetic level statistics with closed-form
answers: each term returns sums whose sample mean and variance are exactly
(mu_t, sigma_t^2), so the final level L, the Lagrange-optimal sample split
and the per-level variant choice are known in advance."""
import math

import pytest

from oracle import mlmc

EPS = 1e-3


class Synthetic:
    """draw() callback: sums of dn samples with cumulative mean mu and
    cumulative unbiased variance var for every term key; records requests."""

    def __init__(self, stats):
        self.stats = stats          # key -> (mu, var)
        self.n = {}
        self.rounds = []

    def __call__(self, requests):
        self.rounds.append(requests)
        out = []
        for key, dn, off in requests:
            mu, var = self.stats(key)
            n0 = self.n.get(key, 0)
            assert off == n0, "path offsets must be the samples already drawn"
            n1 = n0 + dn

            def cum(n):
                return (n - 1) * var + n * mu * mu if n else 0.0
            out.append((n1 * mu - n0 * mu, cum(n1) - cum(n0)))
            self.n[key] = n1
        return out


def _cost(key):
    l, kind = key[0], key[1]
    return 2.0 ** l * (2.0 if kind else 1.0)


def test_standard_estimator_stops_at_the_closed_form_level_with_the_optimal_split():
    m0, v0 = 0.3, 0.04
    syn = Synthetic(lambda k: (m0 * 2.0 ** -k[0], v0 * 2.0 ** -k[0]))
    r = mlmc.adaptive_mlmc(EPS, syn, _cost, nested=False, n0=1000)
    # Y_l = m0 2^-l: the bias test max(|Y_L|, |Y_{L-1}|/2, |Y_{L-2}|/4) / (2 - 1)
    # <= eps / sqrt(2) first holds at L = ceil(log2(m0 sqrt(2) / eps))
    L = math.ceil(math.log2(m0 * math.sqrt(2.0) / EPS))
    assert r["converged"] and r["levels"] == L + 1
    # the weak-error test runs after every round: the warm-up round of levels
    # 0..2, then one round per added level (which also carries the top-ups);
    # testing only once the top-ups are done would take one round more
    assert r["rounds"] == r["levels"] - 2
    assert abs(r["estimate"] - sum(m0 * 2.0 ** -l for l in range(L + 1))) < 1e-12
    # the final split: N_l = round8(ceil(2 eps^-2 sqrt(V_l / C_l) sum sqrt(V C))) (Sec. 3)
    V = [v0 * 2.0 ** -l for l in range(L + 1)]
    C = [2.0 ** l for l in range(L + 1)]
    opt = mlmc.optimal_samples(V, C, EPS)
    for (key, n, _, var), N in zip(r["terms"], opt):
        assert abs(var - V[key[0]]) <= 1e-12 * V[key[0]]
        assert n == max((1000 + 7) // 8 * 8, (int(N) + 7) // 8 * 8), (key, n, N)
    assert r["variance"] <= EPS * EPS / 2
    # the closed-form cost T = 2 eps^-2 (sum sqrt(V C))^2 of the split, to rounding
    spent = sum(n * C[key[0]] for key, n, _, _ in r["terms"])
    assert spent >= mlmc.predicted_cost(V, C, EPS) and spent <= 1.01 * mlmc.predicted_cost(V, C, EPS) + 8 * sum(C)


def test_nested_estimator_splits_between_its_two_terms():
    """theta- with fixed precision: two terms per level; the four-way term's
    variance is 2^-6 of the two-way one (Sec. 3's half precision + Kahan
    gap), its cost twice, so N_4 / N_2 = sqrt(2^-6 / 2) = 2^-3.5 per level."""
    m0, v0 = 0.3, 0.04

    def stats(k):
        l, kind = k[0], k[1]
        return (0.0, v0 * 2.0 ** (-l - 6)) if kind else (m0 * 2.0 ** -l, v0 * 2.0 ** -l)
    syn = Synthetic(stats)
    r = mlmc.adaptive_mlmc(EPS, syn, _cost, nested=True, prec=mlmc.F16, kahan=1, icdf=1, n0=64)
    L = math.ceil(math.log2(m0 * math.sqrt(2.0) / EPS))
    assert r["levels"] == L + 1
    n = {key: cnt for key, cnt, _, _ in r["terms"]}
    keys = [(l, kind, mlmc.F16, 1, 1) for l in range(L + 1) for kind in (0, 1)]
    opt = mlmc.optimal_samples([stats(k)[1] for k in keys], [_cost(k) for k in keys], EPS)
    for k, N in zip(keys, opt):
        assert n[k] == max(64, (int(N) + 7) // 8 * 8), (k, n[k], N)
    for l in range(3):     # where N is large the ratio is the closed form's
        n2, n4 = n[(l, 0, mlmc.F16, 1, 1)], n[(l, 1, mlmc.F16, 1, 1)]
        assert abs(n4 / n2 / 2.0 ** -3.5 - 1.0) < 1e-3, (l, n2, n4)
    assert r["variance"] <= EPS * EPS / 2


def test_per_level_choice_follows_the_scores_and_stops_trying_once_settled():
    """prec = -1: with these statistics the scores sqrt(v c) + sqrt(V C) make
    binary16 + Kahan the choice at levels 0 and 1 (cheaper two-way term,
    small four-way variance: 0.148 and 0.153 against binary32's 0.158) and
    binary32 from level 2 on (the growing binary16 floor: 0.164 against
    0.158); after two binary32 levels finer levels take binary32 without
    candidates.  The initial levels' candidates are drawn in one round."""
    m0, v0 = 0.3, 0.04

    def stats(k):
        l, kind, prec, kahan, icdf = k
        if icdf == 0:                                 # standard term: exact normals
            return m0 * 2.0 ** -l, v0 * 2.0 ** -l
        if kind == 0:
            return m0 * 2.0 ** -l, v0 * 2.0 ** -l * (1.0 + (0.0 if prec == mlmc.F32 else 2.0 ** (l - 8)))
        # the four-way rounding floor of binary16 grows with 2^l (Lemma 2.6),
        # Kahan lowers it; binary32 has none at these levels
        floor = 1e-12 if prec == mlmc.F32 else (4e-5 if kahan else 4e-4) * 2.0 ** l
        return 0.0, v0 * 2.0 ** (-l - 12) + floor

    def cost(k):
        l, kind, prec, kahan, icdf = k
        base = 1.0 if icdf == 0 else (0.5 if prec == mlmc.F16 else 0.6)
        return 2.0 ** l * (1.4 * base if kind else base)
    syn = Synthetic(stats)
    r = mlmc.adaptive_mlmc(EPS, syn, cost, nested=True, prec=-1, icdf=1, n0=64)
    ch = r["choice"]
    assert ch[0] == mlmc.CH_F16K and ch[1] == mlmc.CH_F16K and ch[2] == mlmc.CH_F32
    assert all(c == mlmc.CH_F32 for c in ch[2:])
    # candidates (more than one variant of a level in one round) only while unsettled
    def tried(rounds):
        out = set()
        for rnd in rounds:
            by_level = {}
            for q in rnd:
                by_level.setdefault(q[0][0], set()).add(q[0][2:])
            out |= {l for l, v in by_level.items() if len(v) > 1}
        return out
    assert r["levels"] > 5 and tried(syn.rounds) == {0, 1, 2, 3}
    # the initial levels' candidates share the first round: every variant of
    # levels 0..2 and their standard terms
    first = syn.rounds[0]
    assert {q[0][0] for q in first} == {0, 1, 2} and len(first) == 3 * 7
    assert tried(syn.rounds[1:]) == {3}
    # with trial_all every level is tried
    syn2 = Synthetic(stats)
    r2 = mlmc.adaptive_mlmc(EPS, syn2, cost, nested=True, prec=-1, icdf=1, n0=64, trial_all=True)
    assert tried(syn2.rounds) == set(range(r2["levels"])) and r2["choice"] == ch


def test_standard_term_is_chosen_where_it_is_cheaper():
    """If the nested pair costs more than the standard term at a level (its
    four-way variance is large), the level runs the standard term alone and
    its four-way slot stays empty."""
    def stats(k):
        l, kind, prec, kahan, icdf = k
        if kind == 1:
            return 0.0, 0.04 * 2.0 ** -l        # four-way as large as the two-way
        return 0.3 * 2.0 ** -l, 0.04 * 2.0 ** -l
    syn = Synthetic(stats)
    r = mlmc.adaptive_mlmc(EPS, syn, _cost, nested=True, prec=-1, icdf=1, n0=64)
    assert all(c == mlmc.CH_STANDARD for c in r["choice"])
    assert all(key[1] == 0 and key[4] == 0 for key, _, _, _ in r["terms"])


def test_moments_are_the_sample_mean_and_unbiased_variance():
    from fractions import Fraction
    xs = [0.5, -1.25, 3.0, 0.125, 2.0]
    s1, s2 = sum(xs), sum(x * x for x in xs)
    m, v = mlmc.moments(s1, s2, len(xs))
    fx = [Fraction(x) for x in xs]
    em = sum(fx) / 5
    assert Fraction(m) == em
    assert abs(Fraction(v) - sum((x - em) ** 2 for x in fx) / 4) < Fraction(1, 10 ** 14)
    assert mlmc.moments(2.0, 4.0, 1) == (2.0, 0.0)
