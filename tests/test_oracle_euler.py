"""Pins of the oracle's path layer: Euler-Maruyama GBM/OU, the two-way and
four-way differences (Sec. 3), Kahan summation (Sec. 2.3) and the
rounding-error model (Sec. 2.2, Lemma 2.6)."""
from fractions import Fraction
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import mlmc

SEED = 1234
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, value, _ = line.split()
            vals[name] = float(value)
    return vals


def _mean_var(s1, s2, n):
    m = s1 / n
    return m, (s2 - s1 * s1 / n) / (n - 1)


@pytest.mark.parametrize("l", [0, 1, 2, 3, 5])
def test_twoway_fp64_discrete_closed_form(l):
    n = 100000
    sde = O.gbm(payoff=O.PAYOFF_X)
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_STD, l), nthreads=4)
    m, v = _mean_var(s1, s2, n)
    em, ev = mlmc.euler_twoway_moments(l)
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 4 * math.sqrt(2.0 / n) * 3      # kurtosis allowance


@pytest.mark.parametrize("l", [0, 1, 3, 5])
def test_fourway_fp64_discrete_closed_form(l, pl_table):
    n = 100000
    u = (2 * np.arange(1 << 23) + 1) * 2.0 ** -24
    z, zt = O.ndtri(u), O.approx_icdf(u, O.RV_TABLE, table=pl_table)
    m2, mc = np.mean(zt * zt), np.mean(z * zt)
    sde = O.gbm(payoff=O.PAYOFF_X)
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_FOUR, l), table=pl_table,
                          four=True, var2=O.variant(rv=O.RV_TABLE), nthreads=4)
    m, v = _mean_var(s1, s2, n)
    em, ev = mlmc.euler_fourway_moments(l, m2, mc)
    assert em == 0.0 or abs(em) < 1e-15
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 0.1


def test_per_path_components_consistent(pl_table):
    sde = O.gbm(payoff=O.PAYOFF_CALL)
    idx = np.arange(50, dtype=np.uint64)
    two = O.twoway_paths(4, idx, O.variant(rv=O.RV_TABLE), sde, SEED, O.make_tag(O.KIND_APPROX, 4), table=pl_table)
    assert np.allclose(two[:, 2], two[:, 0] - two[:, 1], rtol=0, atol=0)
    four = O.fourway_paths(4, idx, O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, O.make_tag(O.KIND_FOUR, 4),
                           table=pl_table)
    assert np.array_equal(four[:, 4], (four[:, 0] - four[:, 1]) - (four[:, 2] - four[:, 3]))
    # the four-way bar path is the same computation as the two-way approximate path on the same counters
    two_same = O.twoway_paths(4, idx, O.variant(rv=O.RV_TABLE), sde, SEED, O.make_tag(O.KIND_FOUR, 4), table=pl_table)
    assert np.array_equal(four[:, 2:4], two_same[:, 0:2])


def test_level0_single_step_by_hand():
    # l = 0: one step X1 = x0 + mu x0 T + sigma x0 sqrt(T) Z; the two-way
    # paths 12 .. 15 share call 0 of counter path field 3, path 12 + k taking
    # word k; so do the four-way paths 12 .. 15 (both the exact-normal and the
    # approximate path of a sample take the same word)
    sde = O.gbm(mu=0.05, sigma=0.2, payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_STD, 0)
    w = O.philox4x32_10(O.counters([3], 0, tag), O.seed_key(SEED))[0]
    z = O.ndtri(O.uniforms(w))
    out = O.twoway_paths(0, [12, 13, 14, 15], O.variant(), sde, SEED, tag)
    for k in range(4):
        assert out[k, 1] == 0.0 and out[k, 2] == out[k, 0]
        assert abs(out[k, 0] - (1 + 0.05 + 0.2 * z[k])) < 1e-15
    # path 11 is the last of the previous call (field 2, word 3)
    w2 = O.philox4x32_10(O.counters([2], 0, tag), O.seed_key(SEED))[0]
    out = O.twoway_paths(0, [11], O.variant(), sde, SEED, tag)
    assert abs(out[0, 0] - (1 + 0.05 + 0.2 * O.ndtri(O.uniforms(w2[3:]))[0])) < 1e-15
    four = O.fourway_paths(0, [12, 13, 14, 15], O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, tag)
    for k in range(4):
        assert abs(four[k, 0] - (1 + 0.05 + 0.2 * z[k])) < 1e-15
    # four-way path 11: word 3 of field 2, as the two-way path 11
    four = O.fourway_paths(0, [11], O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, tag)
    assert abs(four[0, 0] - (1 + 0.05 + 0.2 * O.ndtri(O.uniforms(w2[3:]))[0])) < 1e-15


def test_level1_paths_share_a_call_by_hand():
    # l = 1: paths 4 and 5 share call 0 of counter path field 2: path 4 takes
    # words 0, 1 and path 5 words 2, 3; the coarse step adds the pair
    mu, sigma = 0.07, 0.3
    sde = O.gbm(mu=mu, sigma=sigma, payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_STD, 1)
    w = O.philox4x32_10(O.counters([2], 0, tag), O.seed_key(SEED))[0]
    z = O.ndtri(O.uniforms(w))
    out = O.twoway_paths(1, [4, 5], O.variant(), sde, SEED, tag)
    d = 0.5
    for k in range(2):
        za, zb = z[2 * k], z[2 * k + 1]
        xf = 1.0
        for zz in (za, zb):
            xf = xf + (mu * d * xf + (sigma * math.sqrt(d) * xf) * zz)
        xc = 1.0 + (mu * 2 * d * 1.0 + (sigma * math.sqrt(d) * 1.0) * (za + zb))
        assert out[k, 0] == xf and out[k, 1] == xc
    # and the four-way paths of the same counters share the words the same way
    four = O.fourway_paths(1, [4, 5], O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, tag)
    assert np.array_equal(four[:, 0:2], out[:, 0:2])


def test_level2_coarse_uses_pairwise_sums():
    # l = 2: fine 4 steps of T/4; coarse 2 steps of T/2 with dW_c = sqrt(T/4)(Z1 + Z2)
    mu, sigma = 0.07, 0.3
    sde = O.gbm(mu=mu, sigma=sigma, payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_STD, 2)
    w = O.philox4x32_10(O.counters([3], 0, tag), O.seed_key(SEED))[0]
    z = O.ndtri(O.uniforms(w))
    d = 0.25
    xf = 1.0
    for k in range(4):
        xf = xf + (mu * d * xf + sigma * math.sqrt(d) * xf * z[k])
    xc = 1.0
    for k in range(2):
        xc = xc + (mu * 2 * d * xc + sigma * math.sqrt(d) * xc * (z[2 * k] + z[2 * k + 1]))
    out = O.twoway_paths(2, [3], O.variant(), sde, SEED, tag)[0]
    assert abs(out[0] - xf) < 1e-14 and abs(out[1] - xc) < 1e-14


def test_level3_five_uniforms_per_call_by_hand():
    # l = 3: 8 fine steps from the path's own calls, five uniforms each: the
    # four words, then the spare word (the low bytes of x, y, z as bits
    # 8..15, 16..23, 24..31); steps 0..4 from call 0, steps 5..7 from the
    # words 0..2 of call 1
    mu, sigma = 0.07, 0.3
    sde = O.gbm(mu=mu, sigma=sigma, payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_STD, 3)
    path = 5
    c0 = O.philox4x32_10(O.counters([path], 0, tag), O.seed_key(SEED))[0].astype(np.uint64)
    c1 = O.philox4x32_10(O.counters([path], 1, tag), O.seed_key(SEED))[0]
    spare = ((c0[0] & 0xFF) << 8) | ((c0[1] & 0xFF) << 16) | ((c0[2] & 0xFF) << 24)
    words = [int(x) for x in c0] + [int(spare)] + [int(x) for x in c1[:3]]
    z = O.ndtri(O.uniforms(np.array(words, dtype=np.uint32)))
    d = 0.125
    xf = 1.0
    for k in range(8):
        xf = xf + (mu * d * xf + sigma * math.sqrt(d) * xf * z[k])
    xc = 1.0
    for k in range(4):
        xc = xc + (mu * 2 * d * xc + sigma * math.sqrt(d) * xc * (z[2 * k] + z[2 * k + 1]))
    out = O.twoway_paths(3, [path], O.variant(), sde, SEED, tag)[0]
    assert abs(out[0] - xf) < 1e-14 and abs(out[1] - xc) < 1e-14
    # the four-way paths use the same uniforms (hat: exact normals)
    four = O.fourway_paths(3, [path], O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, tag)[0]
    assert four[0] == out[0] and four[1] == out[1]


def test_ou_mean_reversion_closed_form():
    # Euler OU: E X_{n+1} = m + (1 - theta delta)(E X_n - m); Var via (1 - theta delta)^2 V + s^2 delta
    theta, m, s, l = 2.0, 0.5, 0.4, 4
    sde = O.ou(theta, m, s, x0=1.0)
    n = 100000
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_STD, l), nthreads=4)
    # the two-way D = X_f - X_c; check E D exactly from the two linear recursions
    d = 2.0 ** -l
    ef = m + (1 - theta * d) ** (2 ** l) * (1.0 - m)
    ec = m + (1 - 2 * theta * d) ** (2 ** (l - 1)) * (1.0 - m)
    mean, var = _mean_var(s1, s2, n)
    assert abs(mean - (ef - ec)) < 4 * math.sqrt(var / n)


def test_terminal_law_and_call_telescoping(pl_table):
    # sum of level means (l = 0..6) of the discounted call converges to Black-Scholes
    sde = O.gbm(payoff=O.PAYOFF_CALL)
    total, var_total = 0.0, 0.0
    for l in range(7):
        n = 40000
        s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_STD, l), nthreads=4)
        m, v = _mean_var(s1, s2, n)
        total += m
        var_total += v / n
    bs = mlmc.bs_call()
    assert abs(bs - 0.1045058357) < 1e-9
    # weak bias of Euler at l = 6 is O(2^-6 * 0.01); allow 4 s.e. + 5e-4
    assert abs(total - bs) < 4 * math.sqrt(var_total) + 5e-4
    em, ev = mlmc.gbm_terminal()
    assert abs(em - 1.0512710964) < 1e-9 and abs(ev - 0.0451028808) < 1e-9


def test_kahan_exact_rational_bound():
    # Algorithm 1 in binary16 on an ill-conditioned sequence: error within
    # (2 rho + O(N rho^2)) sum |x| (Sec. 2.3), far below plain summation.
    rng = np.random.default_rng(3)
    x = O.round_bits(np.concatenate([[1.0], rng.uniform(0, 2.0 ** -12, 2000)]), O.F16)
    exact = sum(Fraction(v) for v in x)
    k16 = O.kahan_sum(x, O.F16)
    plain = np.float16(0)
    for v in x:
        plain = np.float16(plain + np.float16(v))
    rho = 2.0 ** -11
    err_k = abs(Fraction(k16) - exact)
    bound = (2 * rho + x.size * rho * rho) * sum(abs(Fraction(v)) for v in x)
    assert err_k <= bound
    assert err_k * 20 < abs(Fraction(float(plain)) - exact)


def test_kahan_exact_on_tiny_cases():
    # cases whose exact sum is representable: Kahan recovers it exactly
    x = [1.0, 2.0 ** -11, 2.0 ** -11, -1.0]
    assert O.kahan_sum(x, O.F16) == 2.0 ** -10
    x = [2048.0, 1.0, 1.0, 1.0, 1.0]
    assert O.kahan_sum(x, O.F16) == 2052.0


def _rounding_log2_vars(prec, kahan, levels, n, pl_table):
    sde = O.gbm(payoff=O.PAYOFF_X)
    out = []
    for l in levels:
        pr = O.rounding_pairs(l, n, 0, O.variant(prec=prec, kahan=kahan, rv=O.RV_TABLE), sde, SEED,
                              O.make_tag(O.KIND_APPROX, l), table=pl_table)
        out.append(math.log2(np.var(pr[:, 0] - pr[:, 1])))
    return np.array(out)


def test_rounding_model_slopes(pl_table):
    """Lemma 2.6: without Kahan the half rounding variance grows like N rho^2
    (slope +1); with Kahan it is O(1) (slope 0); the bfloat16/half gap with
    Kahan is about 2^-6 (Sec. 2.3)."""
    pv = _paper_values()
    levels = np.arange(2, 11)
    no_k = _rounding_log2_vars(O.F16, False, levels, 3000, pl_table)
    with_k = _rounding_log2_vars(O.F16, True, levels, 3000, pl_table)
    bf_k = _rounding_log2_vars(O.BF16, True, levels, 3000, pl_table)
    slope_no = np.polyfit(levels, no_k, 1)[0]
    slope_k = np.polyfit(levels, with_k, 1)[0]
    assert abs(slope_no - pv["half_no_kahan_log2_slope"]) < 0.3
    assert abs(slope_k - pv["half_kahan_log2_slope"]) < 0.3
    gap = np.mean(with_k - bf_k)
    assert abs(gap - pv["kahan_half_bf16_log2_gap"]) < 1.0


def test_leading_rounding_error_is_zero_mean(pl_table):
    """Lemma 2.4: the leading error eta of X (+) R(beta) has mean O(rho^2),
    far below its mean absolute size O(rho)."""
    rng = np.random.default_rng(11)
    alpha = O.round_bits(rng.uniform(1.0, 2.0, 400000), O.F16)
    beta = O.round_bits(0.2 * 2.0 ** -5 * O.approx_icdf(rng.uniform(size=400000), O.RV_TABLE, table=pl_table),
                        O.F16)
    eta = O.round_bits(alpha + beta, O.F16) - (alpha + beta)
    assert abs(eta.mean()) < 0.02 * np.abs(eta).mean()


def test_twoway_double_variance_slope():
    pv = _paper_values()
    sde = O.gbm(payoff=O.PAYOFF_X)
    ls = np.arange(2, 8)
    ev = [mlmc.euler_twoway_moments(int(l))[1] for l in ls]
    assert abs(np.polyfit(ls, np.log2(ev), 1)[0] - pv["twoway_double_log2_slope"]) < 0.05
