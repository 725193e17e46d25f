"""Pins of the oracle's Milstein scheme (named in the paper's conclusions as
the higher-order scheme for which low precision pays most, Sec. 5).

GBM: each fine step multiplies X by 1 + mu d + sigma sqrt(d) Z +
sigma^2 d (Z^2 - 1) / 2; the coarse step uses Z1 + Z2 with
(dW_c)^2 - 2 d = d ((Z1 + Z2)^2 - 2).  The level moments are products over
coarse steps of expectations of polynomials in the step normals
(oracle/mlmc.py: gbm_level_moments), exact for any joint law of (Z, Z~).
They are checked first against the independent Euler closed forms, then
used to pin the oracle's Monte Carlo; the O(delta^2) variance decay (strong
order 1) follows from them.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlmc

SEED = 1234


def _mean_var(s1, s2, n):
    return s1 / n, (s2 - s1 * s1 / n) / (n - 1)


def test_polynomial_moments_reduce_to_euler_closed_forms(pl_table):
    u = (2 * np.arange(1 << 23) + 1) * 2.0 ** -24
    z, zt = O.ndtri(u), O.approx_icdf(u, O.RV_TABLE, table=pl_table)
    grid = mlmc.grid_joint_moments(z, zt)
    m2, mc = grid(0, 2), grid(1, 1)

    def mom(a, b):        # the Euler closed forms take E Z^2 = 1 exactly (the grid's is 1 - 1.6e-7)
        return mlmc.gaussian_moment(a) if b == 0 else grid(a, b)
    for l in range(0, 7):
        a = mlmc.gbm_level_moments(l)
        b = mlmc.euler_twoway_moments(l)
        assert math.isclose(a[0], b[0], rel_tol=1e-12) and math.isclose(a[1], b[1], rel_tol=1e-9)
        a = mlmc.gbm_level_moments(l, mom, four=True)
        b = mlmc.euler_fourway_moments(l, m2, mc)
        # the four-way second moment is a sum of O(1) terms cancelling to 1e-9..1e-6:
        # both closed forms lose ~1e-14 absolute
        assert abs(a[0]) < 1e-15 and math.isclose(a[1], b[1], rel_tol=1e-6, abs_tol=5e-14)


def test_milstein_variance_decays_like_delta_squared():
    v = [mlmc.gbm_level_moments(l, milstein=True)[1] for l in range(2, 9)]
    slopes = np.diff(np.log2(v))
    assert np.all(np.abs(slopes + 2.0) < 0.15)
    # Euler for comparison: O(delta)
    v = [mlmc.gbm_level_moments(l)[1] for l in range(2, 9)]
    assert np.all(np.abs(np.diff(np.log2(v)) + 1.0) < 0.1)
    # the means do not change: E[Z^2 - 1] = 0
    for l in range(0, 6):
        assert math.isclose(mlmc.gbm_level_moments(l, milstein=True)[0], mlmc.gbm_level_moments(l)[0],
                            rel_tol=1e-9)


def test_milstein_level1_by_hand():
    mu, sigma = 0.07, 0.3
    sde = O.gbm(mu=mu, sigma=sigma, payoff=O.PAYOFF_X, scheme=1)
    tag = O.make_tag(O.KIND_STD, 1)
    # path 4 at l = 1: words 0, 1 of call 0 of counter path field 2
    w = O.philox4x32_10(O.counters([2], 0, tag), O.seed_key(SEED))[0]
    z = O.ndtri(O.uniforms(w))
    d = 0.5
    drift, diff, mil = mu * d, sigma * math.sqrt(d), 0.5 * sigma * sigma * d
    xf = 1.0
    for k in range(2):
        inc = (drift * xf + (diff * xf) * z[k]) + (mil * xf) * (z[k] * z[k] - 1.0)
        xf = xf + inc
    zc = z[0] + z[1]
    xc = 1.0 + (((mu * 2 * d) * 1.0 + (diff * 1.0) * zc) + (mil * 1.0) * (zc * zc - 2.0))
    out = O.twoway_paths(1, [4], O.variant(), sde, SEED, tag)[0]
    assert out[0] == xf and out[1] == xc


@pytest.mark.parametrize("l", [0, 1, 2, 3, 5])
def test_milstein_twoway_fp64_closed_form(l):
    n = 100000
    sde = O.gbm(payoff=O.PAYOFF_X, scheme=1)
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_STD, l), nthreads=4)
    m, v = _mean_var(s1, s2, n)
    em, ev = mlmc.gbm_level_moments(l, milstein=True)
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 0.06


@pytest.mark.parametrize("l", [0, 1, 3, 5])
def test_milstein_fourway_fp64_closed_form(l, pl_table):
    n = 100000
    u = (2 * np.arange(1 << 23) + 1) * 2.0 ** -24
    mom = mlmc.grid_joint_moments(O.ndtri(u), O.approx_icdf(u, O.RV_TABLE, table=pl_table))
    sde = O.gbm(payoff=O.PAYOFF_X, scheme=1)
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_FOUR, l), table=pl_table,
                          four=True, var2=O.variant(rv=O.RV_TABLE), nthreads=4)
    m, v = _mean_var(s1, s2, n)
    em, ev = mlmc.gbm_level_moments(l, mom, four=True, milstein=True)
    # unlike Euler the four-way mean is not zero: the bar paths' Milstein
    # term has mean sigma^2 d (E Z~^2 - 1) / 2 per step, which the four-way
    # difference corrects (so the nested sum still telescopes to E P^_L)
    ez2 = mom(2, 0) - mom(0, 2)
    assert em != 0.0 and abs(em) < 0.5 * 0.04 * ez2 * 1.2
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 0.1


def test_milstein_ou_is_euler(pl_table):
    """b' = 0 for OU: the Milstein scheme is the Euler scheme."""
    e = O.ou(2.0, 0.3, 0.5)
    m = O.ou(2.0, 0.3, 0.5)
    m.scheme = 1
    for var in (O.variant(), O.variant(prec=O.F16, kahan=True, rv=O.RV_TABLE)):
        a = O.twoway_paths(6, np.arange(200), var, e, SEED, O.make_tag(O.KIND_APPROX, 6), table=pl_table)
        b = O.twoway_paths(6, np.arange(200), var, m, SEED, O.make_tag(O.KIND_APPROX, 6), table=pl_table)
        assert np.array_equal(a, b)


def test_milstein_half_precision_rounding_model(pl_table):
    """Sec. 2.2 carries over: the binary16 rounding variance of the Milstein
    path still grows like N rho^2 without Kahan and is flat with it."""
    sde = O.gbm(payoff=O.PAYOFF_X, scheme=1)
    levels = np.arange(2, 11)
    out = {}
    for kahan in (False, True):
        row = []
        for l in levels:
            pr = O.rounding_pairs(l, 3000, 0, O.variant(prec=O.F16, kahan=kahan, rv=O.RV_TABLE), sde, SEED,
                                  O.make_tag(O.KIND_APPROX, l), table=pl_table)
            row.append(math.log2(np.var(pr[:, 0] - pr[:, 1])))
        out[kahan] = np.polyfit(levels, row, 1)[0]
    assert abs(out[False] - 1.0) < 0.3
    assert abs(out[True]) < 0.3
