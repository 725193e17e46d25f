"""Pins of the oracle's 16-bit uniform reading (RV_TABLE16).

The paper leaves the random-number generator open.  The library offers, as
a stated design choice, approximate normals drawn from 16-bit uniforms: two
per Philox word on the two-way approximate paths, and the 16-bit cell
centre q16(U) of the shared 24-bit uniform on the four-way bar paths, so
that both estimators see the same law of Z~ and the telescoping sum of
Sec. 3 keeps its expectation.  These tests pin that reading with brute
force over the grids, a by-hand path and the discrete Euler closed forms.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlmc

SEED = 1234


def _grid24():
    return (2 * np.arange(1 << 23) + 1) * 2.0 ** -24


def test_q16_pushes_24bit_grid_onto_16bit_grid():
    q = O.q16(_grid24())
    vals, counts = np.unique(q, return_counts=True)
    assert vals.size == 1 << 16 and np.all(counts == 128)
    assert np.array_equal(vals, O.uniforms16(np.arange(1 << 16)))
    # symmetric about 1/2, never 0 or 1
    assert np.array_equal(np.sort(1.0 - vals), vals)
    assert vals[0] == 2.0 ** -17 and vals[-1] == 1 - 2.0 ** -17


def test_q16_cell_centres_by_definition():
    u = np.array([2.0 ** -24, 2.0 ** -16 - 2.0 ** -24, 2.0 ** -16 + 2.0 ** -24, 0.5 - 2.0 ** -24, 0.5 + 2.0 ** -24,
                  0.3, 1 - 2.0 ** -24])
    cell = np.floor(u * 65536)
    assert np.array_equal(O.q16(u), (cell + 0.5) / 65536)
    assert np.array_equal(O.uniforms16([0, 0x8000, 0xFFFF, 0x1_0005]),
                          np.array([0.5, 32768.5, 65535.5, 5.5]) / 65536)


def test_table16_close_to_table_and_antisymmetric(pl_table):
    """Every dyadic interval edge 2^-k (k <= 16) is a cell edge, so a cell
    never straddles two linear pieces: |Z~(u) - Z~(q16 u)| = |c1| |v - v16|
    <= max|c1| 2^-17 over the whole 24-bit grid."""
    u = _grid24()
    zt = O.approx_icdf(u, O.RV_TABLE, table=pl_table)
    z16 = O.approx_icdf(u, O.RV_TABLE16, table=pl_table)
    c1max = np.abs(pl_table.reshape(16, 2)[:, 1]).max()
    assert np.max(np.abs(zt - z16)) <= c1max * 2.0 ** -17 * (1 + 1e-12)
    assert np.array_equal(z16[::-1], -z16)
    assert np.sum(z16) == 0.0
    # the same law whether Z~ comes from q16 of a 24-bit uniform or a 16-bit one
    g16 = O.approx_icdf(O.uniforms16(np.arange(1 << 16)), O.RV_TABLE, table=pl_table)
    assert math.isclose(np.mean(z16 * z16), np.mean(g16 * g16), rel_tol=1e-13)
    # the quantisation adds a few per cent to the approximation error
    # E|Z - Z~|^2 (4.160e-5 -> 4.277e-5), almost all of it from the last
    # cell (0, 2^-16), where Phi^-1 varies fastest
    z = O.ndtri(u)
    e24, e16 = np.mean((z - zt) ** 2), np.mean((z - z16) ** 2)
    assert e24 < e16 < 1.05 * e24
    tail = u < 2.0 ** -16
    d_tail = np.sum((z - z16)[tail] ** 2 - (z - zt)[tail] ** 2) / u.size
    assert 0.5 * (e16 - e24) < 2 * d_tail


def test_twoway_table16_level3_by_hand(pl_table):
    """l = 3: the 8 fine steps take the low then the high half of words
    0, 1, 2, 3 of call 0; coarse steps add consecutive pairs."""
    mu, sigma = 0.07, 0.3
    sde = O.gbm(mu=mu, sigma=sigma, payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_APPROX, 3)
    w = O.philox4x32_10(O.counters([11], 0, tag), O.seed_key(SEED))[0]
    halves = np.array([[x & 0xFFFF, x >> 16] for x in w.tolist()]).ravel()
    z = O.approx_icdf(O.uniforms16(halves), O.RV_TABLE, table=pl_table)
    d = 0.125
    drift, diff = mu * d, sigma * math.sqrt(d)
    xf = 1.0
    for k in range(8):
        xf = xf + (drift * xf + (diff * xf) * z[k])
    xc, drift_c = 1.0, mu * 2 * d
    for k in range(4):
        xc = xc + (drift_c * xc + (diff * xc) * (z[2 * k] + z[2 * k + 1]))
    out = O.twoway_paths(3, [11], O.variant(rv=O.RV_TABLE16), sde, SEED, tag, table=pl_table)[0]
    assert out[0] == xf and out[1] == xc and out[2] == xf - xc


def test_twoway_table16_level4_second_call(pl_table):
    """l = 4: steps 8..15 come from call 1."""
    sde = O.gbm(payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_APPROX, 4)
    w = np.concatenate([O.philox4x32_10(O.counters([5], j, tag), O.seed_key(SEED))[0] for j in (0, 1)])
    halves = np.array([[x & 0xFFFF, x >> 16] for x in w.tolist()]).ravel()
    z = O.approx_icdf(O.uniforms16(halves), O.RV_TABLE, table=pl_table)
    d = 1 / 16
    drift, diff = 0.05 * d, 0.2 * math.sqrt(d)
    xf = 1.0
    for k in range(16):
        xf = xf + (drift * xf + (diff * xf) * z[k])
    out = O.twoway_paths(4, [5], O.variant(rv=O.RV_TABLE16), sde, SEED, tag, table=pl_table)[0]
    assert out[0] == xf


@pytest.mark.parametrize("l", [0, 1, 2, 3, 5])
def test_twoway_table16_fp64_closed_form(l, pl_table):
    n = 100000
    g16 = O.approx_icdf(O.uniforms16(np.arange(1 << 16)), O.RV_TABLE, table=pl_table)
    m2 = np.mean(g16 * g16)
    sde = O.gbm(payoff=O.PAYOFF_X)
    s1, s2 = O.level_sums(l, n, 0, O.variant(rv=O.RV_TABLE16), sde, SEED, O.make_tag(O.KIND_APPROX, l),
                          table=pl_table, nthreads=4)
    m = s1 / n
    v = (s2 - s1 * s1 / n) / (n - 1)
    em, ev = mlmc.euler_twoway_moments(l, m2=m2)
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 0.05


@pytest.mark.parametrize("l", [0, 1, 3, 5])
def test_fourway_table16_fp64_closed_form(l, pl_table):
    """Four-way with the bar paths on Z~(q16(U)): E D = 0 and the variance
    of the closed form with E Z~^2, E Z Z~ over the 24-bit grid."""
    n = 100000
    u = _grid24()
    z, zt = O.ndtri(u), O.approx_icdf(u, O.RV_TABLE16, table=pl_table)
    m2, mc = np.mean(zt * zt), np.mean(z * zt)
    sde = O.gbm(payoff=O.PAYOFF_X)
    s1, s2 = O.level_sums(l, n, 0, O.variant(), sde, SEED, O.make_tag(O.KIND_FOUR, l), table=pl_table,
                          four=True, var2=O.variant(rv=O.RV_TABLE16), nthreads=4)
    m = s1 / n
    v = (s2 - s1 * s1 / n) / (n - 1)
    em, ev = mlmc.euler_fourway_moments(l, m2, mc)
    assert abs(em) < 1e-15
    assert abs(m - em) < 4 * math.sqrt(ev / n)
    assert abs(v / ev - 1) < 0.1


def test_fourway_bar_is_table_at_q16(pl_table):
    """The four-way bar paths are the approximate paths driven by the
    per-step q16 of the shared 24-bit uniforms (computed here from the
    words), while the hat paths still see the 24-bit uniforms."""
    sde = O.gbm(payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_FOUR, 2)
    w = O.philox4x32_10(O.counters([9], 0, tag), O.seed_key(SEED))[0]
    u = O.uniforms(w)
    zb = O.approx_icdf(O.q16(u), O.RV_TABLE, table=pl_table)
    d = 0.25
    xf = 1.0
    for k in range(4):
        xf = xf + (0.05 * d * xf + (0.2 * math.sqrt(d) * xf) * zb[k])
    out = O.fourway_paths(2, [9], O.variant(), O.variant(rv=O.RV_TABLE16), sde, SEED, tag, table=pl_table)[0]
    assert out[2] == xf
    hat = O.fourway_paths(2, [9], O.variant(), O.variant(rv=O.RV_TABLE), sde, SEED, tag, table=pl_table)[0]
    assert out[0] == hat[0] and out[1] == hat[1]


@pytest.mark.parametrize("l", [0, 1, 2])
def test_twoway_table16_coarse_levels_share_a_call(l, pl_table):
    """l <= 2: the S = 8 / 2^l paths S k .. S k + S - 1 share call 0 of
    counter path field k; path p takes the halves (p mod S) 2^l ..
    (p mod S) 2^l + 2^l - 1, low half of each word first."""
    sde = O.gbm(payoff=O.PAYOFF_X)
    tag = O.make_tag(O.KIND_APPROX, l)
    w = O.philox4x32_10(O.counters([10], 0, tag), O.seed_key(SEED))[0]
    halves = np.array([[x & 0xFFFF, x >> 16] for x in w.tolist()]).ravel()
    z = O.approx_icdf(O.uniforms16(halves), O.RV_TABLE, table=pl_table)
    S = 8 >> l
    out = O.twoway_paths(l, list(range(10 * S, 11 * S)), O.variant(rv=O.RV_TABLE16), sde, SEED, tag,
                         table=pl_table)
    n = 1 << l
    d = 1.0 / n
    for k in range(S):
        xf = 1.0
        for zz in z[k * n:(k + 1) * n]:
            xf = xf + (0.05 * d * xf + (0.2 * math.sqrt(d) * xf) * zz)
        assert out[k, 0] == xf
