"""Pins of the oracle's inverse-CDF layer: exact Phi^-1, the piecewise-linear
table (Sec. 2.1), and the per-operation rounding emulation (Sec. 2.2)."""
import numpy as np
import pytest
import scipy.integrate as si
import scipy.special as sp
import torch

import oracle as O
from oracle import table as T

GRID = (2 * np.arange(1 << 23, dtype=np.float64) + 1) * 2.0 ** -24   # every 24-bit uniform


def test_ndtri_matches_library():
    p = np.concatenate([np.linspace(1e-12, 1 - 1e-12, 200001), 2.0 ** -np.arange(1, 60), GRID[::997]])
    x = O.ndtri(p)
    ref = sp.ndtri(p)
    assert np.max(np.abs(x - ref) / np.maximum(np.abs(ref), 1e-300)) < 4e-15


def test_ndtri_erfinv_identity():
    u = GRID[::4099]
    x = O.ndtri(u)
    assert np.allclose(x, np.sqrt(2.0) * sp.erfinv(2 * u - 1), rtol=1e-13, atol=1e-15)
    assert np.all(O.ndtri(u) == -O.ndtri(1 - u))          # exact antisymmetry on the grid


def test_table_normal_equations_independent_quadrature(pl_table):
    # On each interval the residual Phi^-1 - g is orthogonal to 1 and v (L2 fit);
    # checked with adaptive quadrature of scipy's ndtri, independent of the oracle.
    for k in range(1, 17):
        a, b = T.interval_bounds(k)
        c0, c1 = pl_table[k - 1]
        scale = abs(si.quad(lambda v: sp.ndtri(v), a, b, limit=200)[0]) + 1e-300
        r0 = si.quad(lambda v: sp.ndtri(v) - c0 - c1 * v, a, b, limit=200, epsabs=1e-20)[0]
        r1 = si.quad(lambda v: (sp.ndtri(v) - c0 - c1 * v) * v, a, b, limit=200, epsabs=1e-24)[0]
        assert abs(r0) < 1e-9 * scale
        assert abs(r1) < 1e-9 * scale * b


def test_table_l2_invariants(pl_table):
    z = O.ndtri(GRID)
    zt = O.approx_icdf(GRID, O.RV_TABLE, table=pl_table)
    # mirrored: exactly zero mean, exactly antisymmetric
    assert zt.sum() == 0.0
    assert np.all(zt == -zt[::-1])
    # L2 projection: E[Z~^2] = E[Z Z~] holds for the continuous uniform; the
    # 2^23-point grid average departs from it by the grid's own quadrature
    # error (largest on the last interval, where the grid stops at 2^-24)
    m2, mc = np.mean(zt * zt), np.mean(z * zt)
    assert abs(m2 - mc) < 2e-7
    assert abs(m2 - 0.99995838) < 2e-7
    # continuous E|Z - Z~|^2 of the 16-interval fit
    assert abs(T.l2_error(pl_table) - 4.162e-5) < 0.002e-5
    # compact support (Fig. 1): |Z~| bounded by the end value of the last interval
    assert np.abs(zt).max() < 4.71


def test_table_interval_edges(pl_table):
    # v at an exact power of two belongs to the interval above it: [2^-(k+1), 2^-k)
    for k in range(1, 16):
        v = 2.0 ** -(k + 1)
        got = O.approx_icdf([v], O.RV_TABLE, table=pl_table)[0]
        c0, c1 = pl_table[k - 1]
        assert got == c0 + c1 * v
    v = 2.0 ** -20
    assert O.approx_icdf([v], O.RV_TABLE, table=pl_table)[0] == pl_table[15, 0] + pl_table[15, 1] * v


@pytest.mark.parametrize("prec,np_t", [(O.F16, np.float16), (O.F32, np.float32)])
def test_rounding_matches_ieee_casts(prec, np_t):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(200000) * 10.0 ** rng.integers(-9, 6, 200000),
                        [65504.0, 65519.99, 65520.0, 2.0 ** -24, 3 * 2.0 ** -26, 1e-30, -0.0]])
    with np.errstate(over="ignore"):
        ref = x.astype(np_t).astype(np.float64)
    assert np.array_equal(O.round_bits(x, prec), ref)


def test_rounding_bf16_matches_torch():
    # torch converts float64 -> bfloat16 through float32, so the library
    # reference is exact only for float32-representable inputs
    rng = np.random.default_rng(1)
    x = rng.standard_normal(100000) * 10.0 ** rng.integers(-30, 30, 100000)
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bits(x, O.BF16), ref)


def test_pbits_rounding_ties_to_even():
    # 1 + 2^-p halfway cases with a p-bit significand go to the even neighbour
    for p in (7, 10, 16, 23):
        x = np.array([1 + 2.0 ** -p, 1 + 3 * 2.0 ** -p])
        y = O.round_bits(x, O.PBITS, pbits=p)
        assert y.tolist() == [1.0, 1 + 4 * 2.0 ** -p]


def test_half_table_evaluation_operation_order(pl_table):
    # z = R(R(c0) + R(R(c1) R(v))) in binary16, u > 1/2 mirrored
    u = np.array([0.3, 0.9, 2.0 ** -24, 1 - 2.0 ** -20])
    got = O.approx_icdf(u, O.RV_TABLE, prec=O.F16, table=pl_table)
    h = np.float16
    for ui, gi in zip(u, got):
        v = min(ui, 1 - ui)
        k = min(max(-int(np.floor(np.log2(v))) - 1, 1), 16)
        c0, c1 = h(pl_table[k - 1, 0]), h(pl_table[k - 1, 1])
        z = h(c0 + h(c1 * h(v)))
        assert gi == (float(z) if ui <= 0.5 else -float(z))
