"""Pins of the oracle's piecewise-cubic approximate inverse CDF (the
high-fidelity approximation of the Sec. 2.2 experiments) and of the Fig. 2
rounding-error observations it serves.

The cubic is the L2 projection of Phi^-1 onto cubics on each of the 16
dyadic intervals, so the residual is orthogonal to 1, s, s^2, s^3 on every
interval: checked with scipy's adaptive quadrature and scipy's ndtri, which
share nothing with the oracle's Gauss-Legendre construction.  The
working-precision evaluation is checked against IEEE arithmetic done by
numpy (binary32, binary16) and torch (bfloat16).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle as O
from oracle import table as T

SEED = 1234


@pytest.fixture(scope="module")
def cubic():
    return T.build_cubic_table()


def _g(d, s):
    return d[0] + s * (d[1] + s * (d[2] + s * d[3]))


def test_cubic_residual_orthogonal_to_cubics(cubic):
    for k in range(1, 17):
        A, B = T.cubic_map(k)
        a, b = T.interval_bounds(k)
        d = cubic[k - 1]
        for j in range(4):
            def res(v, j=j):
                s = A * v - B
                return (special.ndtri(v) - _g(d, s)) * s ** j
            def mag(v, j=j):
                return abs(special.ndtri(v) * (A * v - B) ** j)
            val, _ = integrate.quad(res, a, b, limit=400, epsabs=0, epsrel=1e-13)
            ref, _ = integrate.quad(mag, a, b, limit=400, epsabs=0, epsrel=1e-13)
            assert abs(val) <= 1e-11 * ref, (k, j, val, ref)


def test_cubic_l2_error_independent_quadrature(cubic):
    total = 0.0
    for k in range(1, 17):
        A, B = T.cubic_map(k)
        a, b = T.interval_bounds(k)
        d = cubic[k - 1]
        val, _ = integrate.quad(lambda v: (special.ndtri(v) - _g(d, A * v - B)) ** 2, a, b, limit=400,
                                epsabs=0, epsrel=1e-10)
        total += val
    assert math.isclose(2 * total, T.cubic_l2_error(cubic), rel_tol=1e-7)
    assert math.isclose(2 * total, 7.6923e-8, rel_tol=1e-4)
    # three orders of magnitude below the piecewise-linear table's error
    assert 2 * total < 2e-3 * T.l2_error(T.build_table())


def test_cubic_fp64_evaluation_and_symmetry(cubic, pl_table):
    u = (2 * np.arange(0, 1 << 23, 13) + 1) * 2.0 ** -24
    z = O.approx_icdf(u, O.RV_CUBIC, table=pl_table, cubic=cubic)
    v = np.minimum(u, 1 - u)
    k = np.minimum(np.maximum(-np.floor(np.log2(v)).astype(int) - 1, 1), 16)   # v in [2^-(k+1), 2^-k)
    A = np.where(k < 16, 2.0 ** (k + 2), 2.0 ** 17)
    B = np.where(k < 16, 3.0, 1.0)
    s = A * v - B
    assert np.all(np.abs(s) <= 1.0)
    d = cubic[k - 1]
    ref = d[:, 0] + s * (d[:, 1] + s * (d[:, 2] + s * d[:, 3]))
    ref = np.where(u > 0.5, -ref, ref)
    assert np.max(np.abs(z - ref)) < 1e-14
    assert np.array_equal(O.approx_icdf(1 - u, O.RV_CUBIC, table=pl_table, cubic=cubic), -z)


def _horner_ieee(d, s, dt):
    s = s.astype(dt)
    d = [np.asarray(d[:, j]).astype(dt) for j in range(4)]
    z = s * d[3]
    z = d[2] + z
    z = s * z
    z = d[1] + z
    z = s * z
    return d[0] + z


@pytest.mark.parametrize("prec,dt", [(O.F32, np.float32), (O.F16, np.float16)])
def test_cubic_working_precision_matches_ieee(prec, dt, cubic, pl_table):
    u = (2 * np.arange(0, 1 << 23, 29) + 1) * 2.0 ** -24
    u = u[u < 0.5]
    z = O.approx_icdf(u, O.RV_CUBIC, prec=prec, table=pl_table, cubic=cubic)
    k = np.minimum(np.maximum(-np.floor(np.log2(u)).astype(int) - 1, 1), 16)
    A = np.where(k < 16, 2.0 ** (k + 2), 2.0 ** 17)
    B = np.where(k < 16, 3.0, 1.0)
    ref = _horner_ieee(cubic[k - 1], A * u - B, dt).astype(np.float64)
    assert np.array_equal(z, ref)


def test_cubic_bf16_matches_torch(cubic, pl_table):
    torch = pytest.importorskip("torch")
    u = (2 * np.arange(0, 1 << 23, 31) + 1) * 2.0 ** -24
    u = u[u < 0.5]
    z = O.approx_icdf(u, O.RV_CUBIC, prec=O.BF16, table=pl_table, cubic=cubic)
    k = np.minimum(np.maximum(-np.floor(np.log2(u)).astype(int) - 1, 1), 16)
    A = np.where(k < 16, 2.0 ** (k + 2), 2.0 ** 17)
    B = np.where(k < 16, 3.0, 1.0)
    s = torch.from_numpy((A * u - B).astype(np.float32)).to(torch.bfloat16)    # exact in binary32
    d = [torch.from_numpy(cubic[k - 1][:, j]).to(torch.float32).to(torch.bfloat16) for j in range(4)]
    # float64 -> float32 -> bfloat16 double-rounds; compare the coefficients' roundings first
    for j in range(4):
        assert np.array_equal(d[j].to(torch.float64).numpy(), O.round_bits(cubic[k - 1][:, j], O.BF16)), j
    zz = s * d[3]
    zz = d[2] + zz
    zz = s * zz
    zz = d[1] + zz
    zz = s * zz
    zz = d[0] + zz
    assert np.array_equal(z, zz.to(torch.float64).numpy())


# ------------------------------------------------------------------ Fig. 2 (Sec. 2.2)


def _fig2_log2_var(prec, pbits, kahan, levels, cubic, pl_table, n=3000):
    """log2 Var(X^_N - X-_N): X^ exact normals in FP64, X- the cubic normals
    in working precision, the same uniforms (Sec. 2.2, Fig. 2)."""
    sde = O.gbm(payoff=O.PAYOFF_X)
    out = []
    for l in levels:
        p = O.fourway_paths(l, np.arange(n), O.variant(), O.variant(prec=prec, pbits=pbits, kahan=kahan,
                                                                     rv=O.RV_CUBIC),
                            sde, SEED, O.make_tag(O.KIND_FOUR, l), table=pl_table, cubic=cubic)
        out.append(math.log2(np.var(p[:, 0] - p[:, 2])))
    return np.array(out)


@pytest.mark.slow
def test_fig2_rounding_variance_by_mantissa_bits(cubic, pl_table):
    """Without Kahan: half grows like N rho^2 (slope 1 in l); bfloat16 sits
    2^6 higher (the rho^2 ratio); binary32 coincides with the FP64 bar path,
    i.e. its variance is the approximation error alone (O(1) in l); the
    16-bit intermediate precision coincides with it while the approximation
    error dominates (coarse levels).  The approximation error of the cubic
    is concentrated in the last interval (probability 2^-15), so the FP64
    curve is compared with the others sample by sample, not with its mean."""
    levels = np.arange(2, 11, 2)
    f16 = _fig2_log2_var(O.F16, 53, False, levels, cubic, pl_table)
    bf16 = _fig2_log2_var(O.BF16, 53, False, levels, cubic, pl_table)
    p17 = _fig2_log2_var(O.PBITS, 17, False, levels, cubic, pl_table)
    f32 = _fig2_log2_var(O.F32, 53, False, levels, cubic, pl_table)
    f64 = _fig2_log2_var(O.F64, 53, False, levels, cubic, pl_table)
    assert abs(np.polyfit(levels, f16, 1)[0] - 1.0) < 0.15
    assert abs(np.polyfit(levels, bf16, 1)[0] - 1.0) < 0.2
    assert np.all(np.abs((bf16 - f16) - 6.0) < 1.0)
    assert np.all(np.abs(f32 - f64) < 0.3)
    assert np.all(np.abs(p17[:2] - f64[:2]) < 1.0)
    assert np.all(p17 < f16 - 5.0)
    # the FP64 level: sigma^2 T E|Z - Z~|^2 E X^2, of which the sample
    # misses most of the last interval's share
    approx = math.log2(0.04 * 7.6923e-8 * 1.105)
    assert np.all((f64 > approx - 4.5) & (f64 < approx + 2.0))


@pytest.mark.slow
def test_fig2_kahan_removes_growth(cubic, pl_table):
    """With Kahan every precision is O(1) in l, and the half / bfloat16 gap
    is about 2^-6 (Sec. 2.3)."""
    levels = np.arange(2, 11, 2)
    f16 = _fig2_log2_var(O.F16, 53, True, levels, cubic, pl_table)
    bf16 = _fig2_log2_var(O.BF16, 53, True, levels, cubic, pl_table)
    for y in (f16, bf16):
        assert abs(np.polyfit(levels, y, 1)[0]) < 0.25
    assert abs(np.mean(f16 - bf16) + 6.0) < 1.0
