"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bit-exact: Philox words, uniforms, the binary32/binary16/bfloat16 table coefficients,
the approximate normals, and every per-path output of the low-precision
("bar") paths against the oracle's per-operation rounding emulation.
Within tolerance: exact-normal FP32 paths against FP64 (1e-5 relative), and
FP16 + Kahan paths against FP64 (2e-3 relative), per path, with
|error| <= tol * max(1, |P_fine|).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2012_09739_gb300 as M  # noqa: E402

SEED = 1234
TOL32, TOL16K = 1e-5, 2e-3


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def _orc_sde(p):
    return O.SDE(p.sde, p.payoff, p.p0, p.p1, p.p2, p.x0, p.T, p.K, p.disc, p.scheme)


def gpu_paths(four, l, N, prec, kahan, icdf, params, seed=SEED, offset=0):
    w = 5 if four else 3
    out = torch.empty(N * w, dtype=torch.float32, device=_dev())
    M.mlmc_level_paths(four, l, N, prec, kahan, icdf, params, seed, offset, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(N, w)


_OPREC = {M.MLMC_F32: O.F32, M.MLMC_F16: O.F16, M.MLMC_BF16: O.BF16}


def _bar_variant(prec, kahan, icdf=O.RV_TABLE):
    return O.variant(prec=_OPREC[prec], kahan=kahan, rv=icdf)


def _kind_tag(four, icdf, l):
    kind = O.KIND_FOUR if four else (O.KIND_STD if icdf == M.MLMC_ICDF_EXACT else O.KIND_APPROX)
    return O.make_tag(kind, l)


# ------------------------------------------------------------------ RNG


def test_philox_bitexact():
    dev = _dev()
    rng = np.random.default_rng(0)
    n = 100003
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0], key[0] = 0, 0
    ctr[1], key[1] = 0xFFFFFFFF, 0xFFFFFFFF
    out = torch.empty((n, 4), dtype=torch.int32, device=dev)
    M.mlmc_philox4x32_10(torch.from_numpy(ctr.view(np.int32)).to(dev), torch.from_numpy(key.view(np.int32)).to(dev),
                         out)
    torch.cuda.synchronize()
    assert np.array_equal(_u32(out), O.philox4x32_10(ctr, key))


def test_uniforms_bitexact():
    dev = _dev()
    w = np.random.default_rng(1).integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    w[:4] = [0, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF]
    u = torch.empty(w.size, dtype=torch.float32, device=dev)
    M.mlmc_uniforms(torch.from_numpy(w.view(np.int32)).to(dev), u)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy().astype(np.float64), O.uniforms(w))


# ------------------------------------------------------------------ table and inverse CDFs


def test_table_matches_oracle(pl_table):
    _dev()
    c64, c32, c16, cbf = M.mlmc_icdf_table()
    assert np.allclose(c64, pl_table, rtol=1e-11, atol=0)
    assert np.array_equal(c32.astype(np.float64), O.round_bits(pl_table, O.F32).reshape(16, 2))
    assert np.array_equal(c16.view(np.float16).astype(np.float64), O.round_bits(pl_table, O.F16).reshape(16, 2))
    bf = (cbf.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(bf, O.round_bits(pl_table, O.BF16).reshape(16, 2))


def _z_host(z, prec):
    if prec == M.MLMC_BF16:
        return (z.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return z.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("prec", [M.MLMC_F32, M.MLMC_F16, M.MLMC_BF16])
def test_approx_icdf_table_bitexact(prec, pl_table):
    dev = _dev()
    rng = np.random.default_rng(2)
    u = np.concatenate([(2 * rng.integers(0, 1 << 23, 200000) + 1) * 2.0 ** -24,
                        [2.0 ** -24, 1 - 2.0 ** -24, 0.5 - 2.0 ** -24, 0.25, 0.75, 2.0 ** -16, 2.0 ** -17,
                         3e-9, 0.5]]).astype(np.float32)
    ut = torch.from_numpy(u).to(dev)
    z = torch.empty(u.size, dtype=torch.float32 if prec == M.MLMC_F32 else torch.int16, device=dev)
    M.approx_icdf(ut, z, M.MLMC_ICDF_TABLE, prec)
    torch.cuda.synchronize()
    ref = O.approx_icdf(u.astype(np.float64), O.RV_TABLE, prec=_OPREC[prec], table=pl_table)
    if prec == M.MLMC_F16:
        got = z.cpu().numpy().view(np.float16).astype(np.float64)
    else:
        got = _z_host(z, prec)
    assert np.array_equal(got, ref)


def test_approx_icdf_exact_bf16_is_rounded_fp32():
    """bfloat16 output of the exact inverse CDF is the round-to-nearest-even
    bfloat16 of the binary32 value."""
    dev = _dev()
    u = ((2 * np.arange(0, 1 << 23, 3) + 1) * 2.0 ** -24).astype(np.float32)
    ut = torch.from_numpy(u).to(dev)
    z32 = torch.empty(u.size, dtype=torch.float32, device=dev)
    zb = torch.empty(u.size, dtype=torch.int16, device=dev)
    M.approx_icdf(ut, z32, M.MLMC_ICDF_EXACT, M.MLMC_F32)
    M.approx_icdf(ut, zb, M.MLMC_ICDF_EXACT, M.MLMC_BF16)
    torch.cuda.synchronize()
    assert np.array_equal(_z_host(zb, M.MLMC_BF16), O.round_bits(z32.cpu().numpy().astype(np.float64), O.BF16))


def test_exact_icdf_whole_grid_within_3_ulp():
    """The kernels' exact normal (per-binade polynomial) at every point of the
    24-bit uniform grid against the oracle's FP64 inverse CDF: within 3 ulp
    of the result, exactly antisymmetric."""
    dev = _dev()
    lower = (2 * np.arange(1 << 22) + 1) * 2.0 ** -24          # all 2^22 grid points below 1/2
    u = np.concatenate([lower, 1.0 - lower]).astype(np.float32)
    z = torch.empty(u.size, dtype=torch.float32, device=dev)
    M.approx_icdf(torch.from_numpy(u).to(dev), z, M.MLMC_ICDF_EXACT, M.MLMC_F32)
    torch.cuda.synchronize()
    zz = z.cpu().numpy()
    ref = O.ndtri(u.astype(np.float64))
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err_ulp = np.abs(zz.astype(np.float64) - ref) / ulp
    assert err_ulp.max() <= 3.0, err_ulp.max()
    assert err_ulp.mean() < 0.8
    assert np.all(zz[lower.size:] == -zz[:lower.size])


def test_exact_icdf_fp32_accuracy():
    dev = _dev()
    lower = (2 * np.arange(0, 1 << 22, 7) + 1) * 2.0 ** -24          # grid points below 1/2
    u = np.concatenate([lower, 1.0 - lower]).astype(np.float32)
    z = torch.empty(u.size, dtype=torch.float32, device=dev)
    M.approx_icdf(torch.from_numpy(u).to(dev), z, M.MLMC_ICDF_EXACT, M.MLMC_F32)
    torch.cuda.synchronize()
    zz = z.cpu().numpy()
    ref = O.ndtri(u.astype(np.float64))
    err = np.abs(zz - ref) / np.maximum(np.abs(ref), 1e-30)
    assert err.max() < 4 * 2.0 ** -23          # a few binary32 ulp
    assert np.all(zz[lower.size:] == -zz[:lower.size])


# ------------------------------------------------------------------ per-path parity


GBM_CALL = dict(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
GBM_X = dict(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_X, p0=0.05, p1=0.2)
OU_X = dict(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=2.0, p1=0.3, p2=0.5, x0=1.0)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_F32, M.MLMC_BF16])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("l", [0, 1, 2, 5, 9])
@pytest.mark.parametrize("sde", ["gbm_call", "ou_x"])
def test_twoway_table_paths_bitexact(prec, kahan, l, sde, pl_table):
    params = M.sde_params(**(GBM_CALL if sde == "gbm_call" else OU_X))
    N = 1537                                  # several blocks' worth of pairs and an odd tail
    got = gpu_paths(0, l, N, prec, kahan, M.MLMC_ICDF_TABLE, params, offset=77)
    ref = O.twoway_paths(l, np.arange(77, 77 + N), _bar_variant(prec, kahan), _orc_sde(params), SEED,
                         _kind_tag(0, M.MLMC_ICDF_TABLE, l), table=pl_table)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_F32, M.MLMC_BF16])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("l", [0, 1, 3, 8])
def test_fourway_table_paths(prec, kahan, l, pl_table):
    params = M.sde_params(**GBM_CALL)
    N = 1025
    got = gpu_paths(1, l, N, prec, kahan, M.MLMC_ICDF_TABLE, params)
    ref = O.fourway_paths(l, np.arange(N), O.variant(), _bar_variant(prec, kahan), _orc_sde(params), SEED,
                          _kind_tag(1, M.MLMC_ICDF_TABLE, l), table=pl_table)
    # bar pair: bit-exact against the emulation
    assert np.array_equal(got[:, 2:4], ref[:, 2:4])
    # hat pair: FP32 + Kahan with exact normals against FP64
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= TOL32 * scale[:, None])
    assert np.all(np.abs(got[:, 4] - ref[:, 4]) <= 2 * TOL32 * scale)


@pytest.mark.parametrize("icdf,rv", [(M.MLMC_ICDF_TABLE, O.RV_TABLE), (M.MLMC_ICDF_TABLE16, O.RV_TABLE16)])
@pytest.mark.parametrize("offset", [6, 2 ** 33 + 3])
def test_fourway_level0_shared_calls_at_unaligned_offsets(icdf, rv, offset, pl_table):
    """At level 0 four four-way paths share one Philox call; a launch whose
    path offset is not a multiple of 4 has slots that span two calls."""
    params = M.sde_params(**GBM_CALL)
    N = 37
    got = gpu_paths(1, 0, N, M.MLMC_F16, True, icdf, params, offset=offset)
    ref = O.fourway_paths(0, offset + np.arange(N), O.variant(), _bar_variant(M.MLMC_F16, True, rv), _orc_sde(params),
                          SEED, _kind_tag(1, icdf, 0), table=pl_table)
    assert np.array_equal(got[:, 2:4], ref[:, 2:4])
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= TOL32 * scale[:, None])


@pytest.mark.parametrize("l", [0, 1, 2, 4, 6])
@pytest.mark.parametrize("kahan", [False, True])
def test_twoway_exact_fp32_within_1e5(l, kahan):
    params = M.sde_params(**GBM_X)
    N = 2049
    got = gpu_paths(0, l, N, M.MLMC_F32, kahan, M.MLMC_ICDF_EXACT, params)
    ref = O.twoway_paths(l, np.arange(N), O.variant(), _orc_sde(params), SEED, _kind_tag(0, 0, l))
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got - ref) <= TOL32 * scale[:, None])


@pytest.mark.parametrize("l", [2, 6, 10, 12])
def test_fp16_kahan_against_fp64_within_2e3(l, pl_table):
    params = M.sde_params(**GBM_CALL)
    N = 1024 if l < 12 else 256
    got = gpu_paths(0, l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params)
    ref = O.twoway_paths(l, np.arange(N), O.variant(rv=O.RV_TABLE), _orc_sde(params), SEED,
                         _kind_tag(0, M.MLMC_ICDF_TABLE, l), table=pl_table)
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    err = np.abs(got - ref) / scale[:, None]
    assert err.max() <= TOL16K, err.max()


# ------------------------------------------------------------------ sums and statistics


@pytest.mark.parametrize("four", [0, 1])
def test_sums_equal_per_path_sums(four):
    params = M.sde_params(**GBM_CALL)
    N, l = 100001, 4
    paths = gpu_paths(four, l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params)
    fn = M.mlmc_nested_level if four else M.mlmc_level
    s = fn(l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, SEED)
    d = paths[:, -1]
    assert s.n == N
    assert abs(s.s1 - d.sum()) <= 1e-5 * np.abs(d).sum()
    assert abs(s.s2 - (d * d).sum()) <= 1e-5 * (d * d).sum()


def test_sums_independent_of_launch_shape(monkeypatch):
    """Each warp chunk of 32 pairs has its own partial sum, so the level sums
    are bit-identical whatever block size and grid the launch uses."""
    params = M.sde_params(**GBM_CALL)
    res = []
    for bt, k in [("256", "3"), ("160", "2"), ("128", "1")]:
        monkeypatch.setenv("MLMC_BLOCK", bt)
        monkeypatch.setenv("MLMC_BLOCKS_PER_SM", k)
        s = M.mlmc_nested_level(5, 700001, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, SEED)
        res.append((s.s1, s.s2))
    assert res[0] == res[1] == res[2]


def test_deterministic_repeat():
    params = M.sde_params(**GBM_CALL)
    a = M.mlmc_nested_level(6, 300000, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, SEED)
    b = M.mlmc_nested_level(6, 300000, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, SEED)
    assert (a.s1, a.s2) == (b.s1, b.s2)


@pytest.mark.parametrize("l", [0, 1, 3, 6])
def test_config1_level_means_closed_form(l):
    """Plain MLMC, GBM, P = X, FP32 exact normals, N = 1e5: level mean and
    variance within statistical error of the exact Euler moments."""
    from oracle import mlmc
    params = M.sde_params(**GBM_X)
    N = 100000
    s = M.mlmc_level(l, N, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, params, SEED)
    em, ev = mlmc.euler_twoway_moments(l)
    assert abs(s.mean - em) < 4 * math.sqrt(ev / N)
    assert abs(s.var / ev - 1) < 0.05


def test_level_sums_match_oracle_sums(pl_table):
    params = M.sde_params(**GBM_CALL)
    N, l = 20000, 5
    s = M.mlmc_level(l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, SEED)
    o1, o2 = O.level_sums(l, N, 0, _bar_variant(M.MLMC_F16, True), _orc_sde(params), SEED,
                          _kind_tag(0, 1, l), table=pl_table, nthreads=4)
    assert abs(s.s1 - o1) <= 1e-6 * (abs(o1) + math.sqrt(o2))
    assert abs(s.s2 - o2) <= 1e-6 * o2


# ------------------------------------------------------------------ full size, sampled


def test_full_size_level12_sampled_paths(pl_table):
    """N = 2^20 at l = 12 in the bench's launch configuration: per-path outputs
    of sampled samples against the oracle computing those samples alone."""
    params = M.sde_params(**GBM_CALL)
    N, l = 1 << 20, 12
    got = gpu_paths(1, l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params)
    idx = np.unique(np.concatenate([np.random.default_rng(3).integers(0, N, 48), [0, 1, N - 2, N - 1]]))
    ref = O.fourway_paths(l, idx, O.variant(), _bar_variant(M.MLMC_F16, True), _orc_sde(params), SEED,
                          _kind_tag(1, 1, l), table=pl_table)
    assert np.array_equal(got[idx, 2:4], ref[:, 2:4])
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[idx, 0:2] - ref[:, 0:2]) <= TOL32 * scale[:, None])
    # every sample's D is the FP32 combination of its four payoffs
    f = got.astype(np.float32)
    d = (f[:, 0] - f[:, 1]) - (f[:, 2] - f[:, 3])
    assert np.array_equal(d, f[:, 4])
    # fine payoffs: Black-Scholes within statistical error plus the Euler weak
    # bias at l = 12 (hat) and the binary16 rounding bias (bar)
    from oracle import mlmc
    bs = mlmc.bs_call()
    for col, extra in ((0, 2e-4), (2, 2e-3)):
        p = got[:, col]
        assert abs(p.mean() - bs) < 5 * p.std() / math.sqrt(N) + extra


def test_edge_cases(pl_table):
    params = M.sde_params(**GBM_CALL)
    # N = 1 (a single sample, half of a pair) and the deepest level with few samples
    got = gpu_paths(0, 3, 1, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, offset=5)
    ref = O.twoway_paths(3, [5], _bar_variant(M.MLMC_F16, True), _orc_sde(params), SEED, _kind_tag(0, 1, 3),
                         table=pl_table)
    assert np.array_equal(got, ref)
    got = gpu_paths(0, 18, 3, M.MLMC_F32, True, M.MLMC_ICDF_TABLE, params, offset=2 ** 33 + 1)
    ref = O.twoway_paths(18, 2 ** 33 + 1 + np.arange(3), _bar_variant(M.MLMC_F32, True), _orc_sde(params), SEED,
                         _kind_tag(0, 1, 18), table=pl_table)
    assert np.array_equal(got, ref)
    s = M.mlmc_level(0, 1, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, params, SEED)
    assert s.n == 1 and s.var == 0.0
    got = gpu_paths(0, 18, 3, M.MLMC_BF16, True, M.MLMC_ICDF_TABLE, params, offset=2 ** 40 + 3)
    ref = O.twoway_paths(18, 2 ** 40 + 3 + np.arange(3), _bar_variant(M.MLMC_BF16, True), _orc_sde(params), SEED,
                         _kind_tag(0, 1, 18), table=pl_table)
    assert np.array_equal(got, ref)


def test_invalid_arguments_raise():
    _dev()
    params = M.sde_params(**GBM_CALL)
    with pytest.raises(M.MlmcError) as e:
        M.mlmc_level(19, 10, M.MLMC_F32, False, 0, params, SEED)
    assert e.value.status == M.MLMC_EINVAL
    with pytest.raises(M.MlmcError):
        M.mlmc_nested_level(3, 10, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, params, SEED)


# ------------------------------------------------------------------ 16-bit uniforms (TABLE16)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_F32, M.MLMC_BF16])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("l", [0, 1, 2, 3, 4, 7, 10])
def test_twoway_table16_paths_bitexact(prec, kahan, l, pl_table):
    """Two 16-bit uniforms per Philox word; levels 0-2 use part of one call."""
    params = M.sde_params(**GBM_CALL)
    N = 1537
    got = gpu_paths(0, l, N, prec, kahan, M.MLMC_ICDF_TABLE16, params, offset=123)
    ref = O.twoway_paths(l, np.arange(123, 123 + N), _bar_variant(prec, kahan, O.RV_TABLE16), _orc_sde(params),
                         SEED, _kind_tag(0, M.MLMC_ICDF_TABLE16, l), table=pl_table)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("sde", ["gbm_x", "ou_x"])
def test_twoway_table16_ou_and_x(sde, pl_table):
    params = M.sde_params(**(GBM_X if sde == "gbm_x" else OU_X))
    got = gpu_paths(0, 6, 999, M.MLMC_F16, True, M.MLMC_ICDF_TABLE16, params)
    ref = O.twoway_paths(6, np.arange(999), _bar_variant(M.MLMC_F16, True, O.RV_TABLE16), _orc_sde(params), SEED,
                         _kind_tag(0, M.MLMC_ICDF_TABLE16, 6), table=pl_table)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_BF16, M.MLMC_F32])
@pytest.mark.parametrize("l", [0, 1, 4, 9])
def test_fourway_table16_paths(prec, l, pl_table):
    params = M.sde_params(**GBM_CALL)
    N = 1025
    got = gpu_paths(1, l, N, prec, True, M.MLMC_ICDF_TABLE16, params)
    ref = O.fourway_paths(l, np.arange(N), O.variant(), _bar_variant(prec, True, O.RV_TABLE16), _orc_sde(params),
                          SEED, _kind_tag(1, M.MLMC_ICDF_TABLE16, l), table=pl_table)
    assert np.array_equal(got[:, 2:4], ref[:, 2:4])
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= TOL32 * scale[:, None])
    # the hat pair is the same as with 24-bit table normals on the bar pair
    hat = gpu_paths(1, l, N, prec, True, M.MLMC_ICDF_TABLE, params)
    assert np.array_equal(got[:, 0:2], hat[:, 0:2])


@pytest.mark.parametrize("prec", [M.MLMC_F32, M.MLMC_F16, M.MLMC_BF16])
def test_approx_icdf_table16_bitexact(prec, pl_table):
    dev = _dev()
    rng = np.random.default_rng(4)
    u = np.concatenate([rng.random(100000), (2 * rng.integers(0, 1 << 23, 100000) + 1) * 2.0 ** -24,
                        [2.0 ** -24, 2.0 ** -16, 2.0 ** -16 - 2.0 ** -24, 0.5, 0.5 - 2.0 ** -24,
                         1 - 2.0 ** -24]]).astype(np.float32)
    u = u[(u > 0) & (u < 1)]
    z = torch.empty(u.size, dtype=torch.float32 if prec == M.MLMC_F32 else torch.int16, device=dev)
    M.approx_icdf(torch.from_numpy(u).to(dev), z, M.MLMC_ICDF_TABLE16, prec)
    torch.cuda.synchronize()
    ref = O.approx_icdf(u.astype(np.float64), O.RV_TABLE16, prec=_OPREC[prec], table=pl_table)
    got = z.cpu().numpy().view(np.float16).astype(np.float64) if prec == M.MLMC_F16 else _z_host(z, prec)
    assert np.array_equal(got, ref)


def test_table16_level_sums_match_oracle(pl_table):
    params = M.sde_params(**GBM_CALL)
    for four, l, N in ((0, 5, 30001), (1, 4, 20001)):
        fn = M.mlmc_nested_level if four else M.mlmc_level
        s = fn(l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE16, params, SEED)
        bar = _bar_variant(M.MLMC_F16, True, O.RV_TABLE16)
        o1, o2 = O.level_sums(l, N, 0, O.variant() if four else bar, _orc_sde(params), SEED,
                              _kind_tag(four, M.MLMC_ICDF_TABLE16, l), table=pl_table, four=bool(four),
                              var2=bar, nthreads=4)
        assert abs(s.s1 - o1) <= 2e-5 * (abs(o1) + math.sqrt(o2 * N)), (four, s.s1, o1)
        assert abs(s.s2 - o2) <= 1e-5 * o2


def test_full_size_level12_table16_sampled(pl_table):
    """N = 2^20 at l = 12, two-way TABLE16 (the bench's launch shape):
    sampled per-path outputs against the oracle."""
    params = M.sde_params(**GBM_CALL)
    N, l = 1 << 20, 12
    got = gpu_paths(0, l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE16, params)
    idx = np.unique(np.concatenate([np.random.default_rng(5).integers(0, N, 40), [0, 1, N - 2, N - 1]]))
    ref = O.twoway_paths(l, idx, _bar_variant(M.MLMC_F16, True, O.RV_TABLE16), _orc_sde(params), SEED,
                         _kind_tag(0, 1, l), table=pl_table)
    assert np.array_equal(got[idx], ref)


# ------------------------------------------------------------------ piecewise cubic (CUBIC)


@pytest.fixture(scope="module")
def cubic_table():
    from oracle import table
    return table.build_cubic_table()


def test_cubic_table_matches_oracle(cubic_table):
    _dev()
    d64, d32, d16, dbf = M.mlmc_icdf_cubic()
    assert np.allclose(d64, cubic_table, rtol=1e-11, atol=1e-13)
    assert np.array_equal(d32.astype(np.float64), O.round_bits(cubic_table, O.F32).reshape(16, 4))
    assert np.array_equal(d16.view(np.float16).astype(np.float64), O.round_bits(cubic_table, O.F16).reshape(16, 4))
    bf = (dbf.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    assert np.array_equal(bf, O.round_bits(cubic_table, O.BF16).reshape(16, 4))


@pytest.mark.parametrize("prec", [M.MLMC_F32, M.MLMC_F16, M.MLMC_BF16])
def test_approx_icdf_cubic_bitexact(prec, pl_table, cubic_table):
    dev = _dev()
    rng = np.random.default_rng(6)
    u = np.concatenate([(2 * rng.integers(0, 1 << 23, 200000) + 1) * 2.0 ** -24,
                        [2.0 ** -24, 1 - 2.0 ** -24, 0.5 - 2.0 ** -24, 0.5 + 2.0 ** -24, 0.25 + 2.0 ** -24,
                         0.25 - 2.0 ** -24, 2.0 ** -16 + 2.0 ** -24, 2.0 ** -16 - 2.0 ** -24]]).astype(np.float32)
    z = torch.empty(u.size, dtype=torch.float32 if prec == M.MLMC_F32 else torch.int16, device=dev)
    M.approx_icdf(torch.from_numpy(u).to(dev), z, M.MLMC_ICDF_CUBIC, prec)
    torch.cuda.synchronize()
    ref = O.approx_icdf(u.astype(np.float64), O.RV_CUBIC, prec=_OPREC[prec], table=pl_table, cubic=cubic_table)
    got = z.cpu().numpy().view(np.float16).astype(np.float64) if prec == M.MLMC_F16 else _z_host(z, prec)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_F32, M.MLMC_BF16])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("l", [0, 1, 2, 5, 9])
@pytest.mark.parametrize("sde", ["gbm_call", "ou_x"])
def test_twoway_cubic_paths_bitexact(prec, kahan, l, sde, pl_table, cubic_table):
    params = M.sde_params(**(GBM_CALL if sde == "gbm_call" else OU_X))
    N = 1537
    got = gpu_paths(0, l, N, prec, kahan, M.MLMC_ICDF_CUBIC, params, offset=31)
    ref = O.twoway_paths(l, np.arange(31, 31 + N), _bar_variant(prec, kahan, O.RV_CUBIC), _orc_sde(params), SEED,
                         _kind_tag(0, M.MLMC_ICDF_CUBIC, l), table=pl_table, cubic=cubic_table)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_BF16, M.MLMC_F32])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("l", [0, 3, 8])
def test_fourway_cubic_paths(prec, kahan, l, pl_table, cubic_table):
    params = M.sde_params(**GBM_CALL)
    N = 1025
    got = gpu_paths(1, l, N, prec, kahan, M.MLMC_ICDF_CUBIC, params)
    ref = O.fourway_paths(l, np.arange(N), O.variant(), _bar_variant(prec, kahan, O.RV_CUBIC), _orc_sde(params),
                          SEED, _kind_tag(1, M.MLMC_ICDF_CUBIC, l), table=pl_table, cubic=cubic_table)
    assert np.array_equal(got[:, 2:4], ref[:, 2:4])
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= TOL32 * scale[:, None])


def test_cubic_level_sums_match_oracle(pl_table, cubic_table):
    params = M.sde_params(**GBM_CALL)
    for four, l, N in ((0, 6, 30001), (1, 5, 20001)):
        fn = M.mlmc_nested_level if four else M.mlmc_level
        s = fn(l, N, M.MLMC_F16, True, M.MLMC_ICDF_CUBIC, params, SEED)
        bar = _bar_variant(M.MLMC_F16, True, O.RV_CUBIC)
        o1, o2 = O.level_sums(l, N, 0, O.variant() if four else bar, _orc_sde(params), SEED,
                              _kind_tag(four, M.MLMC_ICDF_CUBIC, l), table=pl_table, cubic=cubic_table,
                              four=bool(four), var2=bar, nthreads=4)
        assert abs(s.s1 - o1) <= 2e-5 * (abs(o1) + math.sqrt(o2 * N)), (four, s.s1, o1)
        assert abs(s.s2 - o2) <= 1e-5 * o2
