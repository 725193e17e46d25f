"""The Milstein scheme on the GPU (GBM; named in the paper's conclusions):
bit-exact per-path parity of the low-precision paths with the oracle's
emulation, FP32 exact-normal paths against FP64, the O(delta^2) level
variance against the exact step-polynomial moments, batch and adaptive
driver with Milstein."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2012_09739_gb300 as M  # noqa: E402
from oracle import mlmc  # noqa: E402

SEED = 1234
_OPREC = {M.MLMC_F32: O.F32, M.MLMC_F16: O.F16, M.MLMC_BF16: O.BF16}
_ORV = {M.MLMC_ICDF_TABLE: O.RV_TABLE, M.MLMC_ICDF_CUBIC: O.RV_CUBIC, M.MLMC_ICDF_TABLE16: O.RV_TABLE16}


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _osde(p):
    return O.SDE(p.sde, p.payoff, p.p0, p.p1, p.p2, p.x0, p.T, p.K, p.disc, p.scheme)


def _paths(four, l, N, prec, kahan, icdf, params, offset=0):
    w = 5 if four else 3
    out = torch.empty(N * w, dtype=torch.float32, device=_dev())
    M.mlmc_level_paths(four, l, N, prec, kahan, icdf, params, SEED, offset, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64).reshape(N, w)


def _tag(four, icdf, l):
    kind = O.KIND_FOUR if four else (O.KIND_STD if icdf == M.MLMC_ICDF_EXACT else O.KIND_APPROX)
    return O.make_tag(kind, l)


@pytest.fixture(scope="module")
def tables():
    from oracle import table
    return table.build_table(), table.build_cubic_table()


MIL_CALL = dict(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0, scheme=M.MLMC_MILSTEIN)
MIL_X = dict(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_X, p0=0.05, p1=0.2, scheme=M.MLMC_MILSTEIN)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_F32, M.MLMC_BF16])
@pytest.mark.parametrize("kahan", [True, False])
@pytest.mark.parametrize("icdf", [M.MLMC_ICDF_TABLE, M.MLMC_ICDF_CUBIC, M.MLMC_ICDF_TABLE16])
@pytest.mark.parametrize("l", [0, 1, 3, 8])
def test_milstein_twoway_paths_bitexact(prec, kahan, icdf, l, tables):
    params = M.sde_params(**MIL_CALL)
    N = 1029
    got = _paths(0, l, N, prec, kahan, icdf, params, offset=9)
    ref = O.twoway_paths(l, np.arange(9, 9 + N), O.variant(prec=_OPREC[prec], kahan=kahan, rv=_ORV[icdf]),
                         _osde(params), SEED, _tag(0, icdf, l), table=tables[0], cubic=tables[1])
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", [M.MLMC_F16, M.MLMC_BF16, M.MLMC_F32])
@pytest.mark.parametrize("l", [0, 2, 7])
def test_milstein_fourway_paths(prec, l, tables):
    params = M.sde_params(**MIL_CALL)
    N = 1025
    got = _paths(1, l, N, prec, True, M.MLMC_ICDF_TABLE, params)
    ref = O.fourway_paths(l, np.arange(N), O.variant(), O.variant(prec=_OPREC[prec], kahan=True, rv=O.RV_TABLE),
                          _osde(params), SEED, _tag(1, M.MLMC_ICDF_TABLE, l), table=tables[0], cubic=tables[1])
    assert np.array_equal(got[:, 2:4], ref[:, 2:4])
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= 1e-5 * scale[:, None])


@pytest.mark.parametrize("l", [0, 2, 5])
def test_milstein_exact_fp32_within_1e5(l):
    params = M.sde_params(**MIL_X)
    N = 2049
    got = _paths(0, l, N, M.MLMC_F32, True, M.MLMC_ICDF_EXACT, params)
    ref = O.twoway_paths(l, np.arange(N), O.variant(), _osde(params), SEED, _tag(0, M.MLMC_ICDF_EXACT, l))
    scale = np.maximum(1.0, np.abs(ref[:, 0]))
    assert np.all(np.abs(got - ref) <= 1e-5 * scale[:, None])


def test_milstein_level_variance_order_delta_squared():
    """FP32 exact normals, P = X: level means and variances against the exact
    step-polynomial moments; V_l decays like delta^2 (strong order 1)."""
    params = M.sde_params(**MIL_X)
    logv = []
    for l in range(0, 9):
        N = 1 << 20
        s = M.mlmc_level(l, N, M.MLMC_F32, True, M.MLMC_ICDF_EXACT, params, SEED)
        em, ev = mlmc.gbm_level_moments(l, milstein=True)
        assert abs(s.mean - em) < 4 * math.sqrt(ev / N), l
        assert abs(s.var / ev - 1) < 0.05, l
        logv.append(math.log2(s.var))
    assert abs(np.polyfit(np.arange(2, 9), logv[2:], 1)[0] + 2.0) < 0.1


def test_milstein_ou_is_euler():
    _dev()
    e = M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=2.0, p1=0.3, p2=0.5)
    m = M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=2.0, p1=0.3, p2=0.5, scheme=M.MLMC_MILSTEIN)
    a = _paths(0, 6, 777, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, e)
    b = _paths(0, 6, 777, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, m)
    assert np.array_equal(a, b)


def test_milstein_batch_equals_level_kernels():
    _dev()
    p = M.sde_params(**MIL_CALL)
    items = [M.mlmc_work(p, l, kind, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 20001, 0) for l in (0, 3, 7)
             for kind in (0, 1)]
    got = M.mlmc_batch(items, SEED)
    for it, g in zip(items, got):
        fn = M.mlmc_nested_level if it.kind else M.mlmc_level
        ref = fn(it.l, it.N, it.prec, it.kahan, it.icdf, p, SEED)
        assert g.n == ref.n
        assert abs(g.s1 - ref.s1) <= 2e-6 * (abs(ref.s1) + math.sqrt(ref.s2 * ref.n)) + 1e-30
        assert abs(g.s2 - ref.s2) <= 2e-6 * ref.s2 + 1e-30


@pytest.mark.parametrize("estimator", [0, 1])
def test_milstein_mlmc_run_reaches_eps(estimator):
    _dev()
    eps = 5e-4
    p = M.sde_params(**MIL_CALL)
    o = M.mlmc_run_opts(estimator=estimator, prec=M.MLMC_F16, kahan=1, icdf=M.MLMC_ICDF_TABLE, max_level=18,
                        min_levels=3, n0=10000, seed=77, alpha=1.0, timeout_s=300.0)
    r = M.mlmc_run(eps, p, o)
    assert abs(r.estimate - mlmc.bs_call()) < 4 * eps
    assert r.variance <= eps * eps / 2 * 1.05
