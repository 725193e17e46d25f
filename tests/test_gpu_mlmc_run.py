"""Adaptive MLMC (mlmc_run) on the GPU: the standard FP32 exact-normal
estimator and the nested FP16 + Kahan estimator reach the target RMSE around
the Black-Scholes price, with sample counts that satisfy the Sec. 3
allocation and a last level that passes the weak-error rule (checked with
the oracle's own implementations of both)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2012_09739_gb300 as M  # noqa: E402
from oracle import mlmc  # noqa: E402


def _opts(estimator, prec=M.MLMC_F16, kahan=1, icdf=M.MLMC_ICDF_TABLE, seed=1234):
    return M.mlmc_run_opts(estimator=estimator, prec=prec, kahan=kahan, icdf=icdf, max_level=18, min_levels=3,
                           n0=10000, seed=seed, alpha=1.0, timeout_s=300.0)


@pytest.mark.parametrize("estimator,icdf,prec", [(0, M.MLMC_ICDF_TABLE, M.MLMC_F16),
                                                 (1, M.MLMC_ICDF_TABLE, M.MLMC_F16),
                                                 (1, M.MLMC_ICDF_TABLE16, M.MLMC_F16),
                                                 (1, M.MLMC_ICDF_TABLE, M.MLMC_BF16)])
def test_mlmc_run_reaches_eps(estimator, icdf, prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps = 1e-3
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    r = M.mlmc_run(eps, params, _opts(estimator, prec=prec, icdf=icdf))
    bs = mlmc.bs_call()
    assert r.levels >= 3 and r.rounds >= 1
    assert r.variance <= eps * eps / 2 * 1.05
    assert abs(r.estimate - bs) < 4 * eps
    kinds = [0, 1] if estimator == 1 else [0]
    V = [r.var[k][l] for l in range(r.levels) for k in kinds]
    C = [r.cost[k][l] for l in range(r.levels) for k in kinds]
    N = np.array([r.n[k][l] for l in range(r.levels) for k in kinds], dtype=np.float64)
    # the final split satisfies the variance target with the returned V
    assert np.sum(np.array(V) / N) <= eps * eps / 2 * 1.05
    Y = [sum(r.mean[k][l] for k in kinds) for l in range(r.levels)]
    assert mlmc.weak_converged(Y, eps)


def test_mlmc_run_invalid():
    params = M.sde_params()
    with pytest.raises(M.MlmcError):
        M.mlmc_run(-1.0, params, _opts(0))
    with pytest.raises(M.MlmcError):
        M.mlmc_run(1e-3, params, _opts(1, icdf=M.MLMC_ICDF_EXACT))


def test_mlmc_run_auto_precision_per_level():
    """prec = -1: each level keeps the variant with the smallest
    sqrt(v c) + sqrt(V C) (Sec. 3) and reports the per-level efficiency
    factor against the standard estimator."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps = 2e-4
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    r = M.mlmc_run(eps, params, _opts(1, prec=-1))
    assert abs(r.estimate - mlmc.bs_call()) < 4 * eps
    assert r.variance <= eps * eps / 2 * 1.05
    for l in range(r.levels):
        assert r.prec[l] in (M.MLMC_F16, M.MLMC_F32)
        assert r.efficiency[l] > 0.0
        assert r.n[0][l] >= 10000
        # a level either runs the nested pair or the standard estimator alone
        assert (r.n[1][l] >= 10000) if r.nested[l] else (r.n[1][l] == 0)


def test_mlmc_run_auto_with_milstein():
    """Milstein with the per-level choice: each level runs either the nested
    pair or the standard estimator alone (whichever the measured variances
    and the cost model favour); the mixed telescoping sum reaches eps around
    the Black-Scholes price."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    eps = 2e-5
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0,
                          scheme=M.MLMC_MILSTEIN)
    r = M.mlmc_run(eps, params, _opts(1, prec=-1, icdf=M.MLMC_ICDF_TABLE16))
    assert abs(r.estimate - mlmc.bs_call()) < 4 * eps + 2e-5      # plus the l <= L weak bias allowance
    assert r.variance <= eps * eps / 2 * 1.05
    for l in range(r.levels):
        assert r.nested[l] in (0, 1) and r.n[0][l] >= 10000
        assert (r.n[1][l] >= 10000) if r.nested[l] else (r.n[1][l] == 0)


def test_mlmc_run_timeout_is_reported_and_recoverable():
    """A wall-clock limit that cannot be met ends the host wait with
    MLMC_ETIMEOUT (the GPU work itself completes; nothing hangs); the next run
    on the same device succeeds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    o = _opts(0)
    o.timeout_s = 1e-4
    with pytest.raises(M.MlmcError) as e:
        M.mlmc_run(1e-5, params, o)
    assert e.value.status == M.MLMC_ETIMEOUT
    torch.cuda.synchronize()
    r = M.mlmc_run(1e-3, params, _opts(0))
    assert abs(r.estimate - mlmc.bs_call()) < 4e-3
