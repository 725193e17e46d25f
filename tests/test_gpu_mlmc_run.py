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


def _opts(estimator, prec=M.MLMC_F16, kahan=1, icdf=M.MLMC_ICDF_TABLE, seed=1234, trial_all=0, n0=10000):
    return M.mlmc_run_opts(estimator=estimator, prec=prec, kahan=kahan, icdf=icdf, max_level=18, min_levels=3,
                           n0=n0, seed=seed, alpha=1.0, timeout_s=300.0, trial_all=trial_all)


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
    # 3 combined standard errors plus the weak-bias allowance the bias test grants
    assert abs(r.estimate - bs) < 3 * math.sqrt(r.variance) + eps / math.sqrt(2)
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
    r = M.mlmc_run(eps, params, _opts(1, prec=-1, trial_all=1))
    assert abs(r.estimate - mlmc.bs_call()) < 3 * math.sqrt(r.variance) + eps / math.sqrt(2)
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
    assert abs(r.estimate - mlmc.bs_call()) < 3 * math.sqrt(r.variance) + eps / math.sqrt(2)
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


REPLAY_CASES = [  # (eps, estimator, prec, kahan, icdf, scheme, trial_all)
    (1e-3, 0, M.MLMC_F32, 0, M.MLMC_ICDF_EXACT, M.MLMC_EULER, 0),
    (1e-4, 0, M.MLMC_F32, 0, M.MLMC_ICDF_EXACT, M.MLMC_EULER, 0),
    (1e-4, 1, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, M.MLMC_EULER, 0),
    (1e-4, 1, M.MLMC_F32, 0, M.MLMC_ICDF_TABLE16, M.MLMC_EULER, 0),
    (5e-5, 1, -1, 0, M.MLMC_ICDF_TABLE, M.MLMC_EULER, 0),
    (5e-5, 1, -1, 0, M.MLMC_ICDF_TABLE16, M.MLMC_EULER, 1),
    (5e-5, 1, -1, 0, M.MLMC_ICDF_TABLE16, M.MLMC_MILSTEIN, 0),
]


@pytest.mark.parametrize("eps,est,prec,kahan,icdf,scheme,trial_all", REPLAY_CASES)
def test_mlmc_run_decisions_replayed_by_the_oracle_driver(eps, est, prec, kahan, icdf, scheme, trial_all):
    """Every draw of mlmc_run (term, samples, path offset, sums, cost model)
    is fed back through the oracle's adaptive driver, which must ask for
    exactly the same draws round by round -- the same levels, sample counts
    N_t per round and per-level variants -- and so reach the same estimate
    (the same FP64 sums added in the same order)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0, scheme=scheme)
    opts = _opts(est, prec=prec, kahan=kahan, icdf=icdf, trial_all=trial_all, seed=77)
    r, trace = M.mlmc_run(eps, params, opts, trace_cap=8192)
    assert 0 < r.trace_len <= 8192
    rounds = {}
    for rec in trace:
        rounds.setdefault(rec.round, []).append(rec)
    assert sorted(rounds) == list(range(r.rounds))
    costs = {}
    for rec in trace:
        key = (rec.l, rec.kind, rec.prec, rec.kahan, rec.icdf)
        assert costs.setdefault(key, rec.cost_ns) == rec.cost_ns
    seq = iter(range(r.rounds))

    def draw(requests):
        recs = rounds[next(seq)]
        got = [((x.l, x.kind, x.prec, x.kahan, x.icdf), int(x.dn), int(x.path_offset)) for x in recs]
        assert requests == got
        return [(x.s1, x.s2) for x in recs]
    o = mlmc.adaptive_mlmc(eps, draw, lambda k: costs[k], nested=est == 1, prec=prec, kahan=kahan, icdf=icdf,
                           n0=10000, min_levels=3, max_level=18, alpha=1.0, trial_all=bool(trial_all))
    assert o["converged"] and o["rounds"] == r.rounds and o["levels"] == r.levels
    assert o["estimate"] == r.estimate and abs(o["variance"] - r.variance) <= 1e-14 * r.variance
    # per-level variant and the kept / discarded draws
    kinds = [0, 1] if est == 1 else [0]
    final = {key: n for key, n, _, _ in o["terms"]}
    for l in range(r.levels):
        for k in kinds:
            got = [n for key, n in final.items() if key[0] == l and key[1] == k]
            assert r.n[k][l] == (got[0] if got else 0), (l, k)
        if est == 1 and prec == -1:
            c = o["choice"][l]
            assert r.nested[l] == (0 if c == mlmc.CH_STANDARD else 1)
            if c != mlmc.CH_STANDARD:
                assert r.prec[l] == (M.MLMC_F32 if c == mlmc.CH_F32 else M.MLMC_F16)
                assert r.kahan[l] == (1 if c == mlmc.CH_F16K else 0)
    kept = sum(rec.dn * 2.0 ** rec.l for rec in trace if rec.kept)
    assert abs(kept + r.discarded_path_steps - r.path_steps) <= 1e-9 * r.path_steps
    # the accounting: the cost model's time of the samples drawn, and the measured device time
    assert r.model_s > 0 and r.device_s > 0 and r.wall_s >= r.device_s


@pytest.mark.parametrize("est,prec,kahan,icdf,scheme", [
    (0, M.MLMC_F32, 0, M.MLMC_ICDF_EXACT, M.MLMC_EULER),
    (0, M.MLMC_F32, 1, M.MLMC_ICDF_EXACT, M.MLMC_MILSTEIN),
    (1, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE16, M.MLMC_EULER),
    (1, M.MLMC_F32, 0, M.MLMC_ICDF_TABLE, M.MLMC_EULER),
    (1, -1, 0, M.MLMC_ICDF_TABLE16, M.MLMC_EULER),
    (1, -1, 0, M.MLMC_ICDF_TABLE, M.MLMC_EULER),
    (1, -1, 0, M.MLMC_ICDF_TABLE16, M.MLMC_MILSTEIN),
    (1, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE16, M.MLMC_MILSTEIN),
    (1, M.MLMC_F16, 1, M.MLMC_ICDF_MLP, M.MLMC_EULER),
])
def test_fused_small_rounds_give_the_same_runs(monkeypatch, est, prec, kahan, icdf, scheme):
    """Latency-sized rounds of one kernel group run as one fused launch
    (descriptors as kernel parameters, each item's sum by the warp that
    finishes its last tile, larger items' by the last block), and so do the
    per-level choice's rounds of several variants (prec -1: the choice
    kernel, each tile dispatched on its item's variant) and the rounds of
    one variant without a mixed kernel (Milstein, the network); the same
    runs with the two-kernel path (MLMC_ROUND_FUSED=0) must take the same
    draws and get the same sums, bit for bit, at an RMSE where every round
    is small (1e-3) and where the later ones are not (1e-4)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if icdf == M.MLMC_ICDF_MLP:
        from workloads import mlp_initial_weights
        M.mlmc_mlp_set_weights(mlp_initial_weights(5))
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0, scheme=scheme)
    for eps in (1e-3, 1e-4):
        runs = []
        for fused in ("1", "0"):
            monkeypatch.setenv("MLMC_ROUND_FUSED", fused)
            runs.append(M.mlmc_run(eps, params, _opts(est, prec=prec, kahan=kahan, icdf=icdf, seed=91),
                                   trace_cap=4096))
        (a, ta), (b, tb) = runs
        assert a.estimate == b.estimate and a.variance == b.variance and a.rounds == b.rounds, eps
        assert len(ta) == len(tb)
        for x, y in zip(ta, tb):
            assert (x.round, x.l, x.kind, x.dn, x.path_offset, x.s1, x.s2) == \
                (y.round, y.l, y.kind, y.dn, y.path_offset, y.s1, y.s2), eps
