"""Randomised parity: seeded draws of the whole variant space — SDE and its
parameters, payoff, scheme, level, N, path offset (including 64-bit
offsets), working precision, Kahan, approximate inverse CDF, estimator —
each checked per path against the oracle: the low-precision ("bar") paths
bit for bit, the exact-normal FP32 paths within 1e-5 relative."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
import paper_2012_09739_gb300 as M  # noqa: E402

_OPREC = {M.MLMC_F32: O.F32, M.MLMC_F16: O.F16, M.MLMC_BF16: O.BF16}
_ORV = {M.MLMC_ICDF_TABLE: O.RV_TABLE, M.MLMC_ICDF_TABLE16: O.RV_TABLE16, M.MLMC_ICDF_CUBIC: O.RV_CUBIC}


@pytest.fixture(scope="module")
def tables():
    from oracle import table
    return table.build_table(), table.build_cubic_table()


def _draw(rng):
    sde = int(rng.integers(0, 2))
    if sde == M.MLMC_GBM:
        p = M.sde_params(sde=sde, payoff=int(rng.integers(0, 2)), p0=float(rng.uniform(-0.1, 0.15)),
                         p1=float(rng.uniform(0.05, 0.6)), x0=float(rng.uniform(0.5, 2.0)),
                         T=float(rng.choice([0.25, 1.0, 2.0])), K=float(rng.uniform(0.7, 1.3)),
                         scheme=int(rng.integers(0, 2)))
    else:
        p = M.sde_params(sde=sde, payoff=int(rng.integers(0, 2)), p0=float(rng.uniform(0.2, 4.0)),
                         p1=float(rng.normal()), p2=float(rng.uniform(0.05, 1.0)), x0=float(rng.uniform(-1, 2)),
                         T=1.0, K=0.0, disc=1.0, scheme=int(rng.integers(0, 2)))
    four = int(rng.integers(0, 2))
    l = int(rng.integers(0, 11))
    n = int(rng.integers(1, 700))
    off = int(rng.choice([0, 1, int(rng.integers(0, 1 << 40))]))
    prec = int(rng.choice([M.MLMC_F32, M.MLMC_F16, M.MLMC_BF16]))
    kahan = bool(rng.integers(0, 2))
    icdf = int(rng.choice([M.MLMC_ICDF_TABLE, M.MLMC_ICDF_TABLE16, M.MLMC_ICDF_CUBIC]))
    seed = int(rng.integers(0, 1 << 63))
    return p, four, l, n, off, prec, kahan, icdf, seed


@pytest.mark.parametrize("case", range(40))
def test_random_variant_per_path(case, tables):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(9000 + case)
    p, four, l, n, off, prec, kahan, icdf, seed = _draw(rng)
    w = 5 if four else 3
    out = torch.empty(n * w, dtype=torch.float32, device="cuda:0")
    M.mlmc_level_paths(four, l, n, prec, kahan, icdf, p, seed, off, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64).reshape(n, w)
    osde = O.SDE(p.sde, p.payoff, p.p0, p.p1, p.p2, p.x0, p.T, p.K, p.disc, p.scheme)
    bar = O.variant(prec=_OPREC[prec], kahan=kahan, rv=_ORV[icdf])
    idx = off + np.arange(n, dtype=np.uint64)
    kind = O.KIND_FOUR if four else O.KIND_APPROX
    tag = O.make_tag(kind, l)
    if four:
        ref = O.fourway_paths(l, idx, O.variant(), bar, osde, seed, tag, table=tables[0], cubic=tables[1])
        assert np.array_equal(got[:, 2:4], ref[:, 2:4]), (case, l, n, off, prec, kahan, icdf)
        scale = np.maximum(1.0, np.abs(ref[:, 0]))
        assert np.all(np.abs(got[:, 0:2] - ref[:, 0:2]) <= 1e-5 * scale[:, None]), case
    else:
        ref = O.twoway_paths(l, idx, bar, osde, seed, tag, table=tables[0], cubic=tables[1])
        assert np.array_equal(got, ref), (case, l, n, off, prec, kahan, icdf)
