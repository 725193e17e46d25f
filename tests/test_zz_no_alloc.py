"""The allocation-free entry point mlmc_level_noalloc, for callers that cannot
allocate device memory when they request an estimate.  It must agree with the
ordinary entry point (mlmc_level_async, which takes its scratch from the
stream-ordered allocator) on two calls in a row through the same fixed
scratch array, and refuse sizes its scratch cannot hold.

Collected last on purpose (file name), so that a failure here does not hide
the other tests of a run that stops at the first failure."""
import ctypes
import math

import pytest

torch = pytest.importorskip("torch")

import paper_2012_09739_gb300 as M  # noqa: E402

pytestmark = pytest.mark.gpu


def _close(a, b, n):
    # same samples, different block grouping of the FP32 warp sums
    s1a, s2a = a
    s1b, s2b = b
    assert abs(s1a - s1b) <= 1e-6 * (abs(s1b) + math.sqrt(n * s2b)), (a, b)
    assert abs(s2a - s2b) <= 1e-6 * s2b, (a, b)


def test_noalloc_matches_allocating_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    gbm = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    mil = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0, scheme=M.MLMC_MILSTEIN)
    ou = M.sde_params(sde=M.MLMC_OU, payoff=M.MLMC_PAYOFF_X, p0=2.0, p1=0.3, p2=0.5)
    cases = [  # (four, l, N, prec, kahan, icdf, offset, params)
        (1, 8, 1 << 20, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, 0, gbm),
        (0, 5, 300001, M.MLMC_F32, False, M.MLMC_ICDF_EXACT, 12345, gbm),
        (0, 6, 200001, M.MLMC_BF16, True, M.MLMC_ICDF_CUBIC, 3, gbm),
        (1, 7, 100000, M.MLMC_F16, True, M.MLMC_ICDF_TABLE16, 0, mil),
        (0, 9, 65536, M.MLMC_F32, True, M.MLMC_ICDF_TABLE, 1, ou),
    ]
    for four, l, N, prec, kahan, icdf, off, params in cases:
        got = torch.zeros(2, dtype=torch.float64, device=dev)
        ref = torch.zeros(2, dtype=torch.float64, device=dev)
        M.mlmc_level_noalloc(four, l, N, prec, kahan, icdf, params, 1234, off, got)
        M.mlmc_level_async(four, l, N, prec, kahan, icdf, params, 1234, off, ref)
        torch.cuda.synchronize()
        first = got.cpu().tolist()
        _close(first, ref.cpu().tolist(), N)
        # a second call through the same scratch gives the same answer
        got2 = torch.zeros(2, dtype=torch.float64, device=dev)
        M.mlmc_level_noalloc(four, l, N, prec, kahan, icdf, params, 1234, off, got2)
        torch.cuda.synchronize()
        assert got2.cpu().tolist() == first
        _close(got2.cpu().tolist(), ref.cpu().tolist(), N)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    params = M.sde_params()
    out = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MlmcError) as e:
        M.mlmc_level_noalloc(0, 3, (1 << 21) + 1, M.MLMC_F32, False, M.MLMC_ICDF_TABLE, params, 1, 0, out)
    assert e.value.status == M.MLMC_EINVAL
    assert "scratch" in str(e.value)
