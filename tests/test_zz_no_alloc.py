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


def test_noalloc_at_the_scratch_boundary():
    """N = 2^21 fills all 4096 block slots of the fixed scratch (one sample
    pair per thread, 256 threads per block); 2^21 - 1 leaves the last pair
    half full.  Both against the allocating entry point, on the same
    samples, and a level-0 call (4 samples per lane slot) inside the bound."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda:0")
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    for four, l, N, prec, kahan, icdf in ((0, 3, 1 << 21, M.MLMC_F16, True, M.MLMC_ICDF_TABLE),
                                         (1, 2, (1 << 21) - 1, M.MLMC_F32, False, M.MLMC_ICDF_TABLE),
                                         (0, 0, 1 << 21, M.MLMC_F32, False, M.MLMC_ICDF_EXACT)):
        got = torch.zeros(2, dtype=torch.float64, device=dev)
        ref = torch.zeros(2, dtype=torch.float64, device=dev)
        M.mlmc_level_noalloc(four, l, N, prec, kahan, icdf, params, 99, 0, got)
        M.mlmc_level_async(four, l, N, prec, kahan, icdf, params, 99, 0, ref)
        torch.cuda.synchronize()
        _close(got.cpu().tolist(), ref.cpu().tolist(), N)


def test_noalloc_sums_match_the_oracle():
    """The allocation-free call's sums against the oracle's level sums on the
    same samples (binary16 + Kahan paths are bit-exact per sample; the sums
    differ by the FP32 per-lane accumulation only)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as O
    from oracle import table
    params = M.sde_params(sde=M.MLMC_GBM, payoff=M.MLMC_PAYOFF_CALL, p0=0.05, p1=0.2, K=1.0)
    osde = O.SDE(params.sde, params.payoff, params.p0, params.p1, params.p2, params.x0, params.T, params.K,
                 params.disc)
    N, l = 20000, 5
    got = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    M.mlmc_level_noalloc(0, l, N, M.MLMC_F16, True, M.MLMC_ICDF_TABLE, params, 1234, 0, got)
    torch.cuda.synchronize()
    s1, s2 = got.cpu().tolist()
    o1, o2 = O.level_sums(l, N, 0, O.variant(prec=O.F16, kahan=True, rv=O.RV_TABLE), osde, 1234,
                          O.make_tag(O.KIND_APPROX, l), table=table.build_table(), nthreads=4)
    assert abs(s1 - o1) <= 1e-6 * (abs(o1) + math.sqrt(o2))
    assert abs(s2 - o2) <= 1e-6 * o2
