"""CPU checks of the C ABI: the library loads, exports every entry point that
include/mlmc.h declares, rejects invalid arguments before any launch, and
its host-only sample allocation matches the oracle's (Sec. 3)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2012_09739_gb300 as M
from paper_2012_09739_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return M.load()


def _declared():
    with open(os.path.join(ROOT, "include", "mlmc.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:mlmc_status|const char \*|size_t)\s*(\w+)\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mlmc_level", "mlmc_nested_level", "approx_icdf", "mlmc_run", "mlmc_batch", "mlmc_batch_async",
              "mlmc_mlp_train"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    # and the binding wraps each of them
    assert sorted(M.exported_symbols()) == sorted(_declared())


def test_invalid_arguments_rejected_without_gpu(lib):
    p = M.sde_params()
    out = M.mlmc_sums()
    bad = [
        (19, 10, 0, 0, 0, p),       # level above 18
        (-1, 10, 0, 0, 0, p),
        (3, 0, 0, 0, 0, p),         # N = 0
        (3, 10, 7, 0, 0, p),        # precision
        (3, 10, 0, 0, 5, p),        # icdf kind
        (3, 10, 0, 0, 0, M.sde_params(p1=-0.2)),     # sigma <= 0
        (3, 10, 0, 0, 0, M.sde_params(T=0.0)),
        (3, 10, 0, 0, 0, M.sde_params(p0=float("nan"))),
        (3, 10, 0, 0, 0, M.sde_params(sde=M.MLMC_OU, p2=0.0)),
    ]
    for l, N, prec, kahan, icdf, params in bad:
        st = lib.mlmc_level(l, N, prec, kahan, icdf, ctypes.byref(params), 1, 0, ctypes.byref(out), None)
        assert st == M.MLMC_EINVAL, (l, N, prec, icdf)
        assert lib.mlmc_last_error()
    st = lib.mlmc_nested_level(3, 10, 0, 0, M.MLMC_ICDF_EXACT, ctypes.byref(p), 1, 0, ctypes.byref(out), None)
    assert st == M.MLMC_EINVAL
    st = lib.mlmc_level(3, 10, 0, 0, 0, None, 1, 0, ctypes.byref(out), None)
    assert st == M.MLMC_EINVAL
    assert lib.mlmc_strerror(M.MLMC_ETIMEOUT) == b"timeout"


def test_batch_arguments_rejected_without_gpu(lib):
    """Both batch entry points validate every item (and the output pointer)
    before they touch a device."""
    p = M.sde_params()
    good = M.mlmc_work(p, 3, 1, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 1000, 0)
    bad = [M.mlmc_work(p, 3, 2, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 1000, 0),      # kind
           M.mlmc_work(p, 19, 0, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 1000, 0),     # level
           M.mlmc_work(p, 3, 1, M.MLMC_F16, 1, M.MLMC_ICDF_EXACT, 0, 1000, 0),      # four-way exact
           M.mlmc_work(p, 3, 0, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 70000, 1000, 0),  # set id
           M.mlmc_work(p, 3, 0, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 0, 0)]         # N = 0
    out = (M.mlmc_sums * 2)()
    sums = (ctypes.c_double * 4)()
    for b in bad:
        arr = (M.mlmc_work * 2)(good, b)
        assert lib.mlmc_batch(arr, 2, 1, out, None) == M.MLMC_EINVAL
        assert lib.mlmc_batch_async(arr, 2, 1, ctypes.cast(sums, ctypes.c_void_p), None) == M.MLMC_EINVAL
    arr = (M.mlmc_work * 1)(good)
    assert lib.mlmc_batch_async(arr, 1, 1, None, None) == M.MLMC_EINVAL
    assert lib.mlmc_batch(arr, 0, 1, out, None) == M.MLMC_EINVAL
    assert 128 <= M.mlmc_batch_descriptor_bytes() <= 1024 and M.mlmc_batch_descriptor_bytes() % 8 == 0


def test_optimal_samples_match_oracle(lib):
    from oracle import mlmc
    rng = np.random.default_rng(0)
    for _ in range(20):
        n = int(rng.integers(1, 19))
        V = rng.uniform(1e-8, 1e-1, n)
        C = rng.uniform(1.0, 1e4, n)
        eps = float(rng.uniform(1e-4, 1e-2))
        assert np.array_equal(M.mlmc_optimal_samples(V, C, eps).astype(np.int64), mlmc.optimal_samples(V, C, eps))
    with pytest.raises(M.MlmcError):
        M.mlmc_optimal_samples([1.0], [0.0], 1e-3)


def test_binding_checks_device_buffers_without_gpu(lib):
    """The binding hands the library only device pointers it may use: a host
    tensor, a wrong dtype or too few elements is refused before any call."""
    torch = pytest.importorskip("torch")
    p = M.sde_params()
    items = [M.mlmc_work(p, 3, 0, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, 0, 1000, 0)] * 3
    host = torch.zeros(6, dtype=torch.float64)
    for call in (lambda: M.mlmc_batch_async(items, 1, host),
                 lambda: M.mlmc_level_async(0, 3, 1000, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, p, 1, 0, host),
                 lambda: M.mlmc_level_noalloc(0, 3, 1000, M.MLMC_F16, 1, M.MLMC_ICDF_TABLE, p, 1, 0, host),
                 lambda: M.approx_icdf(torch.zeros(8), torch.zeros(8), M.MLMC_ICDF_TABLE, M.MLMC_F32),
                 lambda: M.mlmc_uniforms(torch.zeros(8, dtype=torch.int32), torch.zeros(8))):
        with pytest.raises(ValueError):
            call()
    with pytest.raises(ValueError):
        M._buf(torch.zeros(4, dtype=torch.float32), "x", 8, 1)


def test_moments_match_exact_rational_arithmetic(lib):
    """mlmc_moments (the one routine every result struct and the adaptive
    driver use for a level's mean and variance, Sec. 3) against the same
    statistics in exact rational arithmetic, on samples whose FP64 sums are
    exact (dyadic rationals of few bits): mean to 1 ulp, variance to a few ulp of
    the cancellation-bound s2 (the sums carry no rounding of their own)."""
    from fractions import Fraction
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = int(rng.integers(1, 5000))
        shift = float(rng.choice([0.0, 0.1, 1.0, 100.0]))
        # samples on a 2^-10 grid below 2^8: their sums and sums of squares
        # need at most 49 significant bits, so they are exact in FP64
        x = np.round((shift + rng.standard_normal(n)) * 2 ** 10) / 2 ** 10
        s1 = float(np.sum(x))
        s2 = float(np.sum(x * x))
        fx = [Fraction(v) for v in x.tolist()]
        assert Fraction(s1) == sum(fx) and Fraction(s2) == sum(v * v for v in fx)
        mean, var = M.mlmc_moments(s1, s2, n)
        em = sum(fx) / n
        ev = (sum(v * v for v in fx) - sum(fx) * em) / (n - 1) if n > 1 else Fraction(0)
        assert abs(Fraction(mean) - em) <= abs(em) * Fraction(2) ** -52
        assert abs(Fraction(var) - ev) <= (Fraction(s2) / max(n - 1, 1)) * Fraction(2) ** -50 + Fraction(0)
        assert var >= 0.0
    # a single sample has no spread; n = 0 is refused
    assert M.mlmc_moments(3.0, 9.0, 1) == (3.0, 0.0)
    with pytest.raises(M.MlmcError):
        M.mlmc_moments(1.0, 1.0, 0)
    # the sums struct carries the same moments (filled by the library)
    s = M.mlmc_sums()
    assert hasattr(s, "mean") and hasattr(s, "var")
