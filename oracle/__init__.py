"""Oracle for the nested multilevel Monte Carlo method with low-precision
approximate random variables (Giles & Sheridan-Methven, arXiv 2012.09739).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow FP64 CPU
restatement of the method used to check the CUDA library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline and reference legs of
``bench.py`` may import it.  It imports nothing from the CUDA package and the CUDA package
imports nothing from it.

Modules:
  oracle.c        Philox4x32-10, uniforms, exact inverse CDF, per-operation
                  rounding (binary16/binary32/p-bit), Euler-Maruyama with and
                  without Kahan summation, two-way and four-way samples.
  table.py        L2 piecewise-linear fit of the inverse CDF (Sec. 2.1).
  mlp.py          MLP surrogate forward / backward / Adam in FP64.
  mlmc.py         closed forms and the adaptive MLMC driver (Sec. 3).

Parity status of each function is listed in its docstring; everything here
is pinned by ``tests/test_oracle_*.py`` except where a docstring says
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# precision codes (oracle.c)
F64, F32, F16, BF16, PBITS = 0, 1, 2, 3, 4
# random-variable kinds
RV_EXACT, RV_TABLE, RV_MLP, RV_TABLE16, RV_CUBIC, RV_MLP16 = 0, 1, 2, 3, 4, 5
# SDEs and payoffs
GBM, OU = 0, 1
PAYOFF_X, PAYOFF_CALL = 0, 1
# counter tags: estimator kind
KIND_STD, KIND_APPROX, KIND_FOUR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc: -O2, strict IEEE (no fast-math, no FMA
    contraction, which would change the rounding the oracle emulates)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off",
           "-fno-strict-aliasing", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class SDE(ctypes.Structure):
    """Mirror of orc_sde: GBM (p0, p1) = (mu, sigma); OU (p0, p1, p2) =
    (theta, m, s).  Call payoff disc * max(X_T - K, 0).  scheme 0: Euler,
    1: Milstein."""
    _fields_ = [("sde", ctypes.c_int), ("payoff", ctypes.c_int),
                ("p0", ctypes.c_double), ("p1", ctypes.c_double), ("p2", ctypes.c_double),
                ("x0", ctypes.c_double), ("T", ctypes.c_double), ("K", ctypes.c_double),
                ("disc", ctypes.c_double), ("scheme", ctypes.c_int)]


def gbm(mu=0.05, sigma=0.2, x0=1.0, T=1.0, payoff=PAYOFF_X, K=1.0, disc=None, scheme=0) -> SDE:
    """GBM dX = mu X dt + sigma X dW (Sec. 2.2 experiments); call payoff
    discounted at r = mu unless disc is given; scheme 1: Milstein."""
    if disc is None:
        disc = float(np.exp(-mu * T))
    return SDE(GBM, payoff, mu, sigma, 0.0, x0, T, K, disc, scheme)


def ou(theta, m, s, x0=1.0, T=1.0, payoff=PAYOFF_X, K=0.0, disc=1.0) -> SDE:
    """Ornstein-Uhlenbeck dX = theta (m - X) dt + s dW."""
    return SDE(OU, payoff, theta, m, s, x0, T, K, disc)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            u32p, u64p = P(ctypes.c_uint32), P(ctypes.c_uint64)
            dp, ip = P(ctypes.c_double), P(ctypes.c_int)
            i64 = ctypes.c_int64
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p, i64]
            L.orc_u32_to_uniform.argtypes = [u32p, dp, i64]
            L.orc_ndtri.argtypes = [dp, dp, i64]
            L.orc_ndtri1.argtypes = [ctypes.c_double]
            L.orc_ndtri1.restype = ctypes.c_double
            L.orc_round_bits.argtypes = [dp, dp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_double]
            L.orc_approx_icdf.argtypes = [dp, dp, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            L.orc_twoway_paths.argtypes = [ctypes.c_int, u64p, i64, ip, P(SDE), ctypes.c_uint64,
                                           ctypes.c_uint32, dp, dp, dp]
            L.orc_fourway_paths.argtypes = [ctypes.c_int, u64p, i64, ip, ip, P(SDE), ctypes.c_uint64,
                                            ctypes.c_uint32, dp, dp, dp]
            L.orc_level_sums.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ip, ip,
                                         P(SDE), ctypes.c_uint64, ctypes.c_uint32, dp, dp, ctypes.c_int, dp]
            L.orc_rounding_pairs.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ip, P(SDE),
                                             ctypes.c_uint64, ctypes.c_uint32, dp, dp, dp]
            L.orc_mlp_feature32.argtypes = [ctypes.c_double]
            L.orc_mlp_feature32.restype = ctypes.c_double
            L.orc_tanh16.argtypes = [ctypes.c_double]
            L.orc_tanh16.restype = ctypes.c_double
            L.orc_kahan_sum.argtypes = [dp, i64, ctypes.c_int, ctypes.c_int]
            L.orc_kahan_sum.restype = ctypes.c_double
            L.orc_openmp_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of counters ctr (n, 4) under keys key (n, 2) -> (n, 4) uint32."""
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, dtype=np.uint32), (ctr.shape[0], 2)))
    out = np.empty_like(ctr)
    lib().orc_philox4x32_10(_ptr(ctr, ctypes.c_uint32), _ptr(key, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32), ctr.shape[0])
    return out


def uniforms(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32).ravel()
    u = np.empty(w.shape, np.float64)
    lib().orc_u32_to_uniform(_ptr(w, ctypes.c_uint32), _ptr(u, ctypes.c_double), w.size)
    return u


def uniforms16(halves) -> np.ndarray:
    """u = (h + 1/2) 2^-16 for 16-bit values h (the low 16 bits are used)."""
    h = np.ascontiguousarray(halves, dtype=np.uint32).ravel()
    u = np.empty(h.shape, np.float64)
    lib().orc_u16_to_uniform(_ptr(h, ctypes.c_uint32), _ptr(u, ctypes.c_double), h.size)
    return u


def q16(u) -> np.ndarray:
    """Centre of the 2^-16-wide cell of (0, 1) that contains u."""
    u = _f64(u).ravel()
    q = np.empty_like(u)
    lib().orc_q16(_ptr(u, ctypes.c_double), _ptr(q, ctypes.c_double), u.size)
    return q


def counters(path_idx, j, tag) -> np.ndarray:
    """Counter words (path lo32, path hi32, j, tag) for the given paths."""
    p = np.asarray(path_idx, dtype=np.uint64).ravel()
    c = np.empty((p.size, 4), np.uint32)
    c[:, 0] = (p & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    c[:, 1] = (p >> np.uint64(32)).astype(np.uint32)
    c[:, 2] = np.uint32(j)
    c[:, 3] = np.uint32(tag)
    return c


def seed_key(seed: int) -> np.ndarray:
    return np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)


def make_tag(kind: int, level: int, set_id: int = 0) -> int:
    return int(kind) | (int(level) << 8) | (int(set_id) << 16)


def ndtri(p) -> np.ndarray:
    """Exact inverse Gaussian CDF in FP64 (A&S 26.2.23 guess + Halley)."""
    p = _f64(p).ravel()
    x = np.empty_like(p)
    lib().orc_ndtri(_ptr(p, ctypes.c_double), _ptr(x, ctypes.c_double), p.size)
    return x


_FMT = {F32: (24, -126, 3.4028234663852886e38), F16: (11, -14, 65504.0),
        BF16: (8, -126, 3.3895313892515355e38)}


def round_bits(x, prec: int, pbits: int = 53) -> np.ndarray:
    """Round to binary32/binary16/bfloat16 or a p-bit significand (RNE)."""
    x = _f64(x).ravel()
    y = np.empty_like(x)
    if prec == F64:
        return x.copy()
    p, emin, maxv = _FMT.get(prec, (pbits, -1022, 1.0e308))
    lib().orc_round_bits(_ptr(x, ctypes.c_double), _ptr(y, ctypes.c_double), x.size, p, emin, maxv)
    return y


_NO_MLP = np.zeros(1153)
_NO_TABLE = np.zeros(32)
_NO_CUBIC = np.zeros(64)


def _tables(table, cubic):
    """The linear table (16 x 2) followed by the cubic one (16 x 4), as the C
    entry points take them."""
    t = _f64(table if table is not None else _NO_TABLE).ravel()
    c = _f64(cubic if cubic is not None else _NO_CUBIC).ravel()
    assert t.size == 32 and c.size == 64
    return np.ascontiguousarray(np.concatenate([t, c]))


def mlp_feature32(v) -> np.ndarray:
    """The network input t = sqrt(-2 ln v) from binary32 operations (the
    binary16 inference reading of the learned part)."""
    return np.array([lib().orc_mlp_feature32(float(x)) for x in np.ravel(v)])


def tanh16(x) -> np.ndarray:
    """The activation of the binary16 inference reading: tanh of x rounded to
    binary16, correctly rounded to binary16."""
    return np.array([lib().orc_tanh16(float(a)) for a in np.ravel(x)])


def approx_icdf(u, rv: int, prec: int = F64, pbits: int = 53, table=None, mlp=None, cubic=None) -> np.ndarray:
    """Phi^-1 (rv=RV_EXACT), piecewise-linear table (RV_TABLE), the table at
    the 16-bit cell centre q16(u) (RV_TABLE16), piecewise cubic (RV_CUBIC,
    coefficients `cubic`), the FP64 MLP (RV_MLP) or the MLP in binary16
    inference arithmetic (RV_MLP16), rounded to precision prec."""
    u = _f64(u).ravel()
    z = np.empty_like(u)
    t = _tables(table, cubic)
    w = _f64(mlp if mlp is not None else _NO_MLP)
    lib().orc_approx_icdf(_ptr(u, ctypes.c_double), _ptr(z, ctypes.c_double), u.size, rv, prec, pbits,
                          _ptr(t, ctypes.c_double), _ptr(w, ctypes.c_double))
    return z


def variant(prec=F64, kahan=False, rv=RV_EXACT, pbits=53) -> np.ndarray:
    return np.array([prec, pbits, int(bool(kahan)), rv], dtype=np.int32)


def twoway_paths(l, idx, var, sde: SDE, seed, tag, table=None, mlp=None, cubic=None) -> np.ndarray:
    """Per-path (P_fine, P_coarse, D) of the two-way difference at level l."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64).ravel()
    out = np.empty((idx.size, 3), np.float64)
    t = _tables(table, cubic)
    w = _f64(mlp if mlp is not None else _NO_MLP)
    var = np.ascontiguousarray(var, dtype=np.int32)
    lib().orc_twoway_paths(l, _ptr(idx, ctypes.c_uint64), idx.size, _ptr(var, ctypes.c_int), ctypes.byref(sde),
                           seed, tag, _ptr(t, ctypes.c_double), _ptr(w, ctypes.c_double),
                           _ptr(out, ctypes.c_double))
    return out


def fourway_paths(l, idx, hat, bar, sde: SDE, seed, tag, table=None, mlp=None, cubic=None) -> np.ndarray:
    """Per-path (P^_f, P^_c, P-_f, P-_c, D) of the four-way difference."""
    idx = np.ascontiguousarray(idx, dtype=np.uint64).ravel()
    out = np.empty((idx.size, 5), np.float64)
    t = _tables(table, cubic)
    w = _f64(mlp if mlp is not None else _NO_MLP)
    hat = np.ascontiguousarray(hat, dtype=np.int32)
    bar = np.ascontiguousarray(bar, dtype=np.int32)
    lib().orc_fourway_paths(l, _ptr(idx, ctypes.c_uint64), idx.size, _ptr(hat, ctypes.c_int),
                            _ptr(bar, ctypes.c_int), ctypes.byref(sde), seed, tag, _ptr(t, ctypes.c_double),
                            _ptr(w, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def level_sums(l, N, path_offset, var, sde: SDE, seed, tag, table=None, mlp=None, cubic=None, four=False, var2=None,
               nthreads=1) -> tuple[float, float]:
    """(sum D, sum D^2) over paths path_offset .. path_offset+N-1."""
    t = _tables(table, cubic)
    w = _f64(mlp if mlp is not None else _NO_MLP)
    var = np.ascontiguousarray(var, dtype=np.int32)
    var2 = np.ascontiguousarray(var2 if var2 is not None else var, dtype=np.int32)
    sums = np.zeros(2)
    lib().orc_level_sums(l, N, path_offset, int(four), _ptr(var, ctypes.c_int), _ptr(var2, ctypes.c_int),
                         ctypes.byref(sde), seed, tag, _ptr(t, ctypes.c_double), _ptr(w, ctypes.c_double),
                         nthreads, _ptr(sums, ctypes.c_double))
    return float(sums[0]), float(sums[1])


def rounding_pairs(l, N, path_offset, var, sde: SDE, seed, tag, table=None, mlp=None, cubic=None) -> np.ndarray:
    """(X_T in FP64, X_T in working precision) driven by the same normals."""
    t = _tables(table, cubic)
    w = _f64(mlp if mlp is not None else _NO_MLP)
    var = np.ascontiguousarray(var, dtype=np.int32)
    out = np.empty((N, 2), np.float64)
    lib().orc_rounding_pairs(l, N, path_offset, _ptr(var, ctypes.c_int), ctypes.byref(sde), seed, tag,
                             _ptr(t, ctypes.c_double), _ptr(w, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def kahan_sum(x, prec: int, pbits: int = 53) -> float:
    """Kahan compensated summation (Algorithm 1) in working precision."""
    x = _f64(x).ravel()
    return float(lib().orc_kahan_sum(_ptr(x, ctypes.c_double), x.size, prec, pbits))


def openmp_threads() -> int:
    return int(lib().orc_openmp_threads())
