"""Python binding of libmlmc (include/mlmc.h): nested multilevel Monte Carlo
with low-precision approximate random variables on GB300 (sm_103a).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors on the current CUDA device; the
stream is torch's current stream unless one is given.  If the compiled
library is missing, every call raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmlmc.so")

# enums (include/mlmc.h)
MLMC_OK, MLMC_EINVAL, MLMC_ECUDA, MLMC_ETIMEOUT, MLMC_ENOMEM, MLMC_ENOTCONV, MLMC_ENOTREADY = range(7)
MLMC_GBM, MLMC_OU = 0, 1
MLMC_EULER, MLMC_MILSTEIN = 0, 1
MLMC_PAYOFF_X, MLMC_PAYOFF_CALL = 0, 1
MLMC_F32, MLMC_F16, MLMC_BF16 = 0, 1, 2
MLMC_ICDF_EXACT, MLMC_ICDF_TABLE, MLMC_ICDF_MLP, MLMC_ICDF_TABLE16, MLMC_ICDF_CUBIC = 0, 1, 2, 3, 4
MLMC_MLP_PARAMS = 1153
MLMC_MLP_GRID = 1 << 22
MLMC_MAX_LEVELS = 19


class MlmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mlmc status {status}: {message}")
        self.status = status


class mlmc_sde_params(ctypes.Structure):
    _fields_ = [("sde", ctypes.c_int32), ("payoff", ctypes.c_int32),
                ("p0", ctypes.c_double), ("p1", ctypes.c_double), ("p2", ctypes.c_double),
                ("x0", ctypes.c_double), ("T", ctypes.c_double), ("K", ctypes.c_double), ("disc", ctypes.c_double),
                ("scheme", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mlmc_sums(ctypes.Structure):
    """s1, s2, n, cost_ns as accumulated; mean and var filled by the library."""
    _fields_ = [("s1", ctypes.c_double), ("s2", ctypes.c_double), ("n", ctypes.c_uint64),
                ("cost_ns", ctypes.c_double), ("mean", ctypes.c_double), ("var", ctypes.c_double)]


class mlmc_train_opts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("batch", ctypes.c_uint32), ("lr0", ctypes.c_float),
                ("lr_min", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("seed", ctypes.c_uint64)]


class mlmc_work(ctypes.Structure):
    _fields_ = [("params", mlmc_sde_params), ("l", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("kahan", ctypes.c_int32), ("icdf", ctypes.c_int32),
                ("set_id", ctypes.c_int32), ("N", ctypes.c_uint64), ("path_offset", ctypes.c_uint64)]


class mlmc_round_record(ctypes.Structure):
    _fields_ = [("round", ctypes.c_int32), ("l", ctypes.c_int32), ("kind", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("kahan", ctypes.c_int32), ("icdf", ctypes.c_int32), ("kept", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("dn", ctypes.c_uint64), ("path_offset", ctypes.c_uint64),
                ("s1", ctypes.c_double), ("s2", ctypes.c_double), ("cost_ns", ctypes.c_double)]


class mlmc_run_opts(ctypes.Structure):
    _fields_ = [("estimator", ctypes.c_int32), ("prec", ctypes.c_int32), ("kahan", ctypes.c_int32),
                ("icdf", ctypes.c_int32), ("max_level", ctypes.c_int32), ("min_levels", ctypes.c_int32),
                ("n0", ctypes.c_uint64), ("seed", ctypes.c_uint64), ("alpha", ctypes.c_double),
                ("timeout_s", ctypes.c_double), ("trial_all", ctypes.c_int32), ("trace_cap", ctypes.c_int32),
                ("trace", ctypes.POINTER(mlmc_round_record))]


class mlmc_run_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("variance", ctypes.c_double), ("levels", ctypes.c_int32),
                ("rounds", ctypes.c_int32), ("wall_s", ctypes.c_double), ("path_steps", ctypes.c_double),
                ("n", (ctypes.c_uint64 * MLMC_MAX_LEVELS) * 2), ("mean", (ctypes.c_double * MLMC_MAX_LEVELS) * 2),
                ("var", (ctypes.c_double * MLMC_MAX_LEVELS) * 2), ("cost", (ctypes.c_double * MLMC_MAX_LEVELS) * 2),
                ("prec", ctypes.c_int32 * MLMC_MAX_LEVELS), ("kahan", ctypes.c_int32 * MLMC_MAX_LEVELS),
                ("efficiency", ctypes.c_double * MLMC_MAX_LEVELS), ("nested", ctypes.c_int32 * MLMC_MAX_LEVELS),
                ("trace_len", ctypes.c_int32), ("reserved", ctypes.c_int32), ("model_s", ctypes.c_double),
                ("device_s", ctypes.c_double), ("discarded_path_steps", ctypes.c_double)]


# exported symbols and their signatures
_P = ctypes.POINTER
_vp, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
_SIGS = {
    "mlmc_level": [_i32, _u64, _i32, _i32, _i32, _P(mlmc_sde_params), _u64, _u64, _P(mlmc_sums), _vp],
    "mlmc_nested_level": [_i32, _u64, _i32, _i32, _i32, _P(mlmc_sde_params), _u64, _u64, _P(mlmc_sums), _vp],
    "mlmc_level_async": [_i32, _i32, _u64, _i32, _i32, _i32, _P(mlmc_sde_params), _u64, _u64, _vp, _vp],
    "mlmc_level_noalloc": [_i32, _i32, _u64, _i32, _i32, _i32, _P(mlmc_sde_params), _u64, _u64, _vp, _vp],
    "mlmc_level_paths": [_i32, _i32, _u64, _i32, _i32, _i32, _P(mlmc_sde_params), _u64, _u64, _vp, _vp],
    "approx_icdf": [_vp, _vp, ctypes.c_size_t, _i32, _i32, _vp],
    "mlmc_philox4x32_10": [_vp, _vp, _vp, ctypes.c_size_t, _vp],
    "mlmc_uniforms": [_vp, _vp, ctypes.c_size_t, _vp],
    "mlmc_icdf_table": [_vp, _vp, _vp, _vp],
    "mlmc_icdf_cubic": [_vp, _vp, _vp, _vp],
    "mlmc_mlp_set_weights": [_vp, ctypes.c_size_t],
    "mlmc_mlp_get_weights": [_vp, ctypes.c_size_t],
    "mlmc_mlp_grid_table": [_vp, ctypes.c_size_t],
    "mlmc_mlp_grad": [_vp, _vp, ctypes.c_size_t, _vp, _vp, _vp],
    "mlmc_mlp_train": [_vp, _vp, ctypes.c_size_t, _P(mlmc_train_opts), _vp, _vp],
    "mlmc_batch": [_P(mlmc_work), _i32, _u64, _P(mlmc_sums), _vp],
    "mlmc_batch_async": [_P(mlmc_work), _i32, _u64, _vp, _vp],
    "mlmc_batch_descriptor_bytes": [],
    "mlmc_run": [ctypes.c_double, _P(mlmc_sde_params), _P(mlmc_run_opts), _P(mlmc_run_result)],
    "mlmc_optimal_samples": [_vp, _vp, _i32, ctypes.c_double, _vp],
    "mlmc_moments": [_vp, _u64, _vp, _vp],
    "mlmc_peak_probe": [_i32, _vp, _vp],
    "mlmc_strerror": [_i32],
    "mlmc_last_error": [],
    "mlmc_version": [],
    "mlmc_shutdown": [],
}
_CHAR_RET = {"mlmc_strerror", "mlmc_last_error", "mlmc_version"}
_SIZE_RET = {"mlmc_batch_descriptor_bytes"}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libmlmc.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"libmlmc.so not built ({path}); run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = (ctypes.c_char_p if name in _CHAR_RET
                              else ctypes.c_size_t if name in _SIZE_RET else ctypes.c_int)
            _lib = lib
    return _lib


def _check(status: int):
    if status != MLMC_OK:
        raise MlmcError(status, load().mlmc_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _buf(t, name, itemsize, n, dtype=None):
    """Device pointer of t after checking that the library may read or write n
    elements of itemsize bytes through it: a contiguous CUDA tensor on the
    current device (the one the library launches on), of the given dtype if
    any, with at least n elements."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, the library launches on cuda:{torch.cuda.current_device()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype} (got {t.dtype})")
    if t.element_size() != itemsize:
        raise ValueError(f"{name} must have {itemsize}-byte elements (got {t.dtype})")
    if t.numel() < n:
        raise ValueError(f"{name} needs at least {n} elements (has {t.numel()})")
    return ctypes.c_void_p(t.data_ptr())


def _f64(name, t, n):
    import torch
    return _buf(t, name, 8, n, torch.float64)


def sde_params(sde=MLMC_GBM, payoff=MLMC_PAYOFF_X, p0=0.05, p1=0.2, p2=0.0, x0=1.0, T=1.0, K=1.0,
               disc=None, scheme=0) -> mlmc_sde_params:
    """GBM: (p0, p1) = (mu, sigma); OU: (p0, p1, p2) = (theta, m, s).  The call
    is discounted by disc (default e^{-p0 T} for GBM, 1 for OU).  scheme:
    MLMC_EULER or MLMC_MILSTEIN."""
    import math
    if disc is None:
        disc = math.exp(-p0 * T) if sde == MLMC_GBM else 1.0
    return mlmc_sde_params(sde, payoff, p0, p1, p2, x0, T, K, disc, scheme, 0)


def mlmc_level(l, N, prec, kahan, icdf, params, seed, path_offset=0, stream=None) -> mlmc_sums:
    out = mlmc_sums()
    _check(load().mlmc_level(l, N, prec, int(kahan), icdf, ctypes.byref(params), seed, path_offset,
                             ctypes.byref(out), _stream(stream)))
    return out


def mlmc_nested_level(l, N, prec, kahan, icdf, params, seed, path_offset=0, stream=None) -> mlmc_sums:
    out = mlmc_sums()
    _check(load().mlmc_nested_level(l, N, prec, int(kahan), icdf, ctypes.byref(params), seed, path_offset,
                                    ctypes.byref(out), _stream(stream)))
    return out


def mlmc_level_async(four, l, N, prec, kahan, icdf, params, seed, path_offset, sums_dev, stream=None):
    """sums_dev: float64 CUDA tensor with >= 2 elements (receives sum D, sum D^2)."""
    _check(load().mlmc_level_async(int(four), l, N, prec, int(kahan), icdf, ctypes.byref(params), seed,
                                   path_offset, _f64("sums_dev", sums_dev, 2), _stream(stream)))


def mlmc_level_noalloc(four, l, N, prec, kahan, icdf, params, seed, path_offset, sums_dev, stream=None):
    """Allocation-free variant of mlmc_level_async (fixed device scratch, N <= 2^21)."""
    _check(load().mlmc_level_noalloc(int(four), l, N, prec, int(kahan), icdf, ctypes.byref(params), seed,
                                     path_offset, _f64("sums_dev", sums_dev, 2), _stream(stream)))


def mlmc_level_paths(four, l, N, prec, kahan, icdf, params, seed, path_offset, out_dev, stream=None):
    """out_dev: float32 CUDA tensor of N*3 (two-way) or N*5 (four-way) elements."""
    out = _buf(out_dev, "out_dev", 4, N * (5 if four else 3))
    _check(load().mlmc_level_paths(int(four), l, N, prec, int(kahan), icdf, ctypes.byref(params), seed,
                                   path_offset, out, _stream(stream)))


def approx_icdf(u_dev, z_dev, icdf, prec, stream=None):
    """u_dev float32; z_dev with 4-byte (F32) or 2-byte (F16, BF16: the format's bits) elements, as many."""
    n = u_dev.numel()
    u = _buf(u_dev, "u_dev", 4, n)
    z = _buf(z_dev, "z_dev", 4 if prec == MLMC_F32 else 2, n)
    _check(load().approx_icdf(u, z, n, icdf, prec, _stream(stream)))


def mlmc_philox4x32_10(ctr_dev, key_dev, out_dev, stream=None):
    """ctr_dev (n, 4), key_dev (n, 2), out_dev (n, 4): int32 CUDA tensors holding uint32 bits."""
    n = ctr_dev.shape[0]
    _check(load().mlmc_philox4x32_10(_buf(ctr_dev, "ctr_dev", 4, 4 * n), _buf(key_dev, "key_dev", 4, 2 * n),
                                     _buf(out_dev, "out_dev", 4, 4 * n), n, _stream(stream)))


def mlmc_uniforms(w_dev, u_dev, stream=None):
    n = w_dev.numel()
    _check(load().mlmc_uniforms(_buf(w_dev, "w_dev", 4, n), _buf(u_dev, "u_dev", 4, n), n, _stream(stream)))


def mlmc_icdf_table():
    """(c64, c32, c16 bits, bf16 bits), each (16, 2), as built on the device."""
    import numpy as np
    c64 = np.zeros(32, np.float64)
    c32 = np.zeros(32, np.float32)
    c16 = np.zeros(32, np.uint16)
    cbf = np.zeros(32, np.uint16)
    _check(load().mlmc_icdf_table(c64.ctypes.data_as(_vp), c32.ctypes.data_as(_vp), c16.ctypes.data_as(_vp),
                                  cbf.ctypes.data_as(_vp)))
    return c64.reshape(16, 2), c32.reshape(16, 2), c16.reshape(16, 2), cbf.reshape(16, 2)


def mlmc_icdf_cubic():
    """(d64, d32, d16 bits, bf16 bits), each (16, 4), as built on the device."""
    import numpy as np
    d64 = np.zeros(64, np.float64)
    d32 = np.zeros(64, np.float32)
    d16 = np.zeros(64, np.uint16)
    dbf = np.zeros(64, np.uint16)
    _check(load().mlmc_icdf_cubic(d64.ctypes.data_as(_vp), d32.ctypes.data_as(_vp), d16.ctypes.data_as(_vp),
                                  dbf.ctypes.data_as(_vp)))
    return d64.reshape(16, 4), d32.reshape(16, 4), d16.reshape(16, 4), dbf.reshape(16, 4)


def mlmc_mlp_set_weights(w):
    import numpy as np
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check(load().mlmc_mlp_set_weights(w.ctypes.data_as(_vp), w.size))


def mlmc_mlp_get_weights():
    import numpy as np
    w = np.zeros(MLMC_MLP_PARAMS, np.float32)
    _check(load().mlmc_mlp_get_weights(w.ctypes.data_as(_vp), w.size))
    return w


def mlmc_mlp_grid_table():
    """The network's y on the 2^22 grid points v_k = (2k + 1) 2^-24, as tabulated on the device."""
    import numpy as np
    y = np.zeros(1 << 22, np.float32)
    _check(load().mlmc_mlp_grid_table(y.ctypes.data_as(_vp), y.size))
    return y


def mlmc_mlp_grad(u_dev, z_dev, grad_dev, stream=None) -> float:
    loss = ctypes.c_float(0.0)
    n = u_dev.numel()
    _check(load().mlmc_mlp_grad(_buf(u_dev, "u_dev", 4, n), _buf(z_dev, "z_dev", 4, n), n,
                                _buf(grad_dev, "grad_dev", 4, MLMC_MLP_PARAMS), ctypes.byref(loss), _stream(stream)))
    return float(loss.value)


def mlmc_mlp_train(u_dev, z_dev, opts: mlmc_train_opts, stream=None) -> float:
    loss = ctypes.c_float(0.0)
    n = u_dev.numel()
    zp = _buf(z_dev, "z_dev", 4, n) if z_dev is not None else ctypes.c_void_p(0)
    _check(load().mlmc_mlp_train(_buf(u_dev, "u_dev", 4, n), zp, n, ctypes.byref(opts), ctypes.byref(loss),
                                 _stream(stream)))
    return float(loss.value)


def mlmc_batch(items, seed, stream=None):
    arr = (mlmc_work * len(items))(*items)
    out = (mlmc_sums * len(items))()
    _check(load().mlmc_batch(arr, len(items), seed, out, _stream(stream)))
    return list(out)


def mlmc_batch_async(items, seed, sums_dev, stream=None):
    """sums_dev: float64 CUDA tensor with >= 2 * len(items) elements."""
    arr = (mlmc_work * len(items))(*items)
    _check(load().mlmc_batch_async(arr, len(items), seed, _f64("sums_dev", sums_dev, 2 * len(items)),
                                   _stream(stream)))


def mlmc_batch_descriptor_bytes() -> int:
    return int(load().mlmc_batch_descriptor_bytes())


def mlmc_run(eps, params, opts: mlmc_run_opts, trace_cap: int = 0):
    """Adaptive MLMC to RMSE eps.  With trace_cap > 0 returns (result, the
    run's draws as a list of mlmc_round_record) instead of the result."""
    out = mlmc_run_result()
    trace = None
    if trace_cap > 0:
        trace = (mlmc_round_record * trace_cap)()
        opts = mlmc_run_opts.from_buffer_copy(opts)
        opts.trace_cap = trace_cap
        opts.trace = ctypes.cast(trace, ctypes.POINTER(mlmc_round_record))
    _check(load().mlmc_run(eps, ctypes.byref(params), ctypes.byref(opts), ctypes.byref(out)))
    if trace is None:
        return out
    return out, list(trace[:min(out.trace_len, trace_cap)])


def mlmc_moments(s1, s2, n):
    """(mean, var) of a level from its sums, combined by the library."""
    sums = (ctypes.c_double * 2)(float(s1), float(s2))
    mean, var = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().mlmc_moments(ctypes.cast(sums, _vp), int(n), ctypes.byref(mean), ctypes.byref(var)))
    return mean.value, var.value


def mlmc_optimal_samples(V, C, eps):
    import numpy as np
    V = np.ascontiguousarray(V, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    N = np.zeros(V.size, np.uint64)
    _check(load().mlmc_optimal_samples(V.ctypes.data_as(_vp), C.ctypes.data_as(_vp), V.size, eps,
                                       N.ctypes.data_as(_vp)))
    return N


def mlmc_peak_probe(kind, stream=None) -> float:
    v = ctypes.c_double(0.0)
    _check(load().mlmc_peak_probe(kind, ctypes.byref(v), _stream(stream)))
    return float(v.value)


def mlmc_version() -> str:
    return load().mlmc_version().decode()


def mlmc_shutdown():
    _check(load().mlmc_shutdown())


def exported_symbols():
    return list(_SIGS)
