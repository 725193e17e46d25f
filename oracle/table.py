"""Piecewise-linear approximate inverse Gaussian CDF (Sec. 2.1, Fig. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper defers the construction to its cited work; the reading used here:
on v = min(u, 1-u) the 16 intervals are I_k = [2^-(k+1), 2^-k) for
k = 1..15 and I_16 = (0, 2^-16); on each interval g(v) = c0 + c1 v is the
least-squares (L2 in the uniform measure) linear fit of Phi^-1, and the
approximation is mirrored: Phi~^-1(u) = g(u) for u <= 1/2, -g(1-u) above.

The moments are computed by 24-point Gauss-Legendre quadrature on dyadic
sub-intervals (Phi^-1 is smooth on each; the logarithmic singularity at 0
is resolved by the dyadic refinement), with the oracle's own FP64 Phi^-1.
"""
from __future__ import annotations

import numpy as np

from . import ndtri

N_INTERVALS = 16
_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


def interval_bounds(k: int) -> tuple[float, float]:
    """Bounds (a, b) of interval k = 1..16 on v in (0, 1/2]."""
    if k < N_INTERVALS:
        return 2.0 ** -(k + 1), 2.0 ** -k
    return 0.0, 2.0 ** -N_INTERVALS


def _pieces(a: float, b: float) -> list[tuple[float, float]]:
    if a > 0.0:
        return [(a, b)]
    # (0, b]: dyadic pieces [b 2^-(j+1), b 2^-j], j = 0..199; the remainder
    # below b 2^-200 contributes < 1e-60 to every moment.
    return [(b * 2.0 ** -(j + 1), b * 2.0 ** -j) for j in range(200)]


def moments(a: float, b: float, f=None) -> np.ndarray:
    """[int 1, int v, int v^2, int f, int v f] over (a, b), f = Phi^-1 by default."""
    f = f or ndtri
    acc = np.zeros(5)
    for lo, hi in _pieces(a, b):
        half, mid = 0.5 * (hi - lo), 0.5 * (hi + lo)
        v = mid + half * _GL_X
        w = half * _GL_W
        fv = f(v)
        acc += np.array([w.sum(), (w * v).sum(), (w * v * v).sum(), (w * fv).sum(), (w * v * fv).sum()])
    return acc


def build_table() -> np.ndarray:
    """(16, 2) array of (c0, c1): the L2 linear fit of Phi^-1 on each interval."""
    tab = np.zeros((N_INTERVALS, 2))
    for k in range(1, N_INTERVALS + 1):
        m0, m1, m2, f0, f1 = moments(*interval_bounds(k))
        # normal equations [m0 m1; m1 m2] [c0; c1] = [f0; f1], solved in
        # centred form: c1 = int (v - vbar) f / int (v - vbar)^2
        vbar = m1 / m0
        c1 = (f1 - vbar * f0) / (m2 - vbar * m1)
        c0 = f0 / m0 - c1 * vbar
        tab[k - 1] = (c0, c1)
    return tab


def l2_error(tab: np.ndarray) -> float:
    """E|Z - Z~|^2 for U uniform on (0, 1): twice the integral over (0, 1/2)."""
    total = 0.0
    for k in range(1, N_INTERVALS + 1):
        a, b = interval_bounds(k)
        c0, c1 = tab[k - 1]
        for lo, hi in _pieces(a, b):
            half, mid = 0.5 * (hi - lo), 0.5 * (hi + lo)
            v = mid + half * _GL_X
            total += (half * _GL_W * (ndtri(v) - c0 - c1 * v) ** 2).sum()
    return 2.0 * total
