"""Piecewise-linear and piecewise-cubic approximate inverse Gaussian CDFs
(Sec. 2.1, Fig. 1; the cubic is the high-fidelity approximation the paper
uses for its rounding-error experiments in Sec. 2.2, Fig. 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper defers the construction to its cited work; the reading used here:
on v = min(u, 1-u) the 16 intervals are I_k = [2^-(k+1), 2^-k) for
k = 1..15 and I_16 = (0, 2^-16); on each interval g(v) = c0 + c1 v is the
least-squares (L2 in the uniform measure) linear fit of Phi^-1, and the
approximation is mirrored: Phi~^-1(u) = g(u) for u <= 1/2, -g(1-u) above.
The cubic uses the same intervals and mirroring with the L2 fit of degree 3,
written in the interval's own variable s in [-1, 1] (s = v 2^(k+2) - 3 on
I_k, k <= 15, s = v 2^17 - 1 on I_16): g(v) = d0 + d1 s + d2 s^2 + d3 s^3.
(Readings: the paper takes the cubic from its cited work; the interval set,
the L2 criterion and the local variable s are this oracle's.)

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


def cubic_map(k: int) -> tuple[float, float]:
    """(A, B) of the local variable s = A v - B on interval k = 1..16."""
    if k < N_INTERVALS:
        return 2.0 ** (k + 2), 3.0
    return 2.0 ** (N_INTERVALS + 1), 1.0


def build_cubic_table() -> np.ndarray:
    """(16, 4) array of (d0, d1, d2, d3): the L2 cubic fit of Phi^-1 on each
    interval in its variable s.  Computed as the orthogonal projection on
    the Legendre polynomials P0..P3 of s (a_j = (2j+1)/2 int f P_j ds), then
    expanded in powers of s."""
    tab = np.zeros((N_INTERVALS, 4))
    for k in range(1, N_INTERVALS + 1):
        A, B = cubic_map(k)
        a_lo, b_hi = interval_bounds(k)
        proj = np.zeros(4)
        for lo, hi in _pieces(a_lo, b_hi):
            half, mid = 0.5 * (hi - lo), 0.5 * (hi + lo)
            v = mid + half * _GL_X
            w = half * _GL_W * A            # ds = A dv
            s = A * v - B
            fv = ndtri(v)
            leg = np.array([np.ones_like(s), s, 0.5 * (3 * s * s - 1), 0.5 * (5 * s ** 3 - 3 * s)])
            proj += (leg * (w * fv)).sum(axis=1)
        a = proj * (2 * np.arange(4) + 1) / 2.0
        tab[k - 1] = (a[0] - 0.5 * a[2], a[1] - 1.5 * a[3], 1.5 * a[2], 2.5 * a[3])
    return tab


def cubic_l2_error(tab: np.ndarray) -> float:
    """E|Z - Z~|^2 of the piecewise cubic for U uniform on (0, 1)."""
    total = 0.0
    for k in range(1, N_INTERVALS + 1):
        A, B = cubic_map(k)
        d = tab[k - 1]
        for lo, hi in _pieces(*interval_bounds(k)):
            half, mid = 0.5 * (hi - lo), 0.5 * (hi + lo)
            v = mid + half * _GL_X
            s = A * v - B
            g = d[0] + s * (d[1] + s * (d[2] + s * d[3]))
            total += (half * _GL_W * (ndtri(v) - g) ** 2).sum()
    return 2.0 * total
