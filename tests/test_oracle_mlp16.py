"""Pins of the oracle's binary16 inference arithmetic of the MLP surrogate
(the learned part): the binary32 input map against the FP64 library value,
a hand-built network against numpy's IEEE float16 / float32 roundings, and
the whole network against the FP64 network within the binary16 error."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as OM
from workloads import mlp_initial_weights, uniform_grid_sample


def test_feature_is_sqrt_minus_two_log_to_binary32():
    u = uniform_grid_sample(20000, 3)
    v = np.concatenate([np.minimum(u, 1 - u), [0.5, 2.0 ** -24, 2.0 ** -10, 0.25 + 2.0 ** -24]])
    t = O.mlp_feature32(v)
    ref = np.sqrt(-2.0 * np.log(v))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(t - ref) / ulp) <= 2.0
    assert np.all(t == t.astype(np.float32))
    # v = 2^-k: m = 1, ln m = 0 and t = R32(sqrt(R32(2 k R32(ln 2)))) by IEEE binary32 arithmetic
    for k in range(1, 25):
        ln2 = np.float32(math.log(2.0))
        t2 = np.float32(np.float32(2 * k) * ln2)
        assert O.mlp_feature32(np.array([2.0 ** -k]))[0] == float(np.sqrt(t2)), k


def _fma32(a, b, c):
    """a b + c rounded once to binary32 (nearest even), from the exact value."""
    from fractions import Fraction
    x = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    f = np.float32(float(x))                 # within one binary32 ulp of x
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = min(cands, key=lambda y: (abs(Fraction(float(y)) - x), int(np.float32(y).view(np.uint32)) & 1))
    return np.float32(best)


def _net(W1, b1, W2, b2, W3, b3):
    return OM.pack(np.asarray(W1, float), np.asarray(b1, float), np.asarray(W2, float), np.asarray(b2, float),
                   np.asarray(W3, float), np.asarray([b3], float))


def test_hand_built_network_matches_ieee_float16_steps():
    """Two active hidden units per layer with an asymmetric W2, so that a
    transposed index or a missed rounding point changes the result; each
    step is redone with numpy float16 / float32 casts (IEEE round to
    nearest even)."""
    H = 32
    W1 = np.zeros(H); b1 = np.zeros(H); W2 = np.zeros((H, H)); b2 = np.zeros(H); W3 = np.zeros(H)
    W1[0], b1[0] = 0.37, -0.81
    W1[17], b1[17] = -0.23, 1.1
    W2[3, 0], W2[3, 17] = 0.7, -1.3          # unit 3 reads units 0 and 17 (second k-chunk)
    W2[20, 17] = 2.1                         # unit 20 reads unit 17 only
    b2[3], b2[20] = 0.05, -0.4
    W3[3], W3[20] = 1.9, -0.6
    b3 = 0.3
    w = _net(W1, b1, W2, b2, W3, b3).astype(np.float32).astype(np.float64)
    Wf = OM.unpack(w)
    for u in (0.013, 0.31, 0.5, 0.77, 1 - 2.0 ** -20):
        v = min(u, 1.0 - u)
        t = np.float32(O.mlp_feature32(np.array([v]))[0])

        def act(x):
            return np.float16(np.tanh(np.float64(np.float16(x))))
        h1 = {j: act(_fma32(np.float32(Wf[0][j]), t, np.float32(Wf[1][j]))) for j in (0, 17)}
        w2 = {(o, j): np.float16(Wf[2][o, j]) for o, j in ((3, 0), (3, 17), (20, 17))}
        c3 = np.float32(np.float64(np.float32(Wf[3][3])) + np.float64(w2[3, 0]) * np.float64(h1[0]))
        c3 = np.float32(np.float64(c3) + np.float64(w2[3, 17]) * np.float64(h1[17]))
        c20 = np.float32(np.float64(np.float32(Wf[3][20])))
        c20 = np.float32(np.float64(c20) + np.float64(w2[20, 17]) * np.float64(h1[17]))
        h2_3, h2_20 = act(c3), act(c20)
        # units with zero weights still carry tanh(b2) = 0 and contribute nothing
        y = np.float32(np.float64(np.float32(b3)) + np.float64(np.float16(Wf[4][3])) * np.float64(h2_3))
        y = np.float32(np.float64(y) + np.float64(np.float16(Wf[4][20])) * np.float64(h2_20))
        z = O.approx_icdf(np.array([u]), O.RV_MLP16, mlp=w)[0]
        assert z == (float(y) if u > 0.5 else -float(y)), (u, z, y)


def test_binary16_network_tracks_the_fp64_network():
    """With binary16 activations (relative rounding 2^-11) and weights the
    output stays within a few 1e-3 of the FP64 network: each of the 64
    activations carries at most half an ulp, weighted by |W| <= ~2."""
    w = mlp_initial_weights(1234).astype(np.float32).astype(np.float64)
    u = uniform_grid_sample(50000, 9)
    z64 = O.approx_icdf(u, O.RV_MLP, mlp=w)
    z16 = O.approx_icdf(u, O.RV_MLP16, mlp=w)
    assert not np.any(np.isnan(z16))
    d = np.abs(z16 - z64)
    assert d.max() < 4e-3 and d.mean() < 5e-4
    # antisymmetry is exact (the sign is applied after the network)
    z_lo = O.approx_icdf(u[u < 0.5], O.RV_MLP16, mlp=w)
    z_hi = O.approx_icdf(1.0 - u[u < 0.5], O.RV_MLP16, mlp=w)
    assert np.array_equal(z_lo, -z_hi)
