"""Pins of the oracle's binary16 inference arithmetic of the MLP surrogate
(the learned part): the binary32 input map against the FP64 library value,
the activation against high-precision tanh at every binary16 input, a
hand-built network against exact fused multiply-adds in index order, and
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


def _round16(y):
    """The binary16 number nearest to the high-precision value y (no tie can
    occur for a transcendental value)."""
    import mpmath
    f = np.float16(float(y))
    cands = [f, np.nextafter(f, np.float16(-np.inf)), np.nextafter(f, np.float16(np.inf))]
    return min(cands, key=lambda c: abs(mpmath.mpf(float(c)) - y))


def test_tanh16_is_correctly_rounded_at_every_binary16_input():
    """tanh16 of every finite binary16 x >= 0 equals tanh(x) from 40-digit
    arithmetic rounded to the nearest binary16; odd symmetry for x < 0;
    inputs are rounded to binary16 first, and beyond the binary16 range go
    to +-1."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    bits = np.arange(0x7C00, dtype=np.uint16)
    x = bits.view(np.float16).astype(np.float64)
    got = O.tanh16(x)
    want = np.array([float(_round16(mpmath.tanh(mpmath.mpf(a)))) for a in x])
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (x[bad[:5]], got[bad[:5]], want[bad[:5]])
    assert np.array_equal(O.tanh16(-x), -got)
    assert np.all(np.signbit(O.tanh16(-x[:1])))          # tanh16(-0) = -0
    # a binary32 pre-activation is rounded to binary16 first: on [0.3, 1)
    # (tanh' ~ 0.6..0.9) that moves the result for some inputs
    a = np.linspace(0.3, 1.0, 257, endpoint=False).astype(np.float32).astype(np.float64)
    got = O.tanh16(a)
    first = np.array([float(_round16(mpmath.tanh(mpmath.mpf(float(np.float16(x)))))) for x in a])
    direct = np.array([float(_round16(mpmath.tanh(mpmath.mpf(float(x))))) for x in a])
    assert np.array_equal(got, first) and np.any(got != direct)
    assert list(O.tanh16([7e4, -1e9])) == [1.0, -1.0]


def test_hand_built_network_matches_fma_chain_in_index_order():
    """Three hidden units feed output unit 3 from one 16-wide half of the
    inputs (0, 5) and one from the other (17); unit 9 reads unit 0, unit 20
    reads unit 17 (an asymmetric W2, so a transposed index is seen).  Each
    step is redone with an exact fused multiply-add rounded once to binary32
    and the binary16 activation, in index order.  The output sum mixes a
    large term (unit 3) with small ones carrying low-order bits (units 9,
    20), so the same steps in another order give another y for some inputs
    (inside layer 2 an order change moves c by an ulp of binary32, which the
    rounding of c to binary16 mostly hides)."""
    H = 32
    W1 = np.zeros(H); b1 = np.zeros(H); W2 = np.zeros((H, H)); b2 = np.zeros(H); W3 = np.zeros(H)
    W1[0], b1[0] = 0.013, 0.002              # small activations with fine low-order bits
    W1[5], b1[5] = 1.71, -2.3
    W1[17], b1[17] = -0.023, 0.11
    W2[3, 0], W2[3, 5], W2[3, 17] = 0.7, 1.9, -1.3
    W2[9, 0] = 0.45
    W2[20, 17] = 2.1
    b2[3], b2[9], b2[20] = 0.05, 0.001, -0.04
    W3[3], W3[9], W3[20] = 1.9, 1.3, -0.6
    b3 = 0.3
    w = _net(W1, b1, W2, b2, W3, b3).astype(np.float32).astype(np.float64)
    Wf = OM.unpack(w)
    f32 = np.float32

    def act(x):
        return np.float16(O.tanh16([float(x)])[0])

    def net(t, out_order):
        h1 = {j: act(_fma32(f32(Wf[0][j]), t, f32(Wf[1][j]))) for j in (0, 5, 17)}
        reads = {3: (0, 5, 17), 9: (0,), 20: (17,)}
        h2 = {}
        for o, ins in reads.items():
            c = f32(Wf[3][o])
            for j in ins:
                c = _fma32(np.float16(Wf[2][o, j]), h1[j], c)
            h2[o] = act(c)
        # units with zero weights carry tanh16(b2) = 0 and add nothing
        y = f32(b3)
        for o in out_order:
            y = _fma32(np.float16(Wf[4][o]), h2[o], y)
        return y

    differs = 0
    for u in np.concatenate([[0.013, 0.31, 0.5, 0.77, 1 - 2.0 ** -20], uniform_grid_sample(200, 4)]):
        v = min(u, 1.0 - u)
        t = f32(O.mlp_feature32(np.array([v]))[0])
        y = net(t, (3, 9, 20))
        z = O.approx_icdf(np.array([u]), O.RV_MLP16, mlp=w)[0]
        assert z == (float(y) if u > 0.5 else -float(y)), (u, z, y)
        differs += int(net(t, (20, 9, 3)) != y)
    assert differs > 0


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
