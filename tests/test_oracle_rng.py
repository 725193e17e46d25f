"""Pins of the oracle's random-number layer: Philox4x32-10 and the uniform map."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(x, 16) for x in line.split()])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_philox_known_answers():
    kat = _kat()
    for row in kat:
        out = O.philox4x32_10(row[:4].reshape(1, 4), row[4:6])
        assert out[0].tolist() == row[6:10].tolist()


def test_philox_is_a_bijection_sample():
    # distinct counters give distinct outputs on a sample (no collisions among 2^16)
    ctr = O.counters(np.arange(1 << 16), 0, 0)
    out = O.philox4x32_10(ctr, O.seed_key(1234))
    packed = out[:, 0].astype(np.uint64) << np.uint64(32) | out[:, 1].astype(np.uint64)
    assert np.unique(packed).size == packed.size


def test_philox_word_statistics():
    # chi^2 on the top 8 bits of 2^20 words: uniform at the 1e-4 level
    ctr = O.counters(np.arange(1 << 18), 3, O.make_tag(O.KIND_FOUR, 5))
    w = O.philox4x32_10(ctr, O.seed_key(1234)).ravel()
    counts = np.bincount((w >> 24).astype(np.int64), minlength=256)
    expected = w.size / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert 150 < chi2 < 380  # 255 dof: mean 255, sd 22.6


def test_uniform_grid_closed_form():
    w = np.array([0, 1 << 9, 0xFFFFFFFF, 0x80000000, 0x7FFFFFFF], dtype=np.uint32)
    u = O.uniforms(w)
    expect = [(2 * (int(x) >> 9) + 1) / 2.0 ** 24 for x in w]
    assert u.tolist() == expect
    assert u.min() == 2.0 ** -24 and u.max() == 1 - 2.0 ** -24


def test_uniform_symmetry_and_exactness():
    rng = np.random.default_rng(5)
    w = rng.integers(0, 2 ** 32, size=100000, dtype=np.uint64).astype(np.uint32)
    u = O.uniforms(w)
    u_flip = O.uniforms(~w)
    assert np.all(u + u_flip == 1.0)                     # mirrored grid
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in binary32
    assert np.all((u > 0) & (u < 1))
