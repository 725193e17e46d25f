"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  Parameter draws only -- nothing here computes any step of the
method.

batching_sets(): the batching workload -- 64 GBM parameter sets
(mu ~ U[-0.05, 0.10], sigma ~ U[0.1, 0.5], X0 = 1, T = 1, call strike
K ~ U[0.8, 1.2]) then 64 Ornstein-Uhlenbeck sets (theta ~ U[0.5, 4],
m ~ N(0, 1), s ~ U[0.1, 1], X0 = 1, T = 1, payoff X_T), drawn in that order
with numpy PCG64 seed 1234; every set runs levels 0..16 with
N_l = max(1, round(2^(22 - 1.5 l))) samples.
"""
from __future__ import annotations

import numpy as np

BATCH_SEED = 1234
BATCH_LEVELS = 17


def batch_level_samples(levels: int = BATCH_LEVELS, log2_n0: float = 22.0) -> list[int]:
    return [max(1, int(round(2.0 ** (log2_n0 - 1.5 * l)))) for l in range(levels)]


def batching_sets(n_gbm: int = 64, n_ou: int = 64, seed: int = BATCH_SEED) -> list[dict]:
    """Parameter sets as dicts: kind ('gbm' / 'ou') and the raw parameters."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mu = rng.uniform(-0.05, 0.10, n_gbm)
    sigma = rng.uniform(0.1, 0.5, n_gbm)
    K = rng.uniform(0.8, 1.2, n_gbm)
    theta = rng.uniform(0.5, 4.0, n_ou)
    m = rng.normal(0.0, 1.0, n_ou)
    s = rng.uniform(0.1, 1.0, n_ou)
    sets = [dict(kind="gbm", mu=float(mu[i]), sigma=float(sigma[i]), K=float(K[i]), x0=1.0, T=1.0)
            for i in range(n_gbm)]
    sets += [dict(kind="ou", theta=float(theta[i]), m=float(m[i]), s=float(s[i]), x0=1.0, T=1.0)
             for i in range(n_ou)]
    return sets


def mlp_initial_weights(seed: int = 1234, hidden: int = 32) -> np.ndarray:
    """Xavier-uniform initial weights of the 1 -> 32 -> 32 -> 1 network in the
    1153-value layout (W1, b1, W2 [out][in], b2, W3, b3); biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a1 = np.sqrt(6.0 / (1 + hidden))
    a2 = np.sqrt(6.0 / (hidden + hidden))
    a3 = np.sqrt(6.0 / (hidden + 1))
    W1 = rng.uniform(-a1, a1, hidden)
    W2 = rng.uniform(-a2, a2, (hidden, hidden))
    W3 = rng.uniform(-a3, a3, hidden)
    return np.concatenate([W1, np.zeros(hidden), W2.ravel(), np.zeros(hidden), W3, np.zeros(1)])


def uniform_grid_sample(n: int, seed: int = 1234) -> np.ndarray:
    """n uniforms drawn from the 24-bit grid (2k + 1) 2^-24 (float64, exact in float32)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = rng.integers(0, 1 << 23, n)
    return (2.0 * k + 1.0) * 2.0 ** -24
