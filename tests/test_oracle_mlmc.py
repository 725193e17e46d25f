"""Pins of the oracle's MLMC cost model and allocation (Sec. 3)."""
import math

import numpy as np

from oracle import mlmc


def test_optimal_samples_meet_variance_target_and_minimise_cost():
    V = np.array([0.04, 4e-4, 2e-4, 1e-4, 5e-5])
    C = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    eps = 1e-3
    N = mlmc.optimal_samples(V, C, eps)
    assert np.sum(V / N) <= eps ** 2 / 2 * (1 + 1e-9)
    # Lagrange optimum: perturbing the split at fixed variance raises the cost
    cost = np.sum(N * C)
    for i in range(len(V)):
        for j in range(len(V)):
            if i == j:
                continue
            Np = N.astype(float).copy()
            Np[i] *= 1.05
            # keep sum V/N fixed by adjusting level j
            rem = eps ** 2 / 2 - np.sum(np.delete(V / Np, j))
            if rem <= 0:
                continue
            Np[j] = V[j] / rem
            assert np.sum(Np * C) >= cost * (1 - 1e-6)
    # total cost matches T = 2 eps^-2 (sum sqrt(VC))^2 up to ceil rounding
    assert abs(cost / mlmc.predicted_cost(V, C, eps) - 1) < 1e-3


def test_nested_cost_bound():
    # T- <= T^ max_l { v-c-/(v^c^) (1 + sqrt(V-C-/(v-c-)))^2 } (Sec. 3)
    rng = np.random.default_rng(0)
    for _ in range(50):
        vh, ch = rng.uniform(0.1, 1, 6), rng.uniform(0.1, 1, 6)
        vb, cb = vh * rng.uniform(0.9, 1.1, 6), ch * rng.uniform(0.05, 0.3, 6)
        Vb, Cb = vh * rng.uniform(1e-4, 1e-2, 6), ch * rng.uniform(1.0, 1.3, 6)
        t_hat = mlmc.predicted_cost(vh, ch, 1e-3)
        t_bar = 2e6 * (np.sum(np.sqrt(vb * cb) + np.sqrt(Vb * Cb))) ** 2
        bound = t_hat * np.max(vb * cb / (vh * ch) * (1 + np.sqrt(Vb * Cb / (vb * cb))) ** 2)
        assert t_bar <= bound * (1 + 1e-12)


def test_weak_convergence_rule():
    eps = 1e-3
    # level means halving from 1e-2: converged once |Y_L| <= eps / sqrt(2) (alpha = 1)
    Y = [0.1, 1e-2, 5e-3, 2.5e-3, 1.25e-3, 6.25e-4]
    done = [mlmc.weak_converged(Y[:k], eps) for k in range(1, len(Y) + 1)]
    assert done == [False, False, False, False, False, True]


def test_black_scholes_reference_values():
    assert abs(mlmc.bs_call() - 0.1045058357) < 1e-9
    assert abs(mlmc.bs_call(discounted=False) - 0.1098639645) < 1e-9
