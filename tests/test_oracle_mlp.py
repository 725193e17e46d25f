"""Pins of the oracle's MLP surrogate (FP64 forward / backward / Adam)."""
import numpy as np

import oracle as O
from oracle import mlp


def _rand_weights(seed=0, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp.N_PARAMS) * scale


def test_layout_pinned_by_hand_built_network():
    # W1 = e0, W2[3][0] = 1, W3 = e3  =>  y = tanh(tanh(t)); a transposed W2 gives 0
    w = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(w.copy())
    W1 = np.zeros(32); W1[0] = 1.0
    W2 = np.zeros((32, 32)); W2[3, 0] = 1.0
    W3 = np.zeros(32); W3[3] = 1.0
    w = mlp.pack(W1, np.zeros(32), W2, np.zeros(32), W3, np.array([0.25]))
    t = np.array([0.5, 1.5, 3.0])
    y, _ = mlp.forward(w, t)
    assert np.allclose(y, np.tanh(np.tanh(t)) + 0.25, rtol=0, atol=1e-15)
    # the C oracle evaluates the same layout
    u = np.array([0.3, 0.7, 1e-4])
    z = O.approx_icdf(u, O.RV_MLP, mlp=w)
    yy = np.tanh(np.tanh(mlp.features(u))) + 0.25
    assert np.allclose(z, np.where(u > 0.5, yy, -yy), rtol=0, atol=1e-15)


def test_c_and_numpy_forward_agree():
    w = _rand_weights(1)
    u = np.random.default_rng(2).uniform(1e-7, 1 - 1e-7, 1000)
    assert np.allclose(O.approx_icdf(u, O.RV_MLP, mlp=w), mlp.icdf(w, u), rtol=1e-13, atol=1e-13)


def test_gradient_matches_finite_differences():
    w = _rand_weights(3)
    rng = np.random.default_rng(4)
    t = mlp.features(rng.uniform(1e-6, 0.5, 64))
    target = rng.standard_normal(64)
    _, g = mlp.loss_and_grad(w, t, target)
    h = 1e-6
    idx = np.concatenate([np.arange(0, 64, 7), 64 + np.arange(0, 1024, 53), np.arange(1088, 1153, 5)])
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h; wm[i] -= h
        fd = (mlp.loss_and_grad(wp, t, target)[0] - mlp.loss_and_grad(wm, t, target)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_reduces_to_signed_step():
    # beta1 = beta2 = 0: the update is lr * g / (|g| + eps) = lr * sign(g) for |g| >> eps
    w = np.zeros(5)
    g = np.array([0.3, -2.0, 1e-3, -5e-2, 7.0])
    w2, m, v = mlp.adam_step(w, g, np.zeros(5), np.zeros(5), 1, 0.01, beta1=0.0, beta2=0.0, eps=1e-12)
    assert np.allclose(w2, -0.01 * np.sign(g), rtol=1e-9)


def test_training_fits_inverse_cdf():
    # a few hundred Adam steps reach a loss well below the initial one
    rng = np.random.default_rng(7)
    w = _rand_weights(8, scale=0.2)
    m = np.zeros_like(w); v = np.zeros_like(w)
    u = rng.uniform(2.0 ** -24, 0.5, 4096)
    t, target = mlp.features(u), -O.ndtri(u)
    first = mlp.loss_and_grad(w, t, target)[0]
    for s in range(1, 301):
        loss, g = mlp.loss_and_grad(w, t, target)
        w, m, v = mlp.adam_step(w, g, m, v, s, mlp.cosine_lr(s, 300, 1e-2, 1e-3))
    assert loss < 0.02 * first
