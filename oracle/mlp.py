"""MLP surrogate for the inverse Gaussian CDF, FP64 forward / backward / Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The network approximates |Phi^-1(v)| for v = min(u, 1-u) in (0, 1/2] from
t = sqrt(-2 ln v): y = W3 tanh(W2 tanh(W1 t + b1) + b2) + b3, 1 -> 32 -> 32
-> 1, 1153 parameters; the approximate normal is -y for u <= 1/2 and +y
above, so that it is antisymmetric like the piecewise-linear table
(Sec. 2.1 requires zero-mean approximate variables).  Training minimises
the mean of (y - |Phi^-1(v)|)^2, i.e. E|Z - Z~|^2, the quantity that sets
the four-way variance in Lemma 3.1.

Parameter layout (shared by every implementation, as data):
  W1[32], b1[32], W2[32][32] (row = output unit), b2[32], W3[32], b3[1].
"""
from __future__ import annotations

import numpy as np

H = 32
N_PARAMS = H + H + H * H + H + H + 1  # 1153


def unpack(w: np.ndarray):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H]; o += H
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + H]; o += H
    b3 = w[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2), np.ravel(W3), np.ravel(b3)])


def features(u: np.ndarray) -> np.ndarray:
    """t = sqrt(-2 ln v), v = min(u, 1-u)."""
    u = np.asarray(u, dtype=np.float64)
    v = np.minimum(u, 1.0 - u)
    return np.sqrt(-2.0 * np.log(v))


def forward(w: np.ndarray, t: np.ndarray):
    """Returns y (n,) and the activations needed by backward()."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    t = np.asarray(t, dtype=np.float64).reshape(-1)
    h1 = np.tanh(np.outer(t, W1) + b1)          # (n, 32)
    h2 = np.tanh(h1 @ W2.T + b2)                # (n, 32)
    y = h2 @ W3 + b3[0]                         # (n,)
    return y, (t, h1, h2)


def loss_and_grad(w: np.ndarray, t: np.ndarray, target: np.ndarray):
    """Mean squared error and its gradient with respect to all 1153 parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(w)
    y, (t, h1, h2) = forward(w, t)
    n = t.size
    r = y - np.asarray(target, dtype=np.float64).reshape(-1)
    loss = float(np.mean(r * r))
    gy = 2.0 * r / n                            # dL/dy
    gW3 = h2.T @ gy
    gb3 = np.array([gy.sum()])
    gh2 = np.outer(gy, W3)                      # (n, 32)
    ga2 = gh2 * (1.0 - h2 * h2)
    gW2 = ga2.T @ h1                            # (32 out, 32 in)
    gb2 = ga2.sum(axis=0)
    gh1 = ga2 @ W2
    ga1 = gh1 * (1.0 - h1 * h1)
    gW1 = ga1.T @ t
    gb1 = ga1.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2, gW3, gb3)


def adam_step(w, g, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    w = w - lr * mhat / (np.sqrt(vhat) + eps)
    return w, m, v


def cosine_lr(step: int, total: int, lr0: float, lr_min: float) -> float:
    """Cosine decay from lr0 to lr_min over total steps (step counts from 1)."""
    frac = min(max((step - 1) / max(total - 1, 1), 0.0), 1.0)
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + np.cos(np.pi * frac))


def icdf(w: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Antisymmetric approximate normal from the network."""
    u = np.asarray(u, dtype=np.float64)
    y, _ = forward(w, features(u))
    return np.where(u > 0.5, y, -y)
