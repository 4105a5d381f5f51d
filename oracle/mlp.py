"""The warm-start network's loss, gradient and optimiser step (oracle, FP64 numpy).

Test infrastructure only.  The network is the multilayer perceptron of the learned warm start:
h_0 = x, z_k = h_k W_k^t + b_k, h_{k+1} = GELU(z_k) for the hidden layers, y = z_L (linear output),
GELU(z) = z Phi(z) with Phi the standard normal distribution function (the exact, erf form).
The loss is the mean-squared error L = sum (y - t)^2 / (batch * n_out).

The gradient follows the chain rule layer by layer, written out plainly:
    dL/dz_L = 2 (y - t) / (batch * n_out)
    dL/dW_k = (dL/dz_k)^t h_k,   dL/db_k = sum over the batch of dL/dz_k
    dL/dh_k = dL/dz_k W_k,       dL/dz_{k-1} = dL/dh_k * GELU'(z_{k-1}),
    GELU'(z) = Phi(z) + z phi(z),  phi the standard normal density.
Adam (Kingma & Ba 2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parity: pinned by tests/test_oracle_pins.py (the gradient against central finite differences of
the loss; GELU' against a difference quotient of GELU; Adam against its first-step closed form
p -= lr g / (|g| + eps)).
"""
from __future__ import annotations

import math

import numpy as np

_SQRT2 = math.sqrt(2.0)


def _Phi(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / _SQRT2))


def _phi(z):
    return np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def gelu(z):
    return z * _Phi(z)


def gelu_prime(z):
    return _Phi(z) + z * _phi(z)


def forward(x, W, b):
    """Output y and the pre-activations z_k (FP64)."""
    h = np.asarray(x, dtype=np.float64)
    zs, hs = [], [h]
    for k, (w, bb) in enumerate(zip(W, b)):
        z = h @ np.asarray(w, np.float64).T + (0.0 if bb is None else np.asarray(bb, np.float64))
        zs.append(z)
        if k < len(W) - 1:
            h = gelu(z)
            hs.append(h)
        else:
            h = z
    return h, zs, hs


def loss_and_grad(x, t, W, b):
    """(L, [dL/dW_k], [dL/db_k]) of the mean-squared error."""
    y, zs, hs = forward(x, W, b)
    t = np.asarray(t, np.float64)
    L = float(np.sum((y - t) ** 2) / y.size)
    dz = 2.0 * (y - t) / y.size
    dW = [None] * len(W)
    db = [None] * len(W)
    for k in range(len(W) - 1, -1, -1):
        dW[k] = dz.T @ hs[k]
        db[k] = dz.sum(0)
        if k > 0:
            dh = dz @ np.asarray(W[k], np.float64)
            dz = dh * gelu_prime(zs[k - 1])
    return L, dW, db


def adam_step(p, g, m, v, lr, b1, b2, eps, t):
    """One Adam step; returns the new (p, m, v)."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
