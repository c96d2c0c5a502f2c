"""FP64 CPU oracle of the PP-regime policy network (8 -> 64 -> 64 -> 1).

TEST INFRASTRUCTURE ONLY (see oracle/cp_oracle.py).  The paper's PP regime is
governed by a hand-set tolerance (Alg. 2: enter/stay while every
||dA(i)||_F < eps ||A(i)||_F).  The library can replace that rule by a small
learned scorer; the paper has no counterpart, so this file is pinned only by
mathematics: finite-difference gradients, and the closed forms of the logistic
loss.

Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), z = w3 . h2 + b3,
p = sigmoid(z); loss = mean over the batch of binary cross-entropy
-(y log p + (1 - y) log(1 - p)), written in the overflow-safe form
softplus(z) - y z.  Parameters are stored as one flat vector in the order
W1 (64x8 row-major), b1 (64), W2 (64x64), b2 (64), w3 (64), b3 (1): 4801 values.
Optimiser: Adam (Kingma and Ba, ICLR 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

D_IN, H1, H2 = 8, 64, 64
SHAPES = [("W1", (H1, D_IN)), ("b1", (H1,)), ("W2", (H2, H1)), ("b2", (H2,)),
          ("w3", (H2,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def init_params(u):
    """Parameters from uniforms u in [0,1) (N_PARAMS of them): U(-1/sqrt(fan_in), +) weights, zero biases."""
    theta = np.zeros(N_PARAMS)
    o = 0
    fan = {"W1": D_IN, "W2": H1, "w3": H2}
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        if name in fan:
            theta[o:o + n] = (2.0 * u[o:o + n] - 1.0) / np.sqrt(fan[name])
        o += n
    return theta


def forward(theta, X):
    """Returns (z, cache) for a batch X (B x 8)."""
    P = unpack(theta)
    a1 = X @ P["W1"].T + P["b1"]
    h1 = np.tanh(a1)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.tanh(a2)
    z = h2 @ P["w3"] + P["b3"][0]
    return z, (X, h1, h2)


def predict(theta, X):
    z, _ = forward(theta, X)
    return 1.0 / (1.0 + np.exp(-z))


def loss(theta, X, y):
    z, _ = forward(theta, X)
    sp = np.logaddexp(0.0, z)            # softplus(z) = log(1 + e^z)
    return float(np.mean(sp - y * z))


def grad(theta, X, y):
    """Back-propagation of the mean BCE loss; returns (loss, flat gradient)."""
    P = unpack(theta)
    z, (Xb, h1, h2) = forward(theta, X)
    B = X.shape[0]
    p = 1.0 / (1.0 + np.exp(-z))
    dz = (p - y) / B                                 # d loss / d z
    g = {}
    g["w3"] = h2.T @ dz
    g["b3"] = np.array([dz.sum()])
    da2 = np.outer(dz, P["w3"]) * (1.0 - h2 * h2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    da1 = (da2 @ P["W2"]) * (1.0 - h1 * h1)
    g["W1"] = da1.T @ Xb
    g["b1"] = da1.sum(0)
    flat = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    sp = np.logaddexp(0.0, z)
    return float(np.mean(sp - y * z)), flat


def adam_step(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t is the 1-based step); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
