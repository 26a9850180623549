"""Stopping/lambda network: forward, backward, Adam (oracle, FP64).

Not in the paper.  Architecture: x (20) -> 128 -> 128 -> 2, GELU after the two
hidden layers, linear output.  GELU(x) = x Phi(x) with the exact normal CDF
Phi(x) = (1 + erf(x / sqrt 2)) / 2 (Hendrycks & Gimpel 2016).  Loss: mean
squared error L = sum_{b,o} (y_bo - t_bo)^2 / (2 B).  Adam (Kingma & Ba 2015):
m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, theta <- theta - lr mhat /
(sqrt(vhat) + eps) with mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).

Parameters are one flat vector: W1 (20 x 128, row-major), b1 (128),
W2 (128 x 128), b2 (128), W3 (128 x 2), b3 (2) -- 19458 values.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

N_IN, N_HID, N_OUT = 20, 128, 2
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, off = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = theta[off:off + size].reshape(shape)
        off += size
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, X):
    p = unpack(np.asarray(theta, dtype=np.float64))
    z1 = X @ p["W1"] + p["b1"]
    h1 = gelu(z1)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = gelu(z2)
    y = h2 @ p["W3"] + p["b3"]
    return y, (X, z1, h1, z2, h2)


def loss_and_grad(theta, X, T):
    """L = sum (y - t)^2 / (2B) and dL/dtheta (flat, same layout as theta)."""
    X = np.asarray(X, dtype=np.float64)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    B = X.shape[0]
    p = unpack(np.asarray(theta, dtype=np.float64))
    dy = (y - T) / B
    L = float(np.sum((y - T) ** 2) / (2 * B))
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"].T) * gelu_grad(z2)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * gelu_grad(z1)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return L, np.concatenate([g[name].ravel() for name, _ in SHAPES])


def adam_step(theta, m, v, g, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed=0):
    """Glorot-uniform weights, zero biases (the initial vector is an input to both sides)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for name, shape in SHAPES:
        if name.startswith("W"):
            lim = math.sqrt(6.0 / (shape[0] + shape[1]))
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts)
