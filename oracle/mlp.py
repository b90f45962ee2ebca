"""Plain CPU reference for the batch-split cost model (test infrastructure
only: tests/ and nothing in the product path import it).

The model is a one-hidden-layer ReLU network on standardised inputs,
    z = xs W1 + b1,  h = max(z, 0),  y = h w2 + b2,
with the mean squared error L = mean((y - t)^2).  Weights use the packed
layout of the library's cost model: mu[D], sigma[D], W1[D][H] (row-major),
b1[H], w2[H], b2.  Everything is computed in float64, one definition per
line, so it can be read against the formulas above.
"""
from __future__ import annotations

import numpy as np

NFEAT = 13
D = NFEAT + 1


def unpack(w: np.ndarray, hidden: int):
    w = np.asarray(w, dtype=np.float64)
    mu, sd = w[:D], w[D:2 * D]
    o = 2 * D
    W1 = w[o:o + D * hidden].reshape(D, hidden)
    o += D * hidden
    b1 = w[o:o + hidden]
    o += hidden
    w2 = w[o:o + hidden]
    b2 = w[o + hidden]
    return mu, sd, W1, b1, w2, b2


def forward(x: np.ndarray, w: np.ndarray, hidden: int) -> np.ndarray:
    mu, sd, W1, b1, w2, b2 = unpack(w, hidden)
    xs = (np.asarray(x, np.float64) - mu) / sd
    z = xs @ W1 + b1
    h = np.maximum(z, 0.0)
    return h @ w2 + b2


def loss(x, t, w, hidden) -> float:
    y = forward(x, w, hidden)
    return float(np.mean((y - np.asarray(t, np.float64)) ** 2))


def grad(x: np.ndarray, t: np.ndarray, w: np.ndarray, hidden: int) -> tuple[np.ndarray, float]:
    """Analytic gradient of the loss in the packed layout (zero for mu and
    sigma, which are not trained), and the loss."""
    mu, sd, W1, b1, w2, b2 = unpack(w, hidden)
    xs = (np.asarray(x, np.float64) - mu) / sd
    n = xs.shape[0]
    z = xs @ W1 + b1
    h = np.maximum(z, 0.0)
    y = h @ w2 + b2
    r = y - np.asarray(t, np.float64)
    dy = 2.0 * r / n                     # dL/dy
    g_w2 = h.T @ dy                      # dL/dw2
    g_b2 = dy.sum()                      # dL/db2
    dz = np.outer(dy, w2) * (z > 0)      # dL/dz
    g_W1 = xs.T @ dz                     # dL/dW1
    g_b1 = dz.sum(axis=0)                # dL/db1
    g = np.zeros(2 * D + D * hidden + 2 * hidden + 1)
    o = 2 * D
    g[o:o + D * hidden] = g_W1.ravel()
    o += D * hidden
    g[o:o + hidden] = g_b1
    o += hidden
    g[o:o + hidden] = g_w2
    g[o + hidden] = g_b2
    return g, float(np.mean(r ** 2))
