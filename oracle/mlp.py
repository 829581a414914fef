"""Float64 forward and backward pass of the step-cost MLP (oracle, test
infrastructure only).

Not part of the paper's method: the workload adds a learned model that ranks
contraction trees.  Its GPU gradients are checked against this plain numpy
version, which is itself pinned by central finite differences and a
hand-computed one-sample case (tests/test_oracle_mlp.py).

Architecture: x (16) -> relu(W1 x + b1) (64) -> relu(W2 h1 + b2) (64) ->
w3 . h2 + b3; loss = mean over samples of (y - t)^2.  Flat parameter layout:
W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3.
"""
from __future__ import annotations

import numpy as np

F, H1, H2 = 16, 64, 64
N_PARAMS = H1 * F + H1 + H2 * H1 + H2 + H2 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H1 * F].reshape(H1, F); o += H1 * F
    b1 = p[o:o + H1]; o += H1
    W2 = p[o:o + H2 * H1].reshape(H2, H1); o += H2 * H1
    b2 = p[o:o + H2]; o += H2
    w3 = p[o:o + H2]; o += H2
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(p, X, T):
    y = forward(p, X)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def grad(p, X, T):
    """(loss, gradient) by the chain rule, in the flat parameter layout."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    d = y - T
    L = float(np.mean(d ** 2))
    dy = 2.0 * d / n
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dh2 = np.outer(dy, w3) * (a2 > 0)
    g_W2 = dh2.T @ h1
    g_b2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    g_W1 = dh1.T @ X
    g_b1 = dh1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return L, g
