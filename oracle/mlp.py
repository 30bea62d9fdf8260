"""FP64 reference of the parameter-proposer network (TEST INFRASTRUCTURE ONLY:
only tests/ may import this module).

The network is the one of the C ABI's sog_mlp_*: x -> tanh(W1 x + b1) ->
tanh(W2 h1 + b2) -> y = w3 . h2 + b3, parameters in one flat array
W1 [H][n_in], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]; loss
(1/n) sum (y - t)^2.  Written out plainly with NumPy (matrix products only)
and shared with nothing in the CUDA library.
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, H):
    p = np.asarray(p, dtype=np.float64)
    k = 0
    W1 = p[k:k + H * n_in].reshape(H, n_in); k += H * n_in
    b1 = p[k:k + H]; k += H
    W2 = p[k:k + H * H].reshape(H, H); k += H * H
    b2 = p[k:k + H]; k += H
    w3 = p[k:k + H]; k += H
    b3 = p[k]; k += 1
    assert k == p.size
    return W1, b1, W2, b2, w3, b3


def forward(p, X, n_in, H):
    """Outputs y for the rows of X, and the activations h1, h2."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, h1, h2


def loss_grad(p, X, T, n_in, H):
    """Mean squared error and its gradient by the chain rule, layer by layer."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    y, h1, h2 = forward(p, X, n_in, H)
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n                       # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, g
