"""FP64 reference of the learned capacity predictor's network.  TEST
INFRASTRUCTURE ONLY: used to check the CUDA forward / backward kernels.

Network (same parameter layout as include/sqs.h): x (F) -> tanh(W1 x + b1)
(H) -> tanh(W2 a1 + b2) (H) -> w3 . a2 + b3.  Loss: mean squared error.
The gradient is the chain rule written out layer by layer; the tests pin it
against central finite differences of the forward pass.
"""
from __future__ import annotations

import numpy as np

F, H = 16, 32
N_PARAMS = H * F + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, np.float64)
    i = 0
    W1 = p[i:i + H * F].reshape(H, F); i += H * F
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    w3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    a1 = np.tanh(X @ W1.T + b1)
    a2 = np.tanh(a1 @ W2.T + b2)
    return a2 @ w3 + b3, a1, a2


def loss(p, X, T):
    y, _, _ = forward(p, X)
    return float(np.mean((y - np.asarray(T, np.float64)) ** 2))


def gradient(p, X, T):
    """d loss / d p, same layout as p."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64)
    n = X.shape[0]
    y, a1, a2 = forward(p, X)
    dy = 2.0 * (y - np.asarray(T, np.float64)) / n           # (n,)
    g_w3 = a2.T @ dy
    g_b3 = dy.sum()
    d2 = (dy[:, None] * w3[None, :]) * (1.0 - a2 ** 2)       # (n, H)
    g_W2 = d2.T @ a1
    g_b2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - a1 ** 2)                         # (n, H)
    g_W1 = d1.T @ X
    g_b1 = d1.sum(0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
