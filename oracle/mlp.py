"""FP64 reference of the per-element correction network (the learned smoothing
sweep; the paper has none - it stands in for the paper's element-block Schwarz
smoother of Eq. Mass, which maps an element's residual to a local correction).

Network: y = W2 relu(W1 x + b1) + b2, x, y in R^Np, hidden width H.
Loss over a batch of B samples: L = (1/B) sum_b ||y_b - t_b||^2.
Gradients by the chain rule; Adam (Kingma & Ba 2015) with bias correction.

Arrays use the library's layout: W1 [H][Np], W2 [Np][H], samples row-major [B][Np].
"""
from __future__ import annotations

import numpy as np


def forward(W1, b1, W2, b2, X):
    """Returns (a1 [B,H] pre-activation, h1 [B,H], y [B,Np])."""
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    y = h1 @ W2.T + b2
    return a1, h1, y


def loss_and_grads(W1, b1, W2, b2, X, T):
    """Mean squared error over the batch and its gradients (dW1, db1, dW2, db2)."""
    B = X.shape[0]
    a1, h1, y = forward(W1, b1, W2, b2, X)
    diff = y - T
    loss = float(np.sum(diff * diff) / B)
    dy = 2.0 * diff / B
    dW2 = dy.T @ h1
    db2 = dy.sum(axis=0)
    dh1 = dy @ W2
    da1 = dh1 * (a1 > 0.0)
    dW1 = da1.T @ X
    db1 = da1.sum(axis=0)
    return loss, (dW1, db1, dW2, db2)


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of every array in place."""
    for p, g, mi, vi in zip(params, grads, m, v):
        mi *= beta1
        mi += (1.0 - beta1) * g
        vi *= beta2
        vi += (1.0 - beta2) * g * g
        mhat = mi / (1.0 - beta1 ** t)
        vhat = vi / (1.0 - beta2 ** t)
        p -= lr * mhat / (np.sqrt(vhat) + eps)


def bf16_round(a):
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)
