"""FP64 oracle of the paper's efficiency experiment (Sec. 5, "Algorithm
efficiency"): NNLS(B, y) for a dense B by Algorithm 1 with full-row updates.

TEST INFRASTRUCTURE ONLY: used by the tests and the benchmark's CPU leg, never
by the library.  Each column of Y is an independent problem:
    r = B x - y;  g = B^T r  (Algorithm 1 as printed, no factor 2);
    G += g^2;  x = max(x - eta g / (sqrt(G) + eps), 0)   (Adagrad, projection).
"""
from __future__ import annotations

import numpy as np


def spgd_dense(B, Y, iters: int, step: float, eps: float = 1e-10, X0=None, G0=None):
    """Returns (X [n_cols][m], G, loss [m]) after `iters` full-row updates."""
    B = np.asarray(B, np.float64)
    Y = np.asarray(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    m = Y.shape[1]
    X = np.zeros((B.shape[1], m)) if X0 is None else np.array(X0, np.float64)
    G = np.zeros_like(X) if G0 is None else np.array(G0, np.float64)
    for _ in range(iters):
        R = B @ X - Y
        g = B.T @ R
        G += g * g
        X = np.maximum(X - step * g / (np.sqrt(G) + eps), 0.0)
    loss = ((B @ X - Y) ** 2).sum(axis=0)
    return X, G, loss


def tf32(a):
    """FP32 values as the tensor cores' TF32 operands read them: the 13 low
    mantissa bits dropped (1 sign, 8 exponent, 10 mantissa bits kept)."""
    a = np.asarray(a, np.float32)
    return (a.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def spgd_dense_tf32(B, Y, iters: int, step: float, eps: float = 1e-10):
    """Algorithm 1 as ``spgd_dense`` with each product's operands taken as TF32
    values (B, the iterate X and the residual R cut to TF32 before the
    product; products and sums in FP64): the arithmetic definition of the
    tensor-core form, whose accumulation is FP32."""
    B = np.asarray(B, np.float32)
    Y = np.asarray(Y, np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    Bt = tf32(B).astype(np.float64)
    m = Y.shape[1]
    X = np.zeros((B.shape[1], m), np.float32)
    G = np.zeros((B.shape[1], m), np.float32)
    for _ in range(iters):
        R = (Bt @ tf32(X).astype(np.float64) - Y).astype(np.float32)
        g = (Bt.T @ tf32(R).astype(np.float64)).astype(np.float32)
        G = (G + g * g).astype(np.float32)
        X = np.maximum(X - np.float32(step) * g / (np.sqrt(G) + np.float32(eps)), 0.0).astype(np.float32)
    R = Bt @ tf32(X).astype(np.float64) - Y
    return X, G, (R ** 2).sum(axis=0)
