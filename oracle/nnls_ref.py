"""Exact NNLS on tiny instances -- TEST INFRASTRUCTURE ONLY.

``min ||x - B q||^2 s.t. q >= 0`` (Eq. (nnls), Sec. 3) solved by enumerating
supports: for each subset S of columns the unconstrained least-squares problem
on S is solved; the minimiser is the feasible (all positive on S) candidate of
smallest loss.  Exponential in the number of unknowns, so only for <= ~14.
The KKT check states optimality without reference to any solver.
"""
from __future__ import annotations

import itertools

import numpy as np


def nnls_bruteforce(B: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The minimiser of Eq. (nnls) by enumerating supports (module docstring)."""
    n = B.shape[1]
    assert n <= 16, "support enumeration is exponential"
    best, best_loss = np.zeros(n), float(x @ x)
    for size in range(1, n + 1):
        for S in itertools.combinations(range(n), size):
            cols = list(S)
            sol, *_ = np.linalg.lstsq(B[:, cols], x, rcond=None)
            if np.any(sol <= 0):
                continue
            q = np.zeros(n)
            q[cols] = sol
            r = B @ q - x
            loss = float(r @ r)
            if loss < best_loss - 1e-14 * max(1.0, best_loss):
                best, best_loss = q, loss
    return best


def kkt_violation(B: np.ndarray, x: np.ndarray, q: np.ndarray) -> dict:
    """Scaled KKT residuals of NNLS at q: gradient g = B^T (B q - x).

    * dual feasibility:  g_i >= 0 wherever q_i = 0
    * stationarity:      g_i = 0 wherever q_i > 0
    * complementarity:   q_i g_i = 0
    """
    g = B.T @ (B @ q - x)
    scale = max(1.0, float(np.abs(B.T @ x).max()))
    active = q <= 0
    return {
        "dual": float(np.maximum(-g[active], 0).max(initial=0.0)) / scale,
        "stationarity": float(np.abs(g[~active]).max(initial=0.0)) / scale,
        "complementarity": float(np.abs(q * g).max(initial=0.0)) / (scale * max(1.0, float(q.max()))),
        "projected_gradient": float(np.abs(q - np.maximum(q - g, 0)).max()) / scale,
    }
