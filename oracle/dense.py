"""Exact MBD energy and gradient from a full eigendecomposition (FP64).

Eq. plasmonic: E = (1/2) sum_i sqrt(lambda_i) - (3/2) sum_i w_i over the 3N
eigenvalues of C; the O(N^3) route the stochastic method replaces, used here as
the reference for small systems.  Gradient: dE/dR = (1/4) Tr(C^{-1/2} dC/dR),
evaluated as sum over the 3N unit vectors e_v of (g . C^{-1/2} e_v)^T dT'/dR (g . e_v).
"""
from __future__ import annotations

import numpy as np

from .forces import bilinear_gradient


def dense_energy(c: np.ndarray, omega: np.ndarray) -> float:
    lam = np.linalg.eigvalsh(0.5 * (c + c.T))
    if np.any(lam <= 0.0):
        raise FloatingPointError("C is not positive definite")
    return float(0.5 * np.sum(np.sqrt(lam)) - 1.5 * np.sum(omega))


def inverse_sqrt(c: np.ndarray) -> np.ndarray:
    lam, u = np.linalg.eigh(0.5 * (c + c.T))
    return (u * lam ** -0.5) @ u.T


def dense_gradient(op, c: np.ndarray | None = None) -> np.ndarray:
    """dE/dR (N, 3) for the operator's mode."""
    if c is None:
        c = op.dense()
    m = inverse_sqrt(c)
    n3 = 3 * op.n
    # P_v = g . (M e_v), Q_v = g . e_v = g_v e_v; the scalar g_v is moved onto P_v
    p = (m * op.g[:, None] * op.g[None, :]).T.reshape(n3, op.n, 3)
    q = np.eye(n3).reshape(n3, op.n, 3)
    return 0.25 * bilinear_gradient(op.sys, p, q, op.mode, op.pairs)
