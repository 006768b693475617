"""The MBD coupling matrix C (the paper's V) applied matrix-free or built densely.

Eq. ccd splits V = Omega + V~ with Omega = (+)_i w_i^2 I_3, and Eqs. hadamard,
lk3 write V~ y = Diag(g) T' (g . y).  Hence for any block of vectors x:
    C x = Omega x + g . (T'^pbc (g . x)).
"""
from __future__ import annotations

import numpy as np

from .ewald import apply_T, cutoffs, pair_list, pair_list_tree, real_space_matrix
from .model import g_vector, omega_diag


class Operator:
    """C for one system and one evaluation mode ("exact", "same_split", "spme")."""

    def __init__(self, sys, mode: str = "spme", tree_pairs: bool | None = None):
        self.sys = sys
        self.mode = mode
        self.n = sys.pos.shape[0]
        self.g = g_vector(sys.alpha, sys.omega)
        self.w2 = omega_diag(sys.omega)
        real_mode = "exact" if mode == "exact" else "same_split"
        rmax = max(cutoffs(sys, real_mode))
        if tree_pairs is None:
            tree_pairs = self.n > 2000
        self.pairs = (pair_list_tree if tree_pairs else pair_list)(sys.cell, sys.pos, rmax)
        self.real = real_space_matrix(sys, real_mode, self.pairs)

    def field(self, d: np.ndarray) -> np.ndarray:
        """E* = T'^pbc d for d of shape (nvec, N, 3)."""
        return apply_T(self.sys, d, self.mode, real_matrix=self.real)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        """y = C x for x of shape (nvec, 3N) or (3N,)."""
        x = np.asarray(x, dtype=np.float64)
        one = x.ndim == 1
        xb = x[None] if one else x
        d = (xb * self.g).reshape(xb.shape[0], self.n, 3)
        e = self.field(d).reshape(xb.shape[0], 3 * self.n)
        y = self.w2 * xb + self.g * e
        return y[0] if one else y

    def dense(self, block: int = 384) -> np.ndarray:
        """C as a dense 3N x 3N matrix, built column block by column block."""
        n3 = 3 * self.n
        out = np.empty((n3, n3))
        for c0 in range(0, n3, block):
            cols = np.eye(n3)[c0:c0 + block]
            out[:, c0:c0 + block] = self(cols).T
        return out
