"""Brute-force replica sum of Eq. replica (arXiv 2307.02278, Theory section).

T^pbc_ij = sum_n T'_ij(j in n) over the periodic images n of the cell whose
lattice vector satisfies |n| <= R_cut (whole cells, a spherical cluster of
cells).  The paper uses it as the slowly, conditionally convergent comparison
method; here it only pins ewald.py: for a growing sphere of cells it tends to
the tin-foil Ewald field plus the surface term (4 pi / 3V) sum_j d_j on every
atom (a sphere of cells in vacuum).
"""
from __future__ import annotations

import numpy as np

from .model import dipole_tensor, fermi_damping, wrap_positions


def replica_field(sys, d: np.ndarray, r_cut: float, damped: bool = True) -> np.ndarray:
    """E_i = sum_{|n| <= r_cut} sum_j' s T(R_i - R_j - n) d_j, d of shape (nvec, N, 3)."""
    cell = np.asarray(sys.cell, dtype=np.float64)
    pos = wrap_positions(cell, sys.pos)
    nmax = int(np.ceil(r_cut / np.min(np.linalg.norm(cell, axis=1)))) + 1
    rng = np.arange(-nmax, nmax + 1)
    ints = np.stack(np.meshgrid(rng, rng, rng, indexing="ij"), -1).reshape(-1, 3)
    shifts = ints.astype(np.float64) @ cell
    shifts = shifts[np.linalg.norm(shifts, axis=1) <= r_cut]
    n = pos.shape[0]
    out = np.zeros_like(np.asarray(d, dtype=np.float64))
    for i in range(n):
        for j in range(n):
            r = pos[i] - pos[j] - shifts
            r2 = np.sum(r * r, axis=1)
            r = r[r2 > 0.0]
            t = dipole_tensor(r)
            if damped:
                rho = np.linalg.norm(r, axis=1)
                s = fermi_damping(rho, sys.r_vdw[i] + sys.r_vdw[j], sys.damp_beta, sys.damp_d)
                t = t * s[:, None, None]
            out[:, i] += np.einsum("ab,vb->va", t.sum(axis=0), d[:, j])
    return out
