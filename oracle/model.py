"""MBD model quantities (arXiv 2307.02278, Review of the MBD and SL-MBD section).

Conventions (atomic units).  The dipole tensor is T(r) = grad_i grad_j 1/|R_i-R_j|
= (r^2 I - 3 r r^T) / r^5, so that the coupling block of Eq. ham is
V_ij = w_i w_j sqrt(a_i a_j) T'_ij with T' = s(R;beta) T (the damped tensor of
Eq. ham).  The paper defers the explicit damping to its earlier SL-MBD work;
the Fermi form of the rsSCS family is used:
    s(r) = 1 / (1 + exp(-d (r / (beta * (Rvdw_i + Rvdw_j)) - 1))).
"""
from __future__ import annotations

import numpy as np


def reciprocal_cell(cell: np.ndarray) -> np.ndarray:
    """Rows a*_alpha with a*_alpha . a_beta = delta_alpha_beta (Eq. dir_rec_intvec)."""
    return np.linalg.inv(np.asarray(cell, dtype=np.float64)).T


def cell_volume(cell: np.ndarray) -> float:
    """V = a1 . (a2 x a3) (Theory section)."""
    a1, a2, a3 = np.asarray(cell, dtype=np.float64)
    return float(np.dot(a1, np.cross(a2, a3)))


def fermi_damping(r, rvdw_sum, beta, d):
    """s(R; beta) of Eq. ham (Fermi form)."""
    return 1.0 / (1.0 + np.exp(-d * (r / (beta * rvdw_sum) - 1.0)))


def fermi_damping_dr(r, rvdw_sum, beta, d):
    """ds/dr = d / (beta Rsum) * s (1 - s)."""
    s = fermi_damping(r, rvdw_sum, beta, d)
    return d / (beta * rvdw_sum) * s * (1.0 - s)


def dipole_tensor(rvec: np.ndarray) -> np.ndarray:
    """Bare T(r) = (r^2 I - 3 r r^T) / r^5 for rvec of shape (..., 3) -> (..., 3, 3)."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r2 = np.sum(rvec * rvec, axis=-1)
    r5 = r2 ** 2.5
    eye = np.eye(3)
    return (r2[..., None, None] * eye - 3.0 * rvec[..., :, None] * rvec[..., None, :]) / r5[..., None, None]


def dipole_tensor_grad(rvec: np.ndarray) -> np.ndarray:
    """d T_ab / d r_c for the bare tensor, shape (..., 3, 3, 3) indexed [a, b, c]."""
    rvec = np.asarray(rvec, dtype=np.float64)
    r2 = np.sum(rvec * rvec, axis=-1)
    r = np.sqrt(r2)
    eye = np.eye(3)
    ra = rvec[..., :, None, None]
    rb = rvec[..., None, :, None]
    rc = rvec[..., None, None, :]
    r5 = (r ** 5)[..., None, None, None]
    r7 = (r ** 7)[..., None, None, None]
    return (-3.0 * (eye[:, :, None] * rc + eye[:, None, :] * rb + eye[None, :, :] * ra) / r5
            + 15.0 * ra * rb * rc / r7)


def g_vector(alpha: np.ndarray, omega: np.ndarray) -> np.ndarray:
    """g = (+)_i w_i sqrt(alpha_i) 1_3 (Eq. gvec), length 3N."""
    return np.repeat(np.asarray(omega) * np.sqrt(np.asarray(alpha)), 3)


def omega_diag(omega: np.ndarray) -> np.ndarray:
    """Diagonal of Omega = (+)_i w_i^2 I_3 (Eqs. vmbd, ccd), length 3N."""
    return np.repeat(np.asarray(omega) ** 2, 3)


def wrap_positions(cell: np.ndarray, pos: np.ndarray) -> np.ndarray:
    """Map Cartesian positions into the primary cell (fractional coordinates in [0,1))."""
    frac = np.asarray(pos) @ reciprocal_cell(cell).T
    frac = frac - np.floor(frac)
    return frac @ np.asarray(cell)
