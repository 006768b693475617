"""Periodic generalized field E = T'^pbc d by direct Ewald summation (FP64).

Follows the Theory section of arXiv 2307.02278: the conditionally convergent
replica sum of Eq. replica is replaced by the absolutely convergent split of
Eq. ewalddip, E* = E^dir + E^rec + E^self, with the damping entering through
the short-range correction sum of Eq. fld_ewald.

Readings of the printed formulas (the printed brackets of Eq. fld_ewald and the
prefactors of Eqs. fld_ewald1/fld_ewald2 are garbled; the standard dipolar
Ewald sum in the T = grad grad 1/r convention is used):
  T'^pbc_ij = sum'_n s(|r+n|) T(r+n),  r = R_i - R_j, prime: skip i=j, n=0
            = sum'_n [B1 I - B2 r r^T](r+n)                 (erfc-screened, Smith's B_n)
              + (4 pi / V) sum_{k != 0} exp(-k^2/4b^2)/k^2 k k^T cos(k.r)   (k = 2 pi m)
              - delta_ij (4 b^3 / (3 sqrt(pi))) I            (self term)
              - sum'_n (1 - s) T(r+n)                        (damping correction)
  The k = 0 term is omitted (tin-foil boundary, Eq. fld_ewald2 sums m != 0).

Two truncation modes:
  "exact":      every sum converged to ~1e-16 relative.
  "same_split": real-space erfc sum truncated at sys.r_cut and the damping
                correction at sys.damp_cut (the GPU path's truncation), with a
                converged reciprocal sum; isolates the SPME mesh error.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.special import erfc

from .model import (cell_volume, dipole_tensor, dipole_tensor_grad, fermi_damping,
                    fermi_damping_dr, reciprocal_cell, wrap_positions)

SQRT_PI = np.sqrt(np.pi)
TOL = 1e-17


def smith_b(r, beta):
    """Smith's erfc-screened radial functions B0..B3 (B_n = [(2n-1) B_{n-1}
    + (2 beta^2)^n / (beta sqrt(pi)) exp(-beta^2 r^2)] / r^2)."""
    e = np.exp(-(beta * r) ** 2)
    b0 = erfc(beta * r) / r
    b1 = (b0 + 2.0 * beta / SQRT_PI * e) / r ** 2
    b2 = (3.0 * b1 + 4.0 * beta ** 3 / SQRT_PI * e) / r ** 2
    b3 = (5.0 * b2 + 8.0 * beta ** 5 / SQRT_PI * e) / r ** 2
    return b0, b1, b2, b3


def self_coefficient(beta: float) -> float:
    """E^self = -(4 beta^3 / (3 sqrt(pi))) d in the T = grad grad 1/r convention
    (Eq. fld_ewald1 prints 2 tau^3/(3 sqrt(pi)): the energy coefficient, doubled by
    l_k = (1/2) da_k/dy_k of Eq. lk2, with the sign of this convention)."""
    return -4.0 * beta ** 3 / (3.0 * SQRT_PI)


def exact_real_cutoff(beta: float) -> float:
    """Radius beyond which exp(-beta^2 r^2) < 1e-17."""
    return np.sqrt(-np.log(TOL)) / beta


def exact_damp_cutoff(sys) -> float:
    """Radius beyond which 1 - s < 1e-17 for every pair."""
    rsum = 2.0 * float(np.max(sys.r_vdw))
    return sys.damp_beta * rsum * (1.0 + (-np.log(TOL)) / sys.damp_d)


def cutoffs(sys, mode: str):
    if mode == "exact":
        return exact_real_cutoff(sys.ewald_beta), exact_damp_cutoff(sys)
    return float(sys.r_cut), float(sys.damp_cut)


def lattice_shifts(cell: np.ndarray, rmax: float) -> np.ndarray:
    """All lattice vectors n = n1 a1 + n2 a2 + n3 a3 that can bring an image of an
    atom of the (wrapped) cell within rmax of another atom of the cell."""
    recip = reciprocal_cell(cell)
    nmax = [int(np.ceil(rmax * np.linalg.norm(recip[a]))) + 1 for a in range(3)]
    rng = [np.arange(-n, n + 1) for n in nmax]
    ints = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    return ints.astype(np.float64) @ np.asarray(cell, dtype=np.float64), ints


def pair_list(cell: np.ndarray, pos: np.ndarray, rmax: float, chunk: int = 256):
    """Brute force: all (i, j, r) with r = R_i - R_j - n, 0 < |r| < rmax, over every
    atom pair and every lattice vector n (the i = j, n = 0 term excluded)."""
    pos = wrap_positions(cell, pos)
    shifts, _ = lattice_shifts(cell, rmax)
    n = pos.shape[0]
    out_i, out_j, out_r = [], [], []
    for i0 in range(0, n, chunk):
        diff = pos[i0:i0 + chunk, None, :] - pos[None, :, :]
        for s in shifts:
            r = diff - s
            r2 = np.einsum("ijk,ijk->ij", r, r)
            ii, jj = np.nonzero((r2 < rmax * rmax) & (r2 > 0.0))
            out_i.append(ii + i0)
            out_j.append(jj)
            out_r.append(r[ii, jj])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_r)


def pair_list_tree(cell: np.ndarray, pos: np.ndarray, rmax: float):
    """The same pair set as pair_list for an orthorhombic cell whose shortest
    edge exceeds 2 rmax (each pair then has one image within rmax, the minimum
    image), found with a periodic k-d tree; falls back to pair_list otherwise."""
    cell = np.asarray(cell, dtype=np.float64)
    box = np.diag(cell)
    if np.any(np.abs(cell - np.diag(box)) > 0) or rmax >= 0.5 * box.min():
        return pair_list(cell, pos, rmax)
    from scipy.spatial import cKDTree
    pos = wrap_positions(cell, pos)
    tree = cKDTree(pos, boxsize=box)
    pairs = tree.query_pairs(rmax, output_type="ndarray")
    i = np.concatenate([pairs[:, 0], pairs[:, 1]])
    j = np.concatenate([pairs[:, 1], pairs[:, 0]])
    r = pos[i] - pos[j]
    r -= box * np.round(r / box)
    keep = np.einsum("ij,ij->i", r, r) < rmax * rmax
    order = np.lexsort((j[keep], i[keep]))
    return i[keep][order], j[keep][order], r[keep][order]


def real_space_tensor(sys, i, j, rvec, r_cut: float, damp_cut: float) -> np.ndarray:
    """Pair tensor of E^dir including the damping correction of Eq. fld_ewald:
    A(r) = [|r|<r_cut] (B1 I - B2 r r^T) - [|r|<damp_cut] (1 - s(|r|)) T(r)."""
    rho = np.linalg.norm(rvec, axis=1)
    _, b1, b2, _ = smith_b(rho, sys.ewald_beta)
    eye = np.eye(3)
    a = (b1[:, None, None] * eye - b2[:, None, None] * rvec[:, :, None] * rvec[:, None, :])
    a *= (rho < r_cut)[:, None, None]
    rsum = sys.r_vdw[i] + sys.r_vdw[j]
    one_minus_s = 1.0 - fermi_damping(rho, rsum, sys.damp_beta, sys.damp_d)
    a -= ((rho < damp_cut) * one_minus_s)[:, None, None] * dipole_tensor(rvec)
    return a


def real_space_tensor_grad(sys, i, j, rvec, r_cut: float, damp_cut: float) -> np.ndarray:
    """dA_ab/dr_c of real_space_tensor, shape (P,3,3,3) indexed [a,b,c]."""
    rho = np.linalg.norm(rvec, axis=1)
    _, _, b2, b3 = smith_b(rho, sys.ewald_beta)
    eye = np.eye(3)
    ra = rvec[:, :, None, None]
    rb = rvec[:, None, :, None]
    rc = rvec[:, None, None, :]
    sym = eye[None, :, :, None] * rc + eye[None, :, None, :] * rb + eye[None, None, :, :] * ra
    g = -b2[:, None, None, None] * sym + b3[:, None, None, None] * ra * rb * rc
    g *= (rho < r_cut)[:, None, None, None]
    rsum = sys.r_vdw[i] + sys.r_vdw[j]
    s = fermi_damping(rho, rsum, sys.damp_beta, sys.damp_d)
    ds = fermi_damping_dr(rho, rsum, sys.damp_beta, sys.damp_d)
    t = dipole_tensor(rvec)
    dt = dipole_tensor_grad(rvec)
    corr = -(ds / rho)[:, None, None, None] * t[:, :, :, None] * rvec[:, None, None, :] \
        + (1.0 - s)[:, None, None, None] * dt
    g -= (rho < damp_cut)[:, None, None, None] * corr
    return g


def real_space_matrix(sys, mode: str, pairs=None) -> sp.csr_matrix:
    """Sparse 3N x 3N matrix of E^dir (erfc part + damping correction);
    `pairs` = pair_list(cell, pos, max(cutoffs)) when already at hand."""
    r_cut, damp_cut = cutoffs(sys, mode)
    i, j, r = pairs if pairs is not None else pair_list(sys.cell, sys.pos, max(r_cut, damp_cut))
    a = real_space_tensor(sys, i, j, r, r_cut, damp_cut)
    rows = (3 * i[:, None, None] + np.arange(3)[None, :, None]) + 0 * np.arange(3)[None, None, :]
    cols = (3 * j[:, None, None] + np.arange(3)[None, None, :]) + 0 * np.arange(3)[None, :, None]
    n3 = 3 * sys.pos.shape[0]
    return sp.coo_matrix((a.ravel(), (rows.ravel(), cols.ravel())), shape=(n3, n3)).tocsr()


def reciprocal_vectors(cell: np.ndarray, beta: float):
    """Half space of reciprocal vectors m = sum m_a a*_a (Eq. dir_rec_intvec), m != 0,
    with exp(-pi^2 m^2 / beta^2) > 1e-17; returns Cartesian m (bohr^-1)."""
    recip = reciprocal_cell(cell)
    mmax = np.sqrt(-np.log(TOL)) * beta / np.pi
    nmax = [int(np.ceil(mmax * np.linalg.norm(np.asarray(cell)[a]))) for a in range(3)]
    rng = [np.arange(-n, n + 1) for n in nmax]
    ints = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    half = (ints[:, 0] > 0) | ((ints[:, 0] == 0) & (ints[:, 1] > 0)) | \
        ((ints[:, 0] == 0) & (ints[:, 1] == 0) & (ints[:, 2] > 0))
    ints = ints[half]
    m = ints.astype(np.float64) @ recip
    m2 = np.sum(m * m, axis=1)
    keep = m2 <= mmax * mmax
    return m[keep]


def reciprocal_field_direct(sys, d: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """E^rec of Eq. fld_ewald2 (structure factor of Eq. structurefactor), k = 2 pi m:
    E_i = (4 pi / V) sum_{k != 0} exp(-k^2/4b^2)/k^2 k Re[e^{i k.R_i} S(k)^*],
    S(k) = sum_j (k . d_j) e^{i k.R_j}; the half space is summed twice."""
    pos = wrap_positions(sys.cell, sys.pos)
    vol = cell_volume(sys.cell)
    beta = sys.ewald_beta
    k_all = 2.0 * np.pi * reciprocal_vectors(sys.cell, beta)
    out = np.zeros_like(d)
    for k0 in range(0, k_all.shape[0], chunk):
        k = k_all[k0:k0 + chunk]
        k2 = np.sum(k * k, axis=1)
        pref = 2.0 * (4.0 * np.pi / vol) * np.exp(-k2 / (4.0 * beta * beta)) / k2
        phase = np.exp(1j * (pos @ k.T))                       # (N, nk)
        kd = np.einsum("vna,ka->vnk", d, k)                    # (nvec, N, nk)
        s = np.einsum("vnk,nk->vk", kd, phase)                 # (nvec, nk)
        re = np.real(phase[None, :, :] * np.conj(s)[:, None, :])   # (nvec, N, nk)
        out += np.einsum("vnk,k,ka->vna", re, pref, k)
    return out


def apply_T(sys, d: np.ndarray, mode: str = "exact", real_matrix=None) -> np.ndarray:
    """E* = T'^pbc d for d of shape (nvec, N, 3) (Eq. ewalddip).
    mode: "exact" | "same_split" (direct reciprocal sum) | "spme" (SPME reciprocal)."""
    d = np.asarray(d, dtype=np.float64)
    if real_matrix is None:
        real_matrix = real_space_matrix(sys, "exact" if mode == "exact" else "same_split")
    nvec, n, _ = d.shape
    e_real = (real_matrix @ d.reshape(nvec, 3 * n).T).T.reshape(nvec, n, 3)
    if mode == "spme":
        from .spme import reciprocal_field_spme
        e_rec = reciprocal_field_spme(sys, d)
    else:
        e_rec = reciprocal_field_direct(sys, d)
    return e_real + e_rec + self_coefficient(sys.ewald_beta) * d
