"""Self-consistent screening (SCS) of the atomic polarisabilities: the front
end of the MBD@rsSCS model (plain FP64, dense).

TEST INFRASTRUCTURE ONLY: the independent checker of the library's screening
entry point (see oracle/__init__.py for who may import it).

arXiv 2307.02278 names this step in its review of the MBD model (the atomic
polarisabilities, made frequency-dependent, are screened by a Dyson-like
equation solved at a set of frequencies, and the screened values enter the
MBD matrix) and leaves it out of its own scope: its algorithm takes screened
and unscreened parameters alike.  The published range-separated SCS scheme
(Tkatchenko, DiStasio, Car & Scheffler 2012; Ambrosetti et al. 2014) is
restated here with these readings:

  alpha_i(iu)  = alpha_i / (1 + (u / omega_i)^2)              single-pole polarisability
  sigma_i(u)   = (sqrt(2/pi) alpha_i(iu) / 3)^(1/3)           width of the Gaussian oscillator density
  T_GG(r; s)   = grad_i grad_j erf(|r|/s) / |r|,  s = sqrt(sigma_i^2 + sigma_j^2),  r = R_i - R_j
  T_SR_ij(u)   = sum'_n (1 - f(|r + n|)) T_GG(r + n; s_ij(u))  (f: the Fermi damping of model.py with
                 the system's beta, d and R_vdw; the prime skips i = j, n = 0; pairs with
                 |r + n| < damp_cut, the truncation of the damping correction of the MBD operator)
  B(u)         = (A(u)^-1 + T_SR(u))^-1,  A(u) = diag(alpha_i(iu)) (x) I_3
  alpha_i^SCS(iu) = (1/3) sum_c [B(u) 1_c]_(i,c),  1_c: unit vector along c on every atom
  C6_i         = (3/pi) int_0^inf alpha_i^SCS(iu)^2 du        (Casimir-Polder)
  omega_i^SCS  = 4 C6_i / (3 alpha_i^SCS(0)^2)
  Rvdw_i^SCS   = Rvdw_i (alpha_i^SCS(0) / alpha_i)^(1/3)

The Casimir-Polder integral runs over n Gauss-Legendre nodes t_k on (-1, 1)
mapped to u = u0 (1 + t) / (1 - t) with u0 = 0.5 Ha.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.special import erf

from .ewald import exact_damp_cutoff, pair_list, pair_list_tree
from .model import fermi_damping

U0 = 0.5
TWO_OVER_SQRT_PI = 2.0 / np.sqrt(np.pi)


def frequency_grid(n_freq: int, u0: float = U0):
    """Nodes u_k and weights w_k with sum_k w_k f(u_k) ~ int_0^inf f(u) du
    (Gauss-Legendre in t, u = u0 (1 + t) / (1 - t), du = 2 u0 / (1 - t)^2 dt)."""
    t, w = np.polynomial.legendre.leggauss(n_freq)
    return u0 * (1.0 + t) / (1.0 - t), w * 2.0 * u0 / (1.0 - t) ** 2


def dynamic_polarizability(alpha, omega, u):
    """alpha_i(iu) = alpha_i / (1 + (u / omega_i)^2)."""
    return np.asarray(alpha, dtype=np.float64) / (1.0 + (u / np.asarray(omega, dtype=np.float64)) ** 2)


def gaussian_width(alpha_u):
    """sigma_i = (sqrt(2/pi) alpha_i(iu) / 3)^(1/3)."""
    return (np.sqrt(2.0 / np.pi) * np.asarray(alpha_u, dtype=np.float64) / 3.0) ** (1.0 / 3.0)


def pair_width(sigma_i, sigma_j):
    """Width of the interaction of two Gaussian densities: the potential
    between them is erf(r / s_ij) / r with s_ij = sqrt(sigma_i^2 + sigma_j^2)."""
    return np.sqrt(np.asarray(sigma_i) ** 2 + np.asarray(sigma_j) ** 2)


def gg_tensor(rvec, sigma):
    """T_GG(r; sigma) = -grad grad [erf(|r|/sigma) / |r|] = c_id I - c_rr r r^T for
    rvec (..., 3) and sigma (...), returned as (..., 3, 3).  With x = r/sigma,
    E = erf(x), e = exp(-x^2), k = 2/sqrt(pi):
        c_id = E/r^3 - k e/(sigma r^2)
        c_rr = 3E/r^5 - 3k e/(sigma r^4) - 2k e/(sigma^3 r^2)."""
    rvec = np.asarray(rvec, dtype=np.float64)
    sigma = np.asarray(sigma, dtype=np.float64)
    r2 = np.sum(rvec * rvec, axis=-1)
    r = np.sqrt(r2)
    x = r / sigma
    big_e = erf(x)
    e = np.exp(-x * x)
    k = TWO_OVER_SQRT_PI
    c_id = big_e / (r2 * r) - k * e / (sigma * r2)
    c_rr = 3.0 * big_e / (r2 * r2 * r) - 3.0 * k * e / (sigma * r2 * r2) - 2.0 * k * e / (sigma ** 3 * r2)
    eye = np.eye(3)
    return c_id[..., None, None] * eye - c_rr[..., None, None] * rvec[..., :, None] * rvec[..., None, :]


def sr_sparse(sys, u: float, pairs, damp_cut: float) -> sp.csr_matrix:
    """T_SR(u) as a sparse 3N x 3N matrix over the pairs (i, j, r = R_i - R_j - n)
    with |r| < damp_cut (repeated (i, j) entries, from different images, add)."""
    i, j, r = pairs
    n = sys.pos.shape[0]
    sig = gaussian_width(dynamic_polarizability(sys.alpha, sys.omega, u))
    rho = np.linalg.norm(r, axis=1)
    one_minus_f = 1.0 - fermi_damping(rho, sys.r_vdw[i] + sys.r_vdw[j], sys.damp_beta, sys.damp_d)
    t = gg_tensor(r, pair_width(sig[i], sig[j])) * ((rho < damp_cut) * one_minus_f)[:, None, None]
    rows = 3 * i[:, None, None] + np.arange(3)[None, :, None] + 0 * np.arange(3)[None, None, :]
    cols = 3 * j[:, None, None] + np.arange(3)[None, None, :] + 0 * np.arange(3)[None, :, None]
    return sp.coo_matrix((t.ravel(), (rows.ravel(), cols.ravel())), shape=(3 * n, 3 * n)).tocsr()


def sr_matrix(sys, u: float, pairs, damp_cut: float) -> np.ndarray:
    """Dense 3N x 3N T_SR(u)."""
    return sr_sparse(sys, u, pairs, damp_cut).toarray()


def _unit_columns(n: int) -> np.ndarray:
    ones = np.zeros((3 * n, 3))
    for c in range(3):
        ones[c::3, c] = 1.0
    return ones


def screened_polarizability(sys, u: float, pairs, damp_cut: float) -> np.ndarray:
    """alpha_i^SCS(iu) = (1/3) sum_c [(A(u)^-1 + T_SR(u))^-1 1_c]_(i,c), by a dense solve."""
    n = sys.pos.shape[0]
    a_u = dynamic_polarizability(sys.alpha, sys.omega, u)
    m = sr_matrix(sys, u, pairs, damp_cut) + np.diag(np.repeat(1.0 / a_u, 3))
    x = np.linalg.solve(m, _unit_columns(n))
    return (x[0::3, 0] + x[1::3, 1] + x[2::3, 2]) / 3.0


def screened_polarizability_cg(sys, u: float, pairs, damp_cut: float, rtol: float = 1e-13) -> np.ndarray:
    """The same by scipy's conjugate gradient on the sparse matrix (preconditioner
    A(u)), for systems too large for the dense solve."""
    from scipy.sparse.linalg import LinearOperator, cg
    n = sys.pos.shape[0]
    a3 = np.repeat(dynamic_polarizability(sys.alpha, sys.omega, u), 3)
    m = sr_sparse(sys, u, pairs, damp_cut) + sp.diags(1.0 / a3)
    pre = LinearOperator(m.shape, matvec=lambda v: a3 * np.ravel(v))
    b = _unit_columns(n)
    out = np.zeros(n)
    for c in range(3):
        try:
            x, info = cg(m, b[:, c], x0=a3 * b[:, c], rtol=rtol, atol=0.0, M=pre, maxiter=2000)
        except TypeError:                        # scipy before 1.12 names it tol
            x, info = cg(m, b[:, c], x0=a3 * b[:, c], tol=rtol, atol=0.0, M=pre, maxiter=2000)
        if info != 0:
            raise RuntimeError(f"cg did not converge (info {info})")
        out += x[c::3] / 3.0
    return out


def scs(sys, n_freq: int = 23, mode: str = "same_split", pairs=None, solver: str = "dense") -> dict:
    """Screened static polarisabilities, C6 coefficients, characteristic
    frequencies and vdW radii.  mode "same_split": pairs within sys.damp_cut
    (the library's truncation); "exact": within the radius where 1 - f < 1e-17.
    solver "dense" (np.linalg.solve) or "cg" (sparse, for larger systems).
    alpha_iu[0] is the static value, alpha_iu[k + 1] the value at node u_k."""
    damp_cut = float(sys.damp_cut) if mode == "same_split" else exact_damp_cutoff(sys)
    if pairs is None:
        pairs = (pair_list_tree if sys.pos.shape[0] > 2000 else pair_list)(sys.cell, sys.pos, damp_cut)
    solve = screened_polarizability if solver == "dense" else screened_polarizability_cg
    u, w = frequency_grid(n_freq)
    a0 = solve(sys, 0.0, pairs, damp_cut)
    a_u = np.array([solve(sys, float(uk), pairs, damp_cut) for uk in u])
    c6 = 3.0 / np.pi * np.einsum("k,kn->n", w, a_u ** 2)
    return {"alpha": a0, "omega": 4.0 * c6 / (3.0 * a0 ** 2), "r_vdw": sys.r_vdw * (a0 / sys.alpha) ** (1.0 / 3.0),
            "c6": c6, "alpha_iu": np.vstack([a0[None, :], a_u]), "u": np.concatenate([[0.0], u]), "w": w}
