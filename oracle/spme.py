"""SPME reciprocal-space generalized field (FP64, NumPy).

Follows Eqs. scaledfractional, spme and dipolarr of arXiv 2307.02278 (SPME of
Essmann et al. 1995 with the dipolar pair potential of Sagui et al. 2004):

  u_{alpha j} = K_alpha a*_alpha . R_j                       (scaled fractional coordinates)
  W_j(k) = prod_alpha M_p(u_{alpha j} - k_alpha - K_alpha n_alpha)   (periodic B-spline stencil)
  D(k)   = sum_j d_j . grad_{R_j} W_j(k)                     (dipole array, Eq. dipolarr)
  phi    = F^-1[ G . F[D] ]                                   (convolution by FFT)
  E^rec_i = sum_k grad_{R_i} W_i(k) phi(k)                    (field, Eq. spme)

with G(m) = B(m) exp(-pi^2 |m|^2 / beta^2) / (pi V |m|^2), G(0) = 0 (tin-foil),
B(m) = prod_alpha |b_alpha(m_alpha)|^2 the Euler exponential-spline moduli, and
m the reciprocal vector of the folded mesh index (m_alpha = k_alpha for
k_alpha <= K_alpha/2, else k_alpha - K_alpha).  Both DFTs are unnormalised.

Readings: "p-degree B-spline" in the text is taken as the order-p cardinal
B-spline M_p (p points per dimension, degree p-1); the garbled index
expression of Eq. dipolarr is read as the periodic wrap above.  For a
non-orthogonal cell the Nyquist planes are made symmetric by averaging G(m)
and G(-m), so that the convolution kernel is real and even; for orthorhombic
cells this changes nothing.
"""
from __future__ import annotations

import numpy as np

from .model import cell_volume, reciprocal_cell


def cardinal_bspline(x: np.ndarray, p: int) -> np.ndarray:
    """M_p(x): M_2(x) = 1 - |x - 1| on [0, 2], and
    M_n(x) = x/(n-1) M_{n-1}(x) + (n-x)/(n-1) M_{n-1}(x-1)."""
    x = np.asarray(x, dtype=np.float64)
    if p < 2:
        raise ValueError("order >= 2")
    if p == 2:
        return np.where((x >= 0.0) & (x <= 2.0), 1.0 - np.abs(x - 1.0), 0.0)
    n = p
    return x / (n - 1) * cardinal_bspline(x, n - 1) + (n - x) / (n - 1) * cardinal_bspline(x - 1.0, n - 1)


def cardinal_bspline_deriv(x: np.ndarray, p: int, order: int = 1) -> np.ndarray:
    """d/dx M_p = M_{p-1}(x) - M_{p-1}(x-1); second derivative by applying it twice."""
    if order == 0:
        return cardinal_bspline(x, p)
    return cardinal_bspline_deriv(x, p - 1, order - 1) - cardinal_bspline_deriv(x - 1.0, p - 1, order - 1)


def bspline_moduli(k: int, p: int) -> np.ndarray:
    """|b(m)|^2 = 1 / |sum_{j=0}^{p-2} M_p(j+1) exp(2 pi i m j / K)|^2, m = 0..K-1."""
    j = np.arange(p - 1)
    mj = cardinal_bspline(j + 1.0, p)
    m = np.arange(k)
    den = np.exp(2j * np.pi * np.outer(m, j) / k) @ mj
    return 1.0 / np.abs(den) ** 2


def folded_index(k: int) -> np.ndarray:
    """Mesh index -> signed frequency: m = k for k <= K/2, else k - K."""
    idx = np.arange(k)
    return np.where(idx <= k // 2, idx, idx - k)


def influence_function(sys) -> np.ndarray:
    """G(m) on the full K1 x K2 x K3 mesh of frequencies."""
    k1, k2, k3 = sys.mesh
    p = sys.spline_order
    beta = sys.ewald_beta
    recip = reciprocal_cell(sys.cell)
    vol = cell_volume(sys.cell)
    f = [folded_index(k) for k in sys.mesh]
    m = (f[0][:, None, None, None] * recip[0] + f[1][None, :, None, None] * recip[1]
         + f[2][None, None, :, None] * recip[2])
    m2 = np.sum(m * m, axis=-1)
    bmod = (bspline_moduli(k1, p)[:, None, None] * bspline_moduli(k2, p)[None, :, None]
            * bspline_moduli(k3, p)[None, None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        g = bmod * np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * vol * m2)
    g[0, 0, 0] = 0.0
    # symmetrise G(m) with G(-m mod K) (a no-op except on Nyquist planes of skew cells)
    gneg = g[np.ix_(*[(-np.arange(k)) % k for k in sys.mesh])]
    return 0.5 * (g + gneg)


def stencil(sys, pos: np.ndarray | None = None, deriv: int = 1):
    """Per atom: flat mesh indices (N, p^3) and the Cartesian derivatives of the
    weights W_j(k) wrt R_j: grad (N, p^3, 3) and, for deriv=2, Hessian (N, p^3, 3, 3)."""
    p = sys.spline_order
    kdim = np.asarray(sys.mesh)
    recip = reciprocal_cell(sys.cell)
    pos = np.asarray(sys.pos if pos is None else pos, dtype=np.float64)
    u = (pos @ recip.T) * kdim                     # (N, 3) scaled fractional coordinates
    base = np.floor(u).astype(np.int64)
    t = np.arange(p)
    x = (u - base)[:, :, None] + t[None, None, :]  # argument of M_p for mesh point base - t
    idx = np.mod(base[:, :, None] - t[None, None, :], kdim[None, :, None])  # (N,3,p)
    m0 = cardinal_bspline(x, p)
    m1 = cardinal_bspline_deriv(x, p, 1)
    # chain rule: du_beta / dR_alpha = K_beta a*_{beta alpha}
    cmat = kdim[:, None] * recip                   # (3 beta, 3 alpha)
    n = pos.shape[0]
    flat = (idx[:, 0, :, None, None] * (kdim[1] * kdim[2]) + idx[:, 1, None, :, None] * kdim[2]
            + idx[:, 2, None, None, :]).reshape(n, p ** 3)
    a, b, c = m0[:, 0, :, None, None], m0[:, 1, None, :, None], m0[:, 2, None, None, :]
    da, db, dc = m1[:, 0, :, None, None], m1[:, 1, None, :, None], m1[:, 2, None, None, :]
    du = np.stack([da * b * c, a * db * c, a * b * dc], -1).reshape(n, p ** 3, 3)
    grad = du @ cmat                               # dW/dR_alpha = sum_beta dW/du_beta C_{beta alpha}
    if deriv == 1:
        return flat, grad
    m2 = cardinal_bspline_deriv(x, p, 2)
    ea, eb, ec = m2[:, 0, :, None, None], m2[:, 1, None, :, None], m2[:, 2, None, None, :]
    huu = np.empty((n, p, p, p, 3, 3))
    huu[..., 0, 0] = ea * b * c
    huu[..., 1, 1] = a * eb * c
    huu[..., 2, 2] = a * b * ec
    huu[..., 0, 1] = huu[..., 1, 0] = da * db * c
    huu[..., 0, 2] = huu[..., 2, 0] = da * b * dc
    huu[..., 1, 2] = huu[..., 2, 1] = a * db * dc
    hess = np.einsum("ba,npqrbc,cd->npqrad", cmat, huu, cmat).reshape(n, p ** 3, 3, 3)
    return flat, grad, hess


def spread(sys, d: np.ndarray, st=None) -> np.ndarray:
    """Dipole array D(k) = sum_j d_j . grad W_j(k) (Eq. dipolarr); d (nvec,N,3) -> (nvec,K1,K2,K3)."""
    flat, grad = st if st is not None else stencil(sys)
    kk = int(np.prod(sys.mesh))
    contrib = np.einsum("vna,nsa->vns", d, grad)
    out = np.empty((d.shape[0], kk))
    for v in range(d.shape[0]):
        out[v] = np.bincount(flat.ravel(), weights=contrib[v].ravel(), minlength=kk)
    return out.reshape((d.shape[0],) + tuple(sys.mesh))


def convolve(sys, q: np.ndarray, g: np.ndarray | None = None) -> np.ndarray:
    """phi = F^-1[G F[D]] with unnormalised forward and inverse DFTs."""
    if g is None:
        g = influence_function(sys)
    qh = np.fft.fftn(q, axes=(1, 2, 3))
    return np.real(np.fft.ifftn(qh * g[None], axes=(1, 2, 3), norm="forward"))


def gather(sys, phi: np.ndarray, st=None) -> np.ndarray:
    """E_i = sum_k grad W_i(k) phi(k) (Eq. spme); phi (nvec,K1,K2,K3) -> (nvec,N,3)."""
    flat, grad = st if st is not None else stencil(sys)
    pv = phi.reshape(phi.shape[0], -1)[:, flat]           # (nvec, N, p^3)
    return np.einsum("vns,nsa->vna", pv, grad)


def reciprocal_field_spme(sys, d: np.ndarray) -> np.ndarray:
    st = stencil(sys)
    return gather(sys, convolve(sys, spread(sys, d, st)), st)
