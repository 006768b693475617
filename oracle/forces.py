"""Nuclear gradients (FP64).  The paper computes energies only and names the
gradients as future work (Conclusions); this module states them from the
energy it defines.

With alpha, omega independent of the positions (no SCS screening, Eq. ham
remark), dC/dR = Diag(g) dT'/dR Diag(g), and from Eq. plasmonic2
    dE/dR = (1/4) Tr(C^{-1/2} dC/dR).
The stochastic estimator uses the same normalised probes v_l as the energy:
    dE/dR ~ (1/4) (D/R) sum_l (g.w_l)^T (dT'/dR) (g.v_l),   w_l = C^{-1/2} v_l,
with w_l from the Lanczos basis of probe l (w ~ Y U diag(theta^-1/2) U^T e_1).

bilinear_gradient(P, Q) returns grad_R sum_v P_v^T T'^pbc(R) Q_v with P, Q held
fixed; every gradient above is a call of it.
"""
from __future__ import annotations

import numpy as np

from .ewald import (cutoffs, pair_list, real_space_tensor_grad, reciprocal_vectors)
from .lanczos import inverse_sqrt_action, lanczos, normalised_probes, quadrature
from .model import cell_volume, wrap_positions


def _real_space_gradient(sys, p, q, mode, pairs=None, chunk=20000):
    r_cut, damp_cut = cutoffs(sys, "exact" if mode == "exact" else "same_split")
    i, j, r = pairs if pairs is not None else pair_list(sys.cell, sys.pos, max(r_cut, damp_cut))
    grad = np.zeros(p.shape[1:])
    for c0 in range(0, i.size, chunk):
        ii, jj, rr = i[c0:c0 + chunk], j[c0:c0 + chunk], r[c0:c0 + chunk]
        da = real_space_tensor_grad(sys, ii, jj, rr, r_cut, damp_cut)   # (P,3,3,3)
        # term P_i^T A(R_i - R_j - n) Q_j: +dA/dr on atom i, -dA/dr on atom j
        t = np.einsum("vpa,pabc,vpb->pc", p[:, ii], da, q[:, jj])
        np.add.at(grad, ii, t)
        np.add.at(grad, jj, -t)
    return grad


def _reciprocal_gradient_direct(sys, p, q, chunk=1024):
    pos = wrap_positions(sys.cell, sys.pos)
    vol = cell_volume(sys.cell)
    beta = sys.ewald_beta
    k_all = 2.0 * np.pi * reciprocal_vectors(sys.cell, beta)
    grad = np.zeros(p.shape[1:])
    for k0 in range(0, k_all.shape[0], chunk):
        k = k_all[k0:k0 + chunk]
        k2 = np.sum(k * k, axis=1)
        pref = 2.0 * (4.0 * np.pi / vol) * np.exp(-k2 / (4.0 * beta * beta)) / k2
        phase = np.exp(1j * (pos @ k.T))                        # (N, nk)
        kp = np.einsum("vna,ka->vnk", p, k)
        kq = np.einsum("vna,ka->vnk", q, k)
        sp_ = np.einsum("vnk,nk->vk", kp, phase)
        sq_ = np.einsum("vnk,nk->vk", kq, phase)
        # d/dR_i Re[S_P S_Q^*] = k Re[i (k.P_i) e^{ik.R_i} S_Q^* - i (k.Q_i) e^{-ik.R_i} S_P]
        t = np.real(1j * kp * phase[None] * np.conj(sq_)[:, None, :]
                    - 1j * kq * np.conj(phase)[None] * sp_[:, None, :]).sum(axis=0)
        grad += np.einsum("nk,k,ka->na", t, pref, k)
    return grad


def _reciprocal_gradient_spme(sys, p, q):
    from .spme import convolve, influence_function, spread, stencil
    flat, grad_w, hess = stencil(sys, deriv=2)
    g = influence_function(sys)
    phi_p = convolve(sys, spread(sys, p, (flat, grad_w)), g)
    phi_q = convolve(sys, spread(sys, q, (flat, grad_w)), g)
    n = p.shape[1]
    out = np.zeros((n, 3))
    for v in range(p.shape[0]):
        fp = phi_p[v].ravel()[flat]                            # (N, p^3)
        fq = phi_q[v].ravel()[flat]
        # grad_i = sum_k H_i(k) [P_i phi_Q(k) + Q_i phi_P(k)]
        out += np.einsum("nsab,ns,nb->na", hess, fq, p[v]) + np.einsum("nsab,ns,nb->na", hess, fp, q[v])
    return out


def bilinear_gradient(sys, p: np.ndarray, q: np.ndarray, mode: str = "spme", pairs=None) -> np.ndarray:
    """grad_R sum_v P_v^T T'^pbc(R) Q_v, P and Q of shape (nvec, N, 3) -> (N, 3).
    The self term and Omega do not depend on R.  `pairs`: the pair list of the
    real-space sum when already at hand."""
    p = np.asarray(p, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    grad = _real_space_gradient(sys, p, q, mode, pairs)
    if mode == "spme":
        grad += _reciprocal_gradient_spme(sys, p, q)
    else:
        grad += _reciprocal_gradient_direct(sys, p, q)
    return grad


def estimator_forces(op, n_probes: int, n_steps: int, seed: int, first: int = 0, probes=None,
                     reorth: bool = False):
    """Stochastic force estimate F = -dE/dR with the probes of the energy estimate.
    probes: unit start vectors (n_probes, 3N) in place of the Rademacher rule
    (the pins use the 3N unit vectors, for which the estimate is the exact
    trace); reorth: full reorthogonalisation of the Lanczos basis."""
    n = op.n
    dim = 3 * n
    v = normalised_probes(seed, n_probes, dim, first) if probes is None else np.asarray(probes, dtype=np.float64)
    a, b, length, basis = lanczos(op, v, n_steps, reorth=reorth, keep_basis=True)
    w = np.stack([inverse_sqrt_action(a[l], b[l], length[l], basis[l]) for l in range(n_probes)])
    q = np.array([quadrature(a[l], b[l], length[l]) for l in range(n_probes)])
    pg = (w * op.g).reshape(n_probes, n, 3)
    qg = (v * op.g).reshape(n_probes, n, 3)
    grad = 0.25 * dim / n_probes * bilinear_gradient(op.sys, pg, qg, op.mode, op.pairs)
    energy = 0.5 * dim / n_probes * np.sum(q) - 1.5 * np.sum(op.sys.omega)
    return -grad, energy, dict(w=w, v=v, a=a, b=b, length=length, q=q)
