"""Stochastic Lanczos quadrature of Tr sqrt(C) (FP64).

Follows the Review section of arXiv 2307.02278 and its Algorithms 1 and 2:
  Hutchinson estimator (Eq. hutch) with normalised Rademacher probes (Eq. dds):
      Tr f(C) ~ (D/R) sum_l v_l^T f(C) v_l,  v_l = u_l / ||u_l||,  D = 3N
  Lanczos recurrence (Eqs. recurs, recurs2), y_0 = 0, b_1 = 0:
      y_1 = v;  y*_k = l_{k-1} - a_{k-1} y_{k-1} - b_{k-1} y_{k-2};  b_k = ||y*_k||
      y_k = y*_k / b_k;  l_k = C y_k;  a_k = y_k^T l_k
  Gauss quadrature (Eqs. sl3, sl4, tridiag1, tridiag2): nodes theta_k are the
  eigenvalues of the tridiagonal Delta, weights the squared first components
      v^T sqrt(C) v ~ sum_k U_1k^2 sqrt(theta_k)
  Energy (Eq. plasmonic2): E = (1/2) Tr sqrt(C) - (3/2) sum_i w_i

Probe rule (a counter-based generator, so both implementations draw identical
probes without sharing code): u_{l,i} = +1 when the top bit of
SplitMix64(seed + (l << 32) + i) is 0, else -1, where SplitMix64(x) is the
first output of Steele, Lea & Flood's SplitMix64 generator started at state x:
    z = x + 0x9E3779B97F4A7C15
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    return z ^ (z >> 31)                    (all arithmetic mod 2^64)

Readings: "n Lanczos steps" m is the number of products C y, i.e. the size of
Delta.  The recurrence stops early when b_k <= 1e-14 * |a_1| (breakdown): Delta
is then the leading (k-1) x (k-1) block.  A non-positive Ritz value means C is
not positive definite (polarisation catastrophe) and raises.  No
reorthogonalisation, as in the paper; full reorthogonalisation is an option.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import eigh_tridiagonal

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
MIX1 = np.uint64(0xBF58476D1CE4E5B9)
MIX2 = np.uint64(0x94D049BB133111EB)
BREAKDOWN = 1e-14


def splitmix64(x: np.ndarray) -> np.ndarray:
    """First SplitMix64 output for initial state x (uint64 array)."""
    z = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + GOLDEN
        z = (z ^ (z >> np.uint64(30))) * MIX1
        z = (z ^ (z >> np.uint64(27))) * MIX2
        return z ^ (z >> np.uint64(31))


def rademacher_probes(seed: int, n_probes: int, dim: int, first: int = 0) -> np.ndarray:
    """u_{l,i} in {+1, -1} for l = first .. first+n_probes-1, i = 0..dim-1 (Eq. dds)."""
    l = np.arange(first, first + n_probes, dtype=np.uint64)[:, None]
    i = np.arange(dim, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + (l << np.uint64(32)) + i
    top = splitmix64(x) >> np.uint64(63)
    return np.where(top == 0, 1.0, -1.0)


def normalised_probes(seed: int, n_probes: int, dim: int, first: int = 0) -> np.ndarray:
    u = rademacher_probes(seed, n_probes, dim, first)
    return u / np.linalg.norm(u, axis=1, keepdims=True)


def lanczos(apply_c, v: np.ndarray, m: int, reorth: bool = False, keep_basis: bool = False):
    """Lanczos recurrence for a block of start vectors v (R, D), run in lockstep.
    Returns a (R, m), b (R, m) with b[:, k] the coupling of y_k and y_{k+1}
    (b[:, m-1] unused), the per-probe length (R,), and optionally Y (R, m, D)."""
    v = np.asarray(v, dtype=np.float64)
    r, dim = v.shape
    a = np.zeros((r, m))
    b = np.zeros((r, m))
    length = np.full(r, m, dtype=np.int64)
    basis = np.zeros((r, m, dim)) if (keep_basis or reorth) else None
    y_prev = np.zeros_like(v)
    y = v.copy()
    active = np.ones(r, dtype=bool)
    b_prev = np.zeros(r)
    l = apply_c(y)
    a[:, 0] = np.einsum("rd,rd->r", y, l)
    if basis is not None:
        basis[:, 0] = y
    a1 = np.abs(a[:, 0])
    for k in range(1, m):
        ystar = l - a[:, k - 1, None] * y - b_prev[:, None] * y_prev
        if reorth:
            for _ in range(2):
                coef = np.einsum("rkd,rd->rk", basis[:, :k], ystar)
                ystar = ystar - np.einsum("rk,rkd->rd", coef, basis[:, :k])
        bk = np.linalg.norm(ystar, axis=1)
        stop = active & (bk <= BREAKDOWN * a1)
        length[stop] = k
        active &= ~stop
        bk = np.where(active, bk, 0.0)
        inv = np.where(active, 1.0 / np.where(bk > 0, bk, 1.0), 0.0)
        y_prev, y = y, ystar * inv[:, None]
        b[:, k - 1] = bk
        b_prev = bk
        if basis is not None:
            basis[:, k] = y
        l = apply_c(y)
        a[:, k] = np.where(active, np.einsum("rd,rd->r", y, l), 0.0)
    return a, b, length, basis


def ritz(a: np.ndarray, b: np.ndarray, length: int):
    """Eigenpairs (theta, U) of the symmetric tridiagonal Delta (Eq. tridiag2)."""
    n = int(length)
    return eigh_tridiagonal(a[:n], b[:n - 1])


def quadrature(a: np.ndarray, b: np.ndarray, length: int, f=np.sqrt) -> float:
    """v^T f(C) v ~ sum_k U_1k^2 f(theta_k) for ||v|| = 1 (Eq. sl3)."""
    theta, u = ritz(a, b, length)
    if np.any(theta <= 0.0):
        raise FloatingPointError("non-positive Ritz value: C is not positive definite")
    return float(np.sum(u[0] ** 2 * f(theta)))


def slq(apply_c, dim: int, n_probes: int, n_steps: int, seed: int, first: int = 0,
        reorth: bool = False):
    """Per-probe quadratures q_l and the (a, b, length) of each probe (Algorithm 1)."""
    v = normalised_probes(seed, n_probes, dim, first)
    a, b, length, _ = lanczos(apply_c, v, n_steps, reorth=reorth)
    q = np.array([quadrature(a[l], b[l], length[l]) for l in range(n_probes)])
    return q, a, b, length


def slq_energy(op, n_probes: int, n_steps: int, seed: int, reorth: bool = False):
    """E_MBD ~ (1/2) (3N/R) sum_l q_l - (3/2) sum w (Algorithm 1, Eq. plasmonic2)."""
    dim = 3 * op.n
    q, a, b, length = slq(op, dim, n_probes, n_steps, seed, reorth=reorth)
    trace = dim / n_probes * np.sum(q)
    return 0.5 * trace - 1.5 * np.sum(op.sys.omega), dict(q=q, a=a, b=b, length=length, trace=trace)


def inverse_sqrt_action(a: np.ndarray, b: np.ndarray, length: int, basis: np.ndarray) -> np.ndarray:
    """w = C^{-1/2} v ~ Y U diag(theta^{-1/2}) U^T e_1 for ||v|| = 1."""
    theta, u = ritz(a, b, length)
    c = u @ (theta ** -0.5 * u[0])
    n = int(length)
    return c @ basis[:n]
