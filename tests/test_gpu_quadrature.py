"""Per-probe Gauss quadrature (Eqs. tridiag2, sl3) by the Chebyshev kernel
against QL and against an eigendecomposition in NumPy: q = e1^T Delta^{1/2} e1
= sum_k U_1k^2 sqrt(theta_k) and c = Delta^{-1/2} e1 = U diag(theta^{-1/2}) U^T e1."""
import numpy as np
import pytest
import torch

from oracle.lanczos import lanczos, normalised_probes
from oracle.operator import Operator
from workloads.systems import config

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _reference(a, b):
    """q and c per probe from numpy.linalg.eigh of the leading block (up to the
    first zero coupling)."""
    R, m = a.shape
    q = np.zeros(R)
    c = np.zeros((R, m))
    for r in range(R):
        n = m
        for k in range(m - 1):
            if b[r, k] == 0.0:
                n = k + 1
                break
        T = np.diag(a[r, :n]) + np.diag(b[r, :n - 1], 1) + np.diag(b[r, :n - 1], -1)
        th, U = np.linalg.eigh(T)
        q[r] = np.sum(U[0] ** 2 * np.sqrt(th))
        c[r, :n] = U @ (U[0] / np.sqrt(th))
    return q, c


def _random_tridiagonals(R, m, seed, spread=0.4):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 0.2 + spread, size=(R, m))
    b = rng.uniform(0.0, 0.08, size=(R, m))
    b[:, -1] = 0.0
    return a, b


def _check(mbd, a, b, tol_q=1e-12, tol_c=1e-11):
    q_ref, c_ref = _reference(a, b)
    for method in ("chebyshev", "ql"):
        q, c = mbd.tridiag_functions(a, b, method)
        np.testing.assert_allclose(q, q_ref, rtol=tol_q, err_msg=method)
        scale = np.abs(c_ref).max(axis=1, keepdims=True)
        assert np.all(np.abs(c - c_ref) <= tol_c * scale), method


@pytest.mark.parametrize("m", [1, 2, 7, 32, 33, 50, 64, 100, 128])
def test_random_tridiagonals(mbd, m):
    a, b = _random_tridiagonals(40, m, 100 + m)
    _check(mbd, a, b)


def test_lanczos_tridiagonals_with_converged_ritz_values(mbd):
    """Tridiagonals from the oracle's Lanczos on the 64-atom box (30 and 60
    steps, no reorthogonalisation: copies of converged Ritz values)."""
    s = config(1)
    op = Operator(s, "spme")
    v = normalised_probes(s.probe_seed, 8, 3 * s.n_atoms)
    for m in (30, 60):
        a, b, length, _ = lanczos(op, v, m)
        bb = np.zeros_like(b)
        for r in range(8):
            bb[r, :length[r] - 1] = b[r, :length[r] - 1]
        _check(mbd, a, bb)


def test_breakdown_lengths(mbd):
    a, b = _random_tridiagonals(16, 40, 7)
    for r in range(16):
        b[r, (r * 3) % 39] = 0.0            # length (3 r mod 39) + 1
    _check(mbd, a, b)


def test_ill_conditioned_fallback(mbd):
    """kappa ~ 1e5 is beyond the 256-term expansion: those probes go through QL;
    the well-conditioned ones stay on the Chebyshev kernel."""
    a, b = _random_tridiagonals(8, 24, 9)
    a[::2, 5] = 2e-6                         # a tiny eigenvalue in every other probe
    b[::2, 4] = b[::2, 5] = 1e-6
    _check(mbd, a, b, tol_q=1e-11, tol_c=1e-9)


def test_not_positive_definite(mbd):
    a, b = _random_tridiagonals(4, 10, 3)
    a[2, 3] = -0.5
    with pytest.raises(mbd.MBDError) as e:
        mbd.tridiag_functions(a, b, "chebyshev")
    assert e.value.code == 4


def test_energy_and_forces_methods_agree(mbd):
    s = config(1)
    res = {}
    for method in ("chebyshev", "ql"):
        g = mbd.MBDSystem.from_workload(s, quadrature=method)
        res[method] = g.energy_forces(16, 30, 55)
    (e0, f0), (e1, f1) = res["chebyshev"], res["ql"]
    assert abs(e0 - e1) <= 1e-12 * abs(e1)
    assert float((f0 - f1).abs().max()) <= 1e-10 * float(f1.abs().max())
