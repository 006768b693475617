"""Pins for oracle/lanczos.py and oracle/dense.py: full-Krylov exactness, an
independent Householder tridiagonalisation, breakdown, positivity and the
statistical agreement of the Hutchinson estimator with the dense energy."""
import numpy as np
import pytest
from scipy.linalg import hessenberg

from oracle.dense import dense_energy
from oracle.lanczos import lanczos, normalised_probes, quadrature, slq, slq_energy
from oracle.operator import Operator
from workloads.systems import random_system


@pytest.fixture(scope="module")
def small():
    s = random_system(16, 14.0, 5, mesh=(20, 20, 20), r_cut=6.9, damp_cut=6.9)
    op = Operator(s, "spme")
    return s, op, op.dense()


def test_full_krylov_quadrature_exact(small):
    """With m = D and full reorthogonalisation the Gauss quadrature is exact:
    sum_k U_1k^2 sqrt(theta_k) = v^T sqrt(C) v."""
    s, op, c = small
    lam, u = np.linalg.eigh(c)
    sq = (u * np.sqrt(lam)) @ u.T
    v = normalised_probes(7, 3, c.shape[0])
    a, b, length, _ = lanczos(op, v, c.shape[0], reorth=True)
    for l in range(3):
        assert abs(quadrature(a[l], b[l], length[l]) - v[l] @ sq @ v[l]) < 1e-12


def test_unit_probes_give_exact_trace(small):
    """The D unit vectors as probes and full Krylov reproduce Eq. plasmonic."""
    s, op, c = small
    dim = c.shape[0]
    a, b, length, _ = lanczos(op, np.eye(dim), dim, reorth=True)
    trace = sum(quadrature(a[l], b[l], length[l]) for l in range(dim))
    e = 0.5 * trace - 1.5 * np.sum(s.omega)
    assert abs(e - dense_energy(c, s.omega)) < 1e-12 * abs(e)


def test_lanczos_matches_householder(small):
    """a_k, b_k equal the tridiagonal form of C from Householder reflections in a
    basis whose first vector is v."""
    s, op, c = small
    dim = c.shape[0]
    v = normalised_probes(11, 1, dim)[0]
    e1 = np.zeros(dim)
    e1[0] = 1.0
    w = v - e1
    w /= np.linalg.norm(w)
    h0 = np.eye(dim) - 2.0 * np.outer(w, w)
    t = hessenberg(h0 @ c @ h0)
    a, b, _, _ = lanczos(op, v[None], 12)
    np.testing.assert_allclose(a[0], np.diag(t)[:12], rtol=0, atol=1e-13)
    np.testing.assert_allclose(b[0, :11], np.abs(np.diag(t, -1)[:11]), rtol=0, atol=1e-13)


def test_orthogonality_at_15(small):
    """Numerical results section: with M+1 = 15 the basis stays orthogonal."""
    s, op, c = small
    v = normalised_probes(3, 2, c.shape[0])
    _, _, _, y = lanczos(op, v, 15, keep_basis=True)
    for l in range(2):
        g = y[l] @ y[l].T
        assert np.abs(g - np.eye(15)).max() < 1e-8


def test_breakdown_on_invariant_subspace():
    """A start vector inside an invariant subspace of dimension 2 stops after two
    steps and still gives v^T sqrt(C) v exactly."""
    lam = np.array([1.0, 4.0, 9.0, 16.0])
    c = np.diag(lam)
    v = np.array([[0.6, 0.8, 0.0, 0.0]])
    a, b, length, _ = lanczos(lambda x: x @ c, v, 4)
    assert length[0] == 2
    assert abs(quadrature(a[0], b[0], length[0]) - (0.36 * 1 + 0.64 * 2)) < 1e-14


def test_not_positive_definite_raises():
    c = np.diag([1.0, -0.5, 2.0])
    v = np.ones((1, 3)) / np.sqrt(3)
    a, b, length, _ = lanczos(lambda x: x @ c, v, 3)
    with pytest.raises(FloatingPointError):
        quadrature(a[0], b[0], length[0])


def test_hutchinson_statistics(small):
    """The SLQ energy agrees with the dense energy within its own sampling error
    (5 standard errors over 256 probes)."""
    s, op, c = small
    dim = c.shape[0]
    q, _, _, _ = slq(op, dim, 256, 20, seed=99)
    est = dim * q
    e_ref = dense_energy(c, s.omega)
    e = 0.5 * est.mean() - 1.5 * np.sum(s.omega)
    sem = 0.5 * est.std(ddof=1) / np.sqrt(est.size)
    assert abs(e - e_ref) < 5 * sem
    e2, info = slq_energy(op, 256, 20, seed=99)
    assert abs(e2 - e) < 1e-13
