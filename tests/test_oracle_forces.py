"""Pins for oracle/forces.py and the dense gradient of oracle/dense.py against
central finite differences, momentum conservation and the exact-trace limit."""
import numpy as np
import pytest

from oracle.dense import dense_energy, dense_gradient
from oracle.ewald import apply_T
from oracle.forces import bilinear_gradient, estimator_forces
from oracle.lanczos import inverse_sqrt_action, lanczos
from oracle.operator import Operator
from workloads.systems import random_system


def _sys():
    return random_system(10, 10.5, 21, mesh=(16, 16, 16), r_cut=5.2, damp_cut=5.2)


@pytest.mark.parametrize("mode", ["spme", "exact"])
def test_dense_gradient_fd(mode):
    """dE/dR = (1/4) Tr(C^-1/2 dC/dR) against central differences (h = 1e-4 bohr)."""
    s = _sys()
    op = Operator(s, mode)
    g = dense_gradient(op)
    h = 1e-4
    for i, c in [(0, 0), (4, 1), (9, 2)]:
        e = []
        for sgn in (1.0, -1.0):
            p = s.pos.copy()
            p[i, c] += sgn * h
            e.append(dense_energy(Operator(s.with_(pos=p), mode).dense(), s.omega))
        assert abs((e[0] - e[1]) / (2 * h) - g[i, c]) < 1e-8


def test_exact_gradient_sums_to_zero():
    g = dense_gradient(Operator(_sys(), "exact"))
    assert np.abs(g.sum(axis=0)).max() < 1e-14


@pytest.mark.parametrize("mode", ["spme", "same_split"])
def test_bilinear_gradient_fd(mode):
    s = _sys()
    rng = np.random.default_rng(3)
    p = rng.normal(size=(2, s.n_atoms, 3))
    q = rng.normal(size=(2, s.n_atoms, 3))
    g = bilinear_gradient(s, p, q, mode)
    h = 1e-5
    for i, c in [(1, 0), (6, 2)]:
        val = []
        for sgn in (1.0, -1.0):
            pos = s.pos.copy()
            pos[i, c] += sgn * h
            val.append(np.sum(p * apply_T(s.with_(pos=pos), q, mode)))
        fd = (val[0] - val[1]) / (2 * h)
        assert abs(fd - g[i, c]) < 1e-7 * max(1.0, abs(fd))


def test_estimator_exact_with_unit_probes():
    """With the D unit vectors as probes and full Krylov the estimator equals
    the dense gradient."""
    s = _sys()
    op = Operator(s, "spme")
    dim = 3 * s.n_atoms
    v = np.eye(dim)
    a, b, length, y = lanczos(op, v, dim, reorth=True, keep_basis=True)
    w = np.stack([inverse_sqrt_action(a[l], b[l], length[l], y[l]) for l in range(dim)])
    est = 0.25 * bilinear_gradient(s, (w * op.g).reshape(dim, -1, 3), (v * op.g).reshape(dim, -1, 3), "spme")
    ref = dense_gradient(op)
    assert np.abs(est - ref).max() < 1e-12 * np.abs(ref).max()


def test_estimator_forces_runs():
    s = _sys()
    op = Operator(s, "spme")
    f, e, info = estimator_forces(op, 8, 12, seed=5)
    assert f.shape == (s.n_atoms, 3) and np.isfinite(f).all() and np.isfinite(e)
