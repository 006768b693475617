"""Degenerate and boundary cases through the C ABI, against the oracle: one
and two atoms per cell, a single probe, a single Lanczos step, the Krylov
space exhausted before m (every probe breaks down), the smallest mesh the
spline order allows (K = 2p, generic FFT pass) and spline order 4."""
import numpy as np
import pytest
import torch

from oracle.dense import dense_energy
from oracle.forces import estimator_forces
from oracle.lanczos import slq
from oracle.operator import Operator
from _parity import atom_max, close, rel
from workloads.systems import System, random_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _one_atom():
    return System("one", np.eye(3) * 12.0, np.array([[1.3, 2.2, 5.1]]), np.array([8.0]), np.array([0.5]),
                  np.array([3.5]), r_cut=5.9, damp_cut=5.9, mesh=(16, 16, 16))


def _two_atoms():
    return System("two", np.eye(3) * 11.0, np.array([[0.7, 0.2, 0.1], [4.7, 5.2, 6.1]]), np.array([9.0, 6.0]),
                  np.array([0.45, 0.5]), np.array([3.3, 3.1]), r_cut=5.4, damp_cut=5.4, mesh=(16, 16, 16))




@pytest.mark.parametrize("make", [_one_atom, _two_atoms], ids=["one_atom", "two_atoms"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tiny_cells(mbd, make, precision):
    """One or two atoms per cell (3N = 3 or 6, self-images only through the
    reciprocal sum): C x, the quadratures with m = 3N and the forces against
    the oracle."""
    s = make()
    g = mbd.MBDSystem.from_workload(s, precision=precision)
    op = Operator(s, "spme")
    x = np.random.default_rng(0).normal(size=(2, 3 * s.n_atoms))
    tol = 1e-11 if precision == "fp64" else 2e-6
    close(g.apply_C(torch.tensor(x, device="cuda")).cpu().numpy(), op(x), tol)
    m = 3 * s.n_atoms
    e, det = g.lanczos_energy(4, m, 77, details=True)
    q_ref, _, _, _ = slq(op, 3 * s.n_atoms, 4, m, 77)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8 if precision == "fp64" else 1e-5)
    e2, f = g.energy_forces(4, m, 77)
    f_ref, _, _ = estimator_forces(op, 4, m, 77)
    df = np.abs(f.cpu().numpy() - f_ref).max()
    if s.n_atoms == 1:
        # one atom moves with all its images: the force vanishes up to the mesh
        # error of SPME; compare absolutely (FP32 operator: a few 1e-8 Ha/bohr)
        assert np.abs(f_ref).max() < 1e-4
        assert df <= (1e-12 if precision == "fp64" else 1e-6)
    else:
        assert df <= (1e-8 if precision == "fp64" else 1e-4) * np.abs(f_ref).max()


def test_single_probe_single_step(mbd):
    s = random_system(24, 12.0, 4242, mesh=(16, 16, 16), r_cut=5.9, damp_cut=5.9)
    g = mbd.MBDSystem.from_workload(s)
    op = Operator(s, "spme")
    for R, m in ((1, 1), (1, 7), (3, 1)):
        e, det = g.lanczos_energy(R, m, 11, details=True)
        q_ref, _, _, _ = slq(op, 3 * s.n_atoms, R, m, 11)
        np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8)
        e2, f = g.energy_forces(R, m, 11)
        f_ref, _, _ = estimator_forces(op, R, m, 11)
        assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-8 * np.abs(f_ref).max()


@pytest.mark.parametrize("p,K", [(6, 12), (4, 8), (4, 15)])
def test_smallest_meshes(mbd, p, K):
    """K = 2p (the smallest accepted) and an odd smooth size below 16 use the
    generic FFT pass and the generic spreading."""
    s = random_system(24, 12.0, 4242, mesh=(K, K, K), r_cut=5.9, damp_cut=5.9).with_(spline_order=p)
    g = mbd.MBDSystem.from_workload(s)
    op = Operator(s, "spme")
    x = np.random.default_rng(1).normal(size=(3, 3 * s.n_atoms))
    close(g.apply_C(torch.tensor(x, device="cuda")).cpu().numpy(), op(x), 1e-11)
    e, det = g.lanczos_energy(32, 6, 5, details=True)
    q_ref, _, _, _ = slq(op, 3 * s.n_atoms, 32, 6, 5)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8)


def test_breakdown_beyond_krylov_dimension(mbd):
    """Two atoms, m = 10 > 3N = 6: past the Krylov dimension the recurrence
    either breaks down (b_k <= 1e-14 |a_1|) or, without reorthogonalisation,
    continues with copies of converged Ritz values; either way the quadrature
    is exact: v^T C^{1/2} v from the eigendecomposition of the dense C."""
    from oracle.lanczos import normalised_probes
    s = _two_atoms()
    c = Operator(s, "spme").dense()
    lam, u = np.linalg.eigh(0.5 * (c + c.T))
    g = mbd.MBDSystem.from_workload(s)
    _, det = g.lanczos_energy(3, 10, 123, details=True)
    v = normalised_probes(123, 3, 6)
    exact = np.einsum("li,ij,lj->l", v, (u * np.sqrt(lam)) @ u.T, v)
    np.testing.assert_allclose(det["q"], exact, rtol=1e-10)
    assert np.isfinite(dense_energy(c, s.omega))
