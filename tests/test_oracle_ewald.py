"""Pins for oracle/ewald.py (direct Ewald, tin-foil) and oracle/replica.py."""
import numpy as np
import pytest

from oracle.ewald import (apply_T, pair_list, pair_list_tree, real_space_tensor, real_space_tensor_grad,
                          reciprocal_field_direct)
from oracle.model import cell_volume
from oracle.operator import Operator
from oracle.replica import replica_field
from workloads.systems import System, random_system


def _one_atom(pos, box=12.0, beta=0.35):
    return System("one", np.eye(3) * box, np.array([pos]), np.array([8.0]), np.array([0.5]),
                  np.array([3.5]), ewald_beta=beta, r_cut=5.9, damp_cut=5.9, mesh=(16, 16, 16))


@pytest.mark.parametrize("beta", [0.25, 0.35, 0.5])
@pytest.mark.parametrize("pos", [(0.0, 0.0, 0.0), (1.3, 2.2, 5.1), (11.9, 6.0, 0.4)])
def test_single_atom_cubic(beta, pos):
    """One atom in a cubic cell: every shell of the lattice sum of a traceless
    (damped) T cancels by cubic symmetry, so in tin-foil conditions
    T'^pbc = -(4 pi / 3V) I, whatever beta and the damping."""
    s = _one_atom(pos, beta=beta)
    e = apply_T(s, np.eye(3)[:, None, :], "exact")[:, 0, :]
    np.testing.assert_allclose(e, -4 * np.pi / (3 * 12.0 ** 3) * np.eye(3), rtol=1e-12, atol=1e-17)


def test_bcc_pair_eigenvalues():
    """Two identical atoms at 0 and (L/2)(1,1,1): uniform polarisation of the bcc
    lattice gives -(8 pi / 3V), the antisymmetric mode 0, so C has eigenvalues
    w^2 (1 - 8 pi alpha / 3V) (x3) and w^2 (x3)."""
    box, w, a = 10.0, 0.45, 9.0
    s = System("bcc", np.eye(3) * box, np.array([[0.7, 0.2, 0.1], [5.7, 5.2, 5.1]]),
               np.array([a, a]), np.array([w, w]), np.array([3.3, 3.3]), r_cut=4.9, damp_cut=4.9)
    lam = np.sort(np.linalg.eigvalsh(Operator(s, "exact").dense()))
    ref = np.sort([w * w * (1 - 8 * np.pi * a / (3 * box ** 3))] * 3 + [w * w] * 3)
    np.testing.assert_allclose(lam, ref, rtol=1e-12)


def _small():
    return random_system(12, 11.0, 77, mesh=(16, 16, 16), r_cut=5.4, damp_cut=5.4)


def test_beta_invariance():
    """The exact T'^pbc d does not depend on the Ewald splitting parameter."""
    s = _small()
    d = np.random.default_rng(0).normal(size=(3, s.n_atoms, 3))
    ref = apply_T(s, d, "exact")
    for beta in (0.25, 0.5, 0.7):
        e = apply_T(s.with_(ewald_beta=beta), d, "exact")
        assert np.linalg.norm(e - ref) / np.linalg.norm(ref) < 1e-12


def test_replica_limit():
    """Growing spheres of replica cells (Eq. replica) tend to the tin-foil Ewald
    field plus the surface term (4 pi / 3V) sum_j d_j on every atom."""
    s = System("tri", np.eye(3) * 9.0, np.array([[0.3, 1.1, 2.0], [4.1, 5.3, 2.2], [7.0, 3.5, 8.1]]),
               np.array([6., 8., 10.]), np.array([.4, .5, .6]), np.array([3.1, 3.5, 3.3]))
    d = np.random.default_rng(1).normal(size=(2, 3, 3))
    ew = apply_T(s, d, "exact") + 4 * np.pi / (3 * cell_volume(s.cell)) * d.sum(axis=1, keepdims=True)
    err = [np.linalg.norm(replica_field(s, d, rc) - ew) / np.linalg.norm(ew) for rc in (90.0, 180.0, 360.0)]
    assert err[0] > err[1] > err[2] and err[2] < 5e-6


def test_dense_symmetric_and_reciprocal_psd():
    s = _small()
    c = Operator(s, "exact").dense()
    assert np.abs(c - c.T).max() < 1e-14 * np.abs(c).max()
    d = np.random.default_rng(2).normal(size=(5, s.n_atoms, 3))
    e = reciprocal_field_direct(s, d)
    assert np.all(np.einsum("vna,vna->v", d, e) >= 0.0)


def test_lattice_and_translation_invariance():
    s = _small()
    d = np.random.default_rng(4).normal(size=(2, s.n_atoms, 3))
    ref = apply_T(s, d, "exact")
    pos = s.pos.copy()
    pos[3] += s.cell[1] - 2 * s.cell[2]
    np.testing.assert_allclose(apply_T(s.with_(pos=pos), d, "exact"), ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    e2 = apply_T(s.with_(pos=s.pos + np.array([0.37, -1.3, 2.9])), d, "exact")
    np.testing.assert_allclose(e2, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_pair_list_brute_force():
    """Every (i, j, n) within the cutoff appears once; count against an explicit loop."""
    s = _small()
    i, j, r = pair_list(s.cell, s.pos, 8.0)
    cnt = 0
    pos = np.mod(s.pos, 11.0)
    for a in range(s.n_atoms):
        for b in range(s.n_atoms):
            for n in np.ndindex(5, 5, 5):
                rv = pos[a] - pos[b] - (np.array(n) - 2) * 11.0
                rr = np.linalg.norm(rv)
                cnt += (0 < rr < 8.0)
    assert cnt == i.size
    assert np.all(np.linalg.norm(r, axis=1) < 8.0)


def test_real_space_tensor_grad_fd():
    s = _small()
    i, j, r = pair_list(s.cell, s.pos, 6.0)
    g = real_space_tensor_grad(s, i, j, r, 5.4, 5.8)
    h = 1e-6
    inside = (np.abs(np.linalg.norm(r, axis=1) - 5.4) > 1e-3) & (np.abs(np.linalg.norm(r, axis=1) - 5.8) > 1e-3)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (real_space_tensor(s, i, j, r + e, 5.4, 5.8) - real_space_tensor(s, i, j, r - e, 5.4, 5.8)) / (2 * h)
        np.testing.assert_allclose(g[inside, ..., c], fd[inside], rtol=1e-5, atol=1e-10)


@pytest.mark.parametrize("n,box,rmax", [(40, 22.0, 10.0), (300, 30.0, 7.0)])
def test_pair_list_tree_matches_brute_force(n, box, rmax):
    """The k-d tree pair search returns exactly the brute-force pair set."""
    s = random_system(n, box, 91 + n, mesh=(24, 24, 24))
    i, j, r = pair_list(s.cell, s.pos, rmax)
    i2, j2, r2 = pair_list_tree(s.cell, s.pos, rmax)
    a = sorted(zip(i.tolist(), j.tolist(), np.round(r, 9).tolist()))
    b = sorted(zip(i2.tolist(), j2.tolist(), np.round(r2, 9).tolist()))
    assert a == b
