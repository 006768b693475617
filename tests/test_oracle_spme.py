"""Pins for oracle/spme.py: convergence to the direct Ewald sum, adjointness,
the FFT convolution against a brute-force circular convolution, and the
paper's observation that Delta_11 converges monotonically with the mesh."""
import numpy as np
import pytest

from oracle.ewald import apply_T, reciprocal_field_direct
from oracle.lanczos import normalised_probes
from oracle.operator import Operator
from oracle.spme import convolve, gather, influence_function, reciprocal_field_spme, spread, stencil
from workloads.systems import System, config, random_system


def _small(k=16):
    return random_system(12, 11.0, 77, mesh=(k, k, k), r_cut=5.4, damp_cut=5.4)


def test_spme_converges_to_direct_reciprocal():
    """SPME reciprocal field -> direct Ewald reciprocal field as the mesh is refined."""
    s = _small()
    d = np.random.default_rng(0).normal(size=(2, s.n_atoms, 3))
    ref = reciprocal_field_direct(s, d)
    err = []
    for k in (12, 16, 24, 36):
        e = reciprocal_field_spme(s.with_(mesh=(k, k, k)), d)
        err.append(np.linalg.norm(e - ref) / np.linalg.norm(ref))
    assert all(a > b for a, b in zip(err, err[1:])), err
    assert err[-1] < 1e-5


def test_spme_skew_cell_converges():
    cell = np.array([[11.0, 0.0, 0.0], [1.5, 10.5, 0.0], [-0.8, 1.2, 11.5]])
    base = _small()
    s = base.with_(cell=cell, pos=base.pos @ np.linalg.inv(np.eye(3) * 11.0) @ cell)
    d = np.random.default_rng(1).normal(size=(2, s.n_atoms, 3))
    ref = reciprocal_field_direct(s, d)
    e = reciprocal_field_spme(s.with_(mesh=(40, 40, 40)), d)
    assert np.linalg.norm(e - ref) / np.linalg.norm(ref) < 1e-5


def test_c_x_error_at_configured_mesh():
    """C x with SPME vs direct Ewald at the same split, 64-atom box at mesh 32^3,
    order 6: relative L2 error <= 1e-5."""
    s = config(1)
    x = np.random.default_rng(0).normal(size=(2, 3 * s.n_atoms))
    ys = Operator(s, "spme")(x)
    yd = Operator(s, "same_split")(x)
    assert np.linalg.norm(ys - yd) / np.linalg.norm(yd) <= 1e-5


def _atom_max(a, b):
    """Largest per-atom error |a_i - b_i| over the RMS per-atom norm of b, for
    arrays [..., N, 3]: a large error on one atom that a whole-array norm
    would dilute shows here."""
    a, b = np.asarray(a).reshape(-1, 3), np.asarray(b).reshape(-1, 3)
    return np.linalg.norm(a - b, axis=1).max() / np.sqrt(np.mean(np.sum(b * b, axis=1)))


@pytest.mark.slow
def test_c_x_error_water3000():
    """The same bound on the 3000-atom water box (mesh 64^3, order 6, its
    configured split beta = 0.30, r_cut = 12): SPME C x within 1e-5 (relative
    L2) of the same-split direct Ewald sum, and no atom off by more than 3e-5
    of the RMS atom norm."""
    s = config(2)
    op = Operator(s, "spme")
    x = np.random.default_rng(8).normal(size=(1, 3 * s.n_atoms))
    ys = op(x)
    d = (x * op.g).reshape(1, s.n_atoms, 3)
    e = apply_T(s, d, "same_split", real_matrix=op.real).reshape(1, -1)
    yd = op.w2 * x + op.g * e
    assert np.linalg.norm(ys - yd) / np.linalg.norm(yd) <= 1e-5
    assert _atom_max(ys, yd) <= 3e-5


def test_spread_gather_adjoint():
    s = _small()
    rng = np.random.default_rng(5)
    d = rng.normal(size=(1, s.n_atoms, 3))
    phi = rng.normal(size=(1,) + s.mesh)
    st = stencil(s)
    lhs = np.sum(spread(s, d, st) * phi)
    rhs = np.sum(d * gather(s, phi, st))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_spread_total_is_zero():
    """sum_k grad W_j(k) = grad sum_k W_j(k) = grad 1 = 0 (partition of unity)."""
    s = _small()
    d = np.random.default_rng(6).normal(size=(2, s.n_atoms, 3))
    q = spread(s, d)
    assert np.abs(q.sum(axis=(1, 2, 3))).max() < 1e-12 * np.abs(q).max()


def test_convolution_brute_force():
    """F^-1[G F[Q]] equals the circular convolution with the kernel whose DFT is G."""
    s = _small(k=8).with_(mesh=(6, 8, 5))
    g = np.random.default_rng(7).uniform(size=s.mesh)
    g = 0.5 * (g + g[np.ix_(*[(-np.arange(k)) % k for k in s.mesh])])
    kernel = np.real(np.fft.ifftn(g))        # Phi(c) = (1/K^3) sum_m G e^{+2 pi i m.c/K}
    q = np.random.default_rng(8).normal(size=(1,) + s.mesh)
    brute = np.zeros(s.mesh)
    for a in np.ndindex(*s.mesh):
        for b in np.ndindex(*s.mesh):
            c = tuple((np.array(a) - np.array(b)) % np.array(s.mesh))
            brute[a] += kernel[c] * q[0][b]
    # the SPME convention folds the 1/K^3 into nothing: phi = K^3 * (Phi * Q)
    np.testing.assert_allclose(convolve(s, q, g)[0], brute * np.prod(s.mesh), rtol=1e-12, atol=1e-12)


def test_influence_function_properties():
    s = config(1)
    g = influence_function(s)
    assert g[0, 0, 0] == 0.0 and np.all(g >= 0.0)
    gneg = g[np.ix_(*[(-np.arange(k)) % k for k in s.mesh])]
    np.testing.assert_array_equal(g, gneg)


def test_single_atom_spme_mesh_error():
    """The single-atom closed form -(4 pi/3V) I holds for SPME to mesh error at
    any position; the error falls with the mesh."""
    err = []
    for k in (16, 24, 32):
        s = System("one", np.eye(3) * 12.0, np.array([[1.3, 2.2, 5.1]]), np.array([8.0]),
                   np.array([0.5]), np.array([3.5]), r_cut=5.9, damp_cut=5.9, mesh=(k, k, k))
        e = apply_T(s, np.eye(3)[:, None, :], "spme")[:, 0, :]
        ref = -4 * np.pi / (3 * 12.0 ** 3) * np.eye(3)
        err.append(np.abs(e - ref).max() / abs(ref[0, 0]))
    assert err[0] > err[1] > err[2] and err[2] < 1e-5


def test_delta11_monotone_in_mesh():
    """Numerical results section: Delta_11 = v^T C v for a fixed probe converges
    monotonically as the mesh is refined (no oscillation, unlike the replica sum)."""
    s = config(1)
    v = normalised_probes(s.probe_seed, 1, 3 * s.n_atoms)[0]
    vals = [float(v @ Operator(s.with_(mesh=(k, k, k)), "spme")(v)) for k in (12, 16, 20, 24, 32, 40)]
    assert all(b > a for a, b in zip(vals, vals[1:])), vals
