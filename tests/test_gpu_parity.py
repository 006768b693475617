"""GPU parity: every stage of the CUDA path against the FP64 oracle on the same
seeded inputs, through the C ABI.

Tolerances (FP64 path): stages and C x to 1e-11 relative L2 (different but
exact-arithmetic-equivalent summation orders and FFT algorithms); Lanczos
energies and per-probe quadratures to 1e-8 relative on identical probes;
forces (same estimator, same probes) to 1e-8 of the largest component.
Mixed path (FP32 operator): energy within 1e-5 relative of the FP64 path.
"""
import numpy as np
import pytest
import torch

from oracle import spme as ospme
from oracle.ewald import apply_T, real_space_matrix, self_coefficient
from oracle.forces import estimator_forces
from oracle.lanczos import lanczos, normalised_probes, quadrature, slq, slq_energy
from oracle.operator import Operator
from _parity import atom_max, close, rel
from workloads.systems import System, config, random_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _small(mesh=(16, 16, 16), n=24, box=12.0, seed=4242):
    return random_system(n, box, seed, mesh=mesh, r_cut=5.9, damp_cut=5.9)


def _skew(mesh=(16, 18, 20)):
    cell = np.array([[12.0, 0.0, 0.0], [1.5, 11.5, 0.0], [-0.8, 1.2, 12.5]])
    base = _small()
    frac = base.pos / 12.0
    return base.with_(cell=cell, pos=frac @ cell, mesh=mesh, r_cut=5.4, damp_cut=5.4)




def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


# ------------------------------------------------------------------ a1 probes
@pytest.mark.parametrize("first,R,dim", [(0, 5, 7), (3, 16, 192), (0, 1, 9000)])
def test_probes_bit_exact(mbd, first, R, dim):
    v = mbd.generate_probes(2307022781, R, dim, first=first).cpu().numpy()
    ref = normalised_probes(2307022781, R, dim, first=first)
    np.testing.assert_array_equal(v, ref)


# ------------------------------------------------------------------ a11 quadrature
def test_tridiag_quadrature(mbd):
    s = _small()
    op = Operator(s, "spme")
    v = normalised_probes(9, 7, 3 * s.n_atoms)
    a, b, length, _ = lanczos(op, v, 20)
    q = mbd.tridiag_quadrature(a, b)
    ref = np.array([quadrature(a[l], b[l], length[l]) for l in range(7)])
    np.testing.assert_allclose(q, ref, rtol=1e-13)
    # a zero coupling truncates the tridiagonal (breakdown)
    a2 = np.array([[4.0, 9.0, 1.0]])
    b2 = np.array([[0.0, 0.5, 0.0]])
    np.testing.assert_allclose(mbd.tridiag_quadrature(a2, b2), [2.0], rtol=1e-15)


def test_tridiag_not_positive_definite(mbd):
    with pytest.raises(mbd.MBDError) as e:
        mbd.tridiag_quadrature(np.array([[1.0, -3.0]]), np.array([[0.1, 0.0]]))
    assert e.value.code == 4


# ------------------------------------------------------------------ a3/a4 spreading
@pytest.mark.parametrize("which", ["cubic", "skew", "mesh30"])
def test_spread_parity(mbd, which):
    s = {"cubic": _small(), "skew": _skew(), "mesh30": _small(mesh=(30, 24, 20))}[which]
    g = mbd.MBDSystem.from_workload(s)
    d = np.random.default_rng(1).normal(size=(3, s.n_atoms, 3))
    q = g.spread(_t(d), s.mesh).cpu().numpy()
    ref = ospme.spread(s, d)
    close(q, ref, 1e-13, width=1)


# ------------------------------------------------------------------ a5-a7 FFT convolution
@pytest.mark.parametrize("mesh", [(16, 16, 16), (16, 18, 20), (24, 30, 32), (40, 12, 48)])
def test_convolve_parity(mbd, mesh):
    s = _small(mesh=mesh)
    g = mbd.MBDSystem.from_workload(s)
    q = np.random.default_rng(2).normal(size=(5,) + mesh)
    phi = g.convolve(_t(q)).cpu().numpy()
    ref = ospme.convolve(s, q)
    close(phi, ref, 1e-12, width=1)


# ------------------------------------------------------------------ a8-a10 field terms
@pytest.mark.parametrize("which", ["cubic", "skew"])
def test_field_terms(mbd, which):
    s = _small() if which == "cubic" else _skew()
    g = mbd.MBDSystem.from_workload(s)
    d = np.random.default_rng(3).normal(size=(3, s.n_atoms, 3))
    real = (real_space_matrix(s, "same_split") @ d.reshape(3, -1).T).T.reshape(d.shape)
    rec = ospme.reciprocal_field_spme(s, d)
    slf = self_coefficient(s.ewald_beta) * d
    for terms, ref in [(mbd.MBD_TERM_REAL, real), (mbd.MBD_TERM_RECIP, rec), (mbd.MBD_TERM_SELF, slf),
                       (mbd.MBD_TERM_ALL, real + rec + slf)]:
        e = g.field(_t(d), terms).cpu().numpy()
        close(e, ref, 1e-11)


# ------------------------------------------------------------------ operator C x
@pytest.mark.parametrize("which", ["c1", "skew", "single_atom"])
def test_apply_C_parity(mbd, which):
    if which == "c1":
        s = config(1)
    elif which == "skew":
        s = _skew()
    else:
        s = System("one", np.eye(3) * 12.0, np.array([[1.3, 2.2, 5.1]]), np.array([8.0]), np.array([0.5]),
                   np.array([3.5]), r_cut=5.9, damp_cut=5.9, mesh=(16, 16, 16))
    g = mbd.MBDSystem.from_workload(s)
    x = np.random.default_rng(4).normal(size=(5, 3 * s.n_atoms))
    y = g.apply_C(_t(x)).cpu().numpy()
    close(y, Operator(s, "spme")(x), 1e-11)
    if which == "c1":
        # the operator bound: SPME C x vs direct Ewald at the same split; on
        # 64 atoms the largest atom error is 3.1e-5 of the RMS atom norm
        close(y, Operator(s, "same_split")(x), 1e-5, atom_factor=5.0)


# ------------------------------------------------------------------ Lanczos energy (a1-a11)
def test_lanczos_energy_c1(mbd):
    s = config(1)
    g = mbd.MBDSystem.from_workload(s)
    e, det = g.lanczos_energy(s.n_probes, s.n_steps, s.probe_seed, details=True)
    op = Operator(s, "spme")
    e_ref, info = slq_energy(op, s.n_probes, s.n_steps, s.probe_seed)
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
    np.testing.assert_allclose(det["q"], info["q"], rtol=1e-8)
    np.testing.assert_allclose(det["a"][:, :10], info["a"][:, :10], rtol=1e-10)
    np.testing.assert_allclose(det["b"][:, :9], info["b"][:, :9], rtol=1e-10)


@pytest.mark.parametrize("R,m", [(1, 1), (1, 7), (33, 12), (2, 40)])
def test_lanczos_ragged_sizes(mbd, R, m):
    s = _small()
    g = mbd.MBDSystem.from_workload(s)
    e, det = g.lanczos_energy(R, m, 77, details=True)
    q_ref, a_ref, b_ref, length = slq(Operator(s, "spme"), 3 * s.n_atoms, R, m, 77)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8)
    if m == 1:
        np.testing.assert_allclose(det["q"], np.sqrt(a_ref[:, 0]), rtol=1e-13)


def test_dense_lanczos_layer(mbd):
    """The Lanczos layer alone on a dense operator: same recurrence as the oracle."""
    s = random_system(16, 14.0, 5, mesh=(20, 20, 20), r_cut=6.9, damp_cut=6.9)
    op = Operator(s, "spme")
    c = op.dense()
    c = 0.5 * (c + c.T)
    dim = c.shape[0]
    e, det = mbd.lanczos_energy_dense(_t(c), float(np.sum(s.omega)), 9, 20, 123)
    q_ref, a_ref, b_ref, _ = slq(lambda x: x @ c, dim, 9, 20, 123)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-10)
    np.testing.assert_allclose(det["a"], a_ref, rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------ mixed precision
def test_mixed_precision_energy_c1(mbd):
    s = config(1)
    e64 = mbd.MBDSystem.from_workload(s, precision="fp64").lanczos_energy(s.n_probes, s.n_steps, s.probe_seed)
    e32 = mbd.MBDSystem.from_workload(s, precision="mixed").lanczos_energy(s.n_probes, s.n_steps, s.probe_seed)
    assert abs(e32 - e64) <= 1e-5 * abs(e64)
    x = np.random.default_rng(5).normal(size=(4, 3 * s.n_atoms))
    y32 = mbd.MBDSystem.from_workload(s, precision="mixed").apply_C(_t(x)).cpu().numpy()
    close(y32, Operator(s, "spme")(x), 1e-5)


# ------------------------------------------------------------------ a12 forces
def test_forces_parity(mbd):
    s = _small()
    g = mbd.MBDSystem.from_workload(s)
    R, m, seed = 6, 12, 31
    e, f = g.energy_forces(R, m, seed)
    f = f.cpu().numpy()
    f_ref, e_ref, _ = estimator_forces(Operator(s, "spme"), R, m, seed)
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
    assert np.abs(f - f_ref).max() <= 1e-8 * np.abs(f_ref).max()
    gm = mbd.MBDSystem.from_workload(s, precision="mixed")
    e32, f32 = gm.energy_forces(R, m, seed)
    assert np.abs(f32.cpu().numpy() - f_ref).max() <= 1e-4 * np.abs(f_ref).max()


def test_forces_skew(mbd):
    s = _skew()
    g = mbd.MBDSystem.from_workload(s)
    e, f = g.energy_forces(4, 10, 5)
    f_ref, e_ref, _ = estimator_forces(Operator(s, "spme"), 4, 10, 5)
    assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-8 * np.abs(f_ref).max()


def test_autograd_backward(mbd):
    s = _small()
    g = mbd.MBDSystem.from_workload(s)
    pos = torch.tensor(s.pos, dtype=torch.float64, requires_grad=True)
    e = mbd.mbd_energy(pos, g, 4, 10, 9)
    e.backward()
    _, f = g.energy_forces(4, 10, 9)
    np.testing.assert_allclose(pos.grad.numpy(), -f.cpu().numpy(), rtol=0, atol=1e-15)


# ------------------------------------------------------------------ geometry updates, errors
def test_update_positions(mbd):
    s = _small()
    g = mbd.MBDSystem.from_workload(s)
    pos2 = s.pos + np.random.default_rng(6).normal(scale=0.2, size=s.pos.shape)
    g.update_positions(pos2)
    x = np.random.default_rng(7).normal(size=(2, 3 * s.n_atoms))
    y = g.apply_C(_t(x)).cpu().numpy()
    close(y, Operator(s.with_(pos=pos2), "spme")(x), 1e-11)


def test_polarisation_catastrophe(mbd):
    s = _small()
    s = s.with_(alpha=s.alpha * 60.0)
    g = mbd.MBDSystem.from_workload(s)
    with pytest.raises(mbd.MBDError) as e:
        g.lanczos_energy(4, 20, 1)
    assert e.value.code == 4


# ------------------------------------------------------------------ 3000-atom water box, sampled
@pytest.mark.slow
def test_water3000_sampled(mbd):
    s = config(2)
    g = mbd.MBDSystem.from_workload(s)
    op = Operator(s, "spme")
    x = np.random.default_rng(8).normal(size=(2, 3 * s.n_atoms))
    close(g.apply_C(_t(x)).cpu().numpy(), op(x), 1e-11)
    e, det = g.lanczos_energy(s.n_probes, s.n_steps, s.probe_seed, details=True)
    q_ref, _, _, _ = slq(op, 3 * s.n_atoms, 3, s.n_steps, s.probe_seed)
    np.testing.assert_allclose(det["q"][:3], q_ref, rtol=1e-8)
    em = mbd.MBDSystem.from_workload(s, precision="mixed").lanczos_energy(s.n_probes, s.n_steps, s.probe_seed)
    assert abs(em - e) <= 1e-5 * abs(e)


# ------------------------------------------------------------------ kernel variants
@pytest.mark.parametrize("p", [4, 8])
@pytest.mark.parametrize("nvec", [3, 64, 128])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_C_orders_and_widths(mbd, p, nvec, precision):
    """Spline orders other than 6 and probe blocks of 1, 2 and 4 probes per lane."""
    s = _small(mesh=(20, 16, 18)).with_(spline_order=p)
    g = mbd.MBDSystem.from_workload(s, precision=precision)
    x = np.random.default_rng(10 + p + nvec).normal(size=(nvec, 3 * s.n_atoms))
    y = g.apply_C(_t(x)).cpu().numpy()
    tol = 1e-11 if precision == "fp64" else 2e-6
    close(y, Operator(s, "spme")(x), tol)


@pytest.mark.parametrize("R", [64, 128, 5])
def test_lanczos_probe_widths(mbd, R):
    s = _small()
    e, det = mbd.MBDSystem.from_workload(s).lanczos_energy(R, 8, 1234, details=True)
    q_ref, _, _, _ = slq(Operator(s, "spme"), 3 * s.n_atoms, R, 8, 1234)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8)


@pytest.mark.parametrize("mesh", [(16, 20, 32), (12, 16, 64)])
@pytest.mark.parametrize("R", [32, 64, 128])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_spread_fft_path(mbd, mesh, R, precision):
    """Meshes whose k3 size has the fused spreading + first FFT pass (whole
    probe-pair tiles): Lanczos quadratures and forces against the oracle."""
    s = _small(mesh=mesh)
    g = mbd.MBDSystem.from_workload(s, precision=precision)
    e, det = g.lanczos_energy(R, 6, 4321, details=True)
    op = Operator(s, "spme")
    q_ref, _, _, _ = slq(op, 3 * s.n_atoms, R, 6, 4321)
    np.testing.assert_allclose(det["q"], q_ref, rtol=1e-8 if precision == "fp64" else 2e-6)
    if R == 32:
        e2, f = g.energy_forces(R, 6, 4321)
        f_ref, _, _ = estimator_forces(op, R, 6, 4321)
        tol = 1e-8 if precision == "fp64" else 1e-4
        assert np.abs(f.cpu().numpy() - f_ref).max() <= tol * np.abs(f_ref).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_df64_eigensolver_option(mbd, precision):
    """MBD_QUAD_QL_DF64 changes only the quadrature: identical Lanczos
    coefficients, quadratures within 1e-12 and forces within 1e-11 of FP64."""
    s = _small()
    g64 = mbd.MBDSystem.from_workload(s, precision=precision)
    gdf = mbd.MBDSystem.from_workload(s, precision=precision, quadrature="ql_df64")
    e1, d1 = g64.lanczos_energy(16, 30, 5, details=True)
    e2, d2 = gdf.lanczos_energy(16, 30, 5, details=True)
    np.testing.assert_array_equal(d2["a"], d1["a"])
    np.testing.assert_allclose(d2["q"], d1["q"], rtol=1e-12)
    _, f1 = g64.energy_forces(8, 20, 5)
    _, f2 = gdf.energy_forces(8, 20, 5)
    f1, f2 = f1.cpu().numpy(), f2.cpu().numpy()
    assert np.abs(f2 - f1).max() <= 1e-11 * np.abs(f1).max()


# ------------------------------------------------------------------ real space on clusters
@pytest.mark.parametrize("which", ["cubic", "skew", "c1"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_real_space_clusters(mbd, which, precision):
    """The real-space field evaluated on atom clusters (mbd_set_real_space_method)
    against the oracle and against the per-atom pair loop: the field's real
    term, C x and the Lanczos quadratures."""
    s = {"cubic": _small(), "skew": _skew(), "c1": config(1)}[which]
    tol = 1e-11 if precision == "fp64" else 2e-6
    gc = mbd.MBDSystem.from_workload(s, precision=precision)
    gc.set_real_space_method("clusters")
    gp = mbd.MBDSystem.from_workload(s, precision=precision)
    gp.set_real_space_method("pairs")
    d = np.random.default_rng(11).normal(size=(3, s.n_atoms, 3))
    real = (real_space_matrix(s, "same_split") @ d.reshape(3, -1).T).T.reshape(d.shape)
    close(gc.field(_t(d), mbd.MBD_TERM_REAL).cpu().numpy(), real, tol)
    x = np.random.default_rng(12).normal(size=(5, 3 * s.n_atoms))
    yc = gc.apply_C(_t(x)).cpu().numpy()
    close(yc, Operator(s, "spme")(x), tol)
    close(yc, gp.apply_C(_t(x)).cpu().numpy(), tol)
    _, dc = gc.lanczos_energy(8, 12, 99, details=True)
    _, dp = gp.lanczos_energy(8, 12, 99, details=True)
    np.testing.assert_allclose(dc["q"], dp["q"], rtol=1e-12 if precision == "fp64" else 2e-6)


@pytest.mark.parametrize("nvec", [64, 100])
def test_field_half_warp_atoms(mbd, nvec):
    """Mixed path with 64 to 127 probes on the clusters: the field kernel takes
    one atom per half-warp (four probes per lane); a ragged second chunk at
    100.  Against the oracle and against the pair loop (one atom per warp)."""
    s = config(1)
    gc = mbd.MBDSystem.from_workload(s, precision="mixed")
    gc.set_real_space_method("clusters")
    gp = mbd.MBDSystem.from_workload(s, precision="mixed")
    gp.set_real_space_method("pairs")
    x = np.random.default_rng(13).normal(size=(nvec, 3 * s.n_atoms))
    yc = gc.apply_C(_t(x)).cpu().numpy()
    close(yc, Operator(s, "spme")(x), 2e-6)
    close(yc, gp.apply_C(_t(x)).cpu().numpy(), 2e-6)
    _, dc = gc.lanczos_energy(nvec, 12, 7, details=True)
    _, dp = gp.lanczos_energy(nvec, 12, 7, details=True)
    np.testing.assert_allclose(dc["q"], dp["q"], rtol=2e-6)


def test_real_space_clusters_overflow_falls_back(mbd):
    """More than 256 neighbours per atom on average: the clusters are not built,
    asking for them is refused, and the pair loop gives the oracle's C x."""
    a, n = 2.6, 9                                       # 729 atoms on a jittered cubic lattice, L = 23.4
    grid = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * a
    pos = grid + np.random.default_rng(8).normal(scale=0.1, size=grid.shape)
    base = random_system(8, 10.0, 8)
    k = grid.shape[0]
    s = base.with_(cell=np.eye(3) * (n * a), pos=pos, alpha=np.full(k, 4.0), omega=np.full(k, 0.5),
                   r_vdw=np.full(k, 3.2), mesh=(24, 24, 24), r_cut=11.6, damp_cut=11.6)
    g = mbd.MBDSystem.from_workload(s)
    with pytest.raises(mbd.MBDError) as e:
        g.set_real_space_method("clusters")
    assert e.value.code == 7
    x = np.random.default_rng(13).normal(size=(2, 3 * s.n_atoms))
    close(g.apply_C(_t(x)).cpu().numpy(), Operator(s, "spme")(x), 1e-11)
