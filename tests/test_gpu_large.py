"""GPU parity at the full workload sizes: the 24,000-atom water box (mesh
128^3, 128 probes x 60 steps, the FP32/FP64 batched form), the 12,000-atom box
(mesh 96^3) used for the force checks, and the 100,002-atom box (mesh 192^3).
The oracle computes whole operator products at these sizes; Lanczos and force
outputs are compared on sampled probes (the oracle runs only those probes)."""
import numpy as np
import pytest
import torch

from oracle.forces import estimator_forces
from oracle.lanczos import lanczos, normalised_probes, slq
from oracle.operator import Operator
from _parity import atom_max, close, rel
from workloads.systems import config

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _t(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")




@pytest.fixture(scope="module")
def water24k():
    s = config(3)
    return s, Operator(s, "spme")


def test_water24000_operator(mbd, water24k):
    s, op = water24k
    x = np.random.default_rng(30).normal(size=(2, 3 * s.n_atoms))
    ref = op(x)
    y64 = mbd.MBDSystem.from_workload(s, precision="fp64").apply_C(_t(x)).cpu().numpy()
    close(y64, ref, 1e-11)
    y32 = mbd.MBDSystem.from_workload(s, precision="mixed").apply_C(_t(x)).cpu().numpy()
    close(y32, ref, 2e-6)


def test_water24000_lanczos_sampled(mbd, water24k):
    """The full launch (128 probes x 60 steps) on both paths; probe 0's first
    8 coefficients against the oracle's recurrence for that probe alone; the
    mixed energy within 1e-5 of the FP64 energy."""
    s, op = water24k
    e64, d64 = mbd.MBDSystem.from_workload(s, precision="fp64").lanczos_energy(
        s.n_probes, s.n_steps, s.probe_seed, details=True)
    e32, d32 = mbd.MBDSystem.from_workload(s, precision="mixed").lanczos_energy(
        s.n_probes, s.n_steps, s.probe_seed, details=True)
    v = normalised_probes(s.probe_seed, 1, 3 * s.n_atoms)
    a, b, _, _ = lanczos(op, v, 8)
    np.testing.assert_allclose(d64["a"][0, :8], a[0], rtol=1e-10)
    np.testing.assert_allclose(d64["b"][0, :7], b[0, :7], rtol=1e-10)
    np.testing.assert_allclose(d32["a"][0, :8], a[0], rtol=2e-6)
    assert abs(e32 - e64) <= 1e-5 * abs(e64)


def test_water12000_forces_sampled(mbd):
    """Force estimator on the 12,000-atom box against the oracle's estimator on
    the same 4 probes (12 steps), FP64 path; mixed path within 1e-4."""
    s = config(5, "fd")
    op = Operator(s, "spme")
    f_ref, e_ref, _ = estimator_forces(op, 4, 12, s.probe_seed)
    e, f = mbd.MBDSystem.from_workload(s, precision="fp64").energy_forces(4, 12, s.probe_seed)
    f = f.cpu().numpy()
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
    assert np.abs(f - f_ref).max() <= 1e-8 * np.abs(f_ref).max()
    e32, f32 = mbd.MBDSystem.from_workload(s, precision="mixed").energy_forces(4, 12, s.probe_seed)
    assert np.abs(f32.cpu().numpy() - f_ref).max() <= 1e-4 * np.abs(f_ref).max()


def test_water100k_operator_and_energy(mbd):
    s = config(5)
    op = Operator(s, "spme")
    x = np.random.default_rng(31).normal(size=(1, 3 * s.n_atoms))
    ref = op(x)
    g32 = mbd.MBDSystem.from_workload(s, precision="mixed")
    y = g32.apply_C(_t(x)).cpu().numpy()
    close(y, ref, 2e-6)
    g64 = mbd.MBDSystem.from_workload(s, precision="fp64")
    close(g64.apply_C(_t(x)).cpu().numpy(), ref, 1e-11)
    e32, d32 = g32.lanczos_energy(s.n_probes, s.n_steps, s.probe_seed, details=True)
    e64 = g64.lanczos_energy(s.n_probes, s.n_steps, s.probe_seed)
    assert abs(e32 - e64) <= 1e-5 * abs(e64)
    q_ref, _, _, _ = slq(op, 3 * s.n_atoms, 1, 6, s.probe_seed)
    _, d6 = g64.lanczos_energy(1, 6, s.probe_seed, details=True)
    np.testing.assert_allclose(d6["q"], q_ref, rtol=1e-8)
