"""Error paths made on the host, with no GPU fault: a device allocation that
fails (mbd_debug_fail_allocation makes the library's allocator report
failure without calling cudaMalloc) and results that turn non-finite (a NaN in
the tridiagonal, a NaN in a dense operator, a polarisability that overflows
the FP32 operator).  Each call must return its status code, leave its outputs
untouched and leave the library usable for the next call."""
import ctypes

import numpy as np
import pytest
import torch

from workloads.systems import random_system

pytestmark = pytest.mark.gpu

OOM, NONFINITE = 2, 5


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def lib(mbd):
    from paper_2307_02278_gb300._abi import lib as load
    return load()


def _sys():
    return random_system(12, 11.0, 5, mesh=(16, 16, 16), r_cut=5.4, damp_cut=5.4)


def test_allocation_failure_during_create(mbd, lib):
    """Every device allocation of mbd_create_system failing in turn: each
    attempt returns MBD_ERR_OOM, and a system created afterwards gives the
    energy of one created before."""
    s = _sys()
    ref = mbd.MBDSystem.from_workload(s).lanczos_energy(8, 12, 3)
    failures = 0
    for k in range(200):
        lib.mbd_debug_fail_allocation(k)
        try:
            g = mbd.MBDSystem.from_workload(s)
        except mbd.MBDError as e:
            assert e.code == OOM
            failures += 1
            continue
        finally:
            lib.mbd_debug_fail_allocation(-1)
        g.close()
        break
    assert failures >= 5                      # creation allocates several buffers
    assert mbd.MBDSystem.from_workload(s).lanczos_energy(8, 12, 3) == ref


def test_allocation_failure_in_energy_forces(mbd, lib):
    """A workspace allocation failing in mbd_energy_forces: MBD_ERR_OOM, the
    force buffer and the energy untouched; the same handle then succeeds."""
    s = _sys()
    g = mbd.MBDSystem.from_workload(s)
    forces = torch.full((s.n_atoms, 3), 7.0, dtype=torch.float64, device="cuda")
    energy = ctypes.c_double(-99.0)
    lib.mbd_debug_fail_allocation(0)
    rc = lib.mbd_energy_forces(g._handle, 16, 10, 4, ctypes.byref(energy), forces.data_ptr())
    lib.mbd_debug_fail_allocation(-1)
    assert rc == OOM
    assert energy.value == -99.0
    assert torch.all(forces == 7.0)
    e1, f1 = g.energy_forces(16, 10, 4)
    e2, f2 = mbd.MBDSystem.from_workload(s).energy_forces(16, 10, 4)
    assert e1 == e2 and torch.equal(f1, f2)


def test_nonfinite_tridiagonal(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    a = np.array([[2.0, 3.0, np.nan], [2.0, 3.0, 1.0]])
    b = np.array([[0.5, 0.5, 0.0], [0.5, 0.5, 0.0]])
    q = np.full(2, -1.0)
    rc = lib.mbd_tridiag_quadrature(2, 3, a.ctypes.data_as(dp), b.ctypes.data_as(dp), q.ctypes.data_as(dp))
    assert rc == NONFINITE
    assert np.all(q == -1.0)


def test_nonfinite_dense_operator(mbd, lib):
    """A NaN entry in the dense operator of the Lanczos layer reaches every
    coefficient: MBD_ERR_NONFINITE, energy untouched."""
    dim = 12
    rng = np.random.default_rng(2)
    m = rng.normal(size=(dim, dim))
    c = m @ m.T + dim * np.eye(dim)
    c[3, 5] = c[5, 3] = np.nan
    c_dev = torch.tensor(c, dtype=torch.float64, device="cuda")
    energy = ctypes.c_double(-99.0)
    rc = lib.mbd_lanczos_energy_dense(dim, c_dev.data_ptr(), 1.0, 4, 6, 11, ctypes.byref(energy), None, None)
    assert rc == NONFINITE
    assert energy.value == -99.0


def test_nonfinite_fp32_operator(mbd, lib):
    """alpha = 1e200 bohr^3 on one atom passes validation (finite, positive),
    but its generalized dipole g y overflows FP32 in the mixed-precision
    operator: the mesh and every field turn NaN, and the energy call returns
    MBD_ERR_NONFINITE with the energy untouched.  Other systems still work."""
    s = _sys()
    alpha = s.alpha.copy()
    alpha[0] = 1e200
    g = mbd.MBDSystem.from_workload(s.with_(alpha=alpha), precision="mixed")
    energy = ctypes.c_double(-99.0)
    rc = lib.mbd_lanczos_energy(g._handle, 8, 10, 5, ctypes.byref(energy), None, None, None)
    assert rc == NONFINITE
    assert energy.value == -99.0
    assert np.isfinite(mbd.MBDSystem.from_workload(s, precision="mixed").lanczos_energy(8, 10, 5))
