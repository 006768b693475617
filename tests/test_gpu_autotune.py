"""mbd_autotune: the chosen launch settings are valid, leave C x unchanged bit
for bit (tile widths and atoms per block do not enter the arithmetic of a
product), and leave energies unchanged up to the summation order of a_k: FP64
to 1e-12 (the Chebyshev quadrature's spectral interval is bracketed by Sturm
counts, so a last-bit change of a_k can move it and the expansion's 1e-13-level
truncation with it); with the FP32 operator a last-bit change of y_k can flip
the FP32 rounding of a few dipoles, so 1e-10."""
import numpy as np
import pytest
import torch

from workloads.systems import water_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


@pytest.fixture(scope="module")
def box():
    return water_system(300, 31, mesh=(48, 48, 48))


@pytest.mark.parametrize("precision,R", [("mixed", 64), ("mixed", 32), ("fp64", 32)])
def test_autotune_keeps_results(mbd, box, precision, R):
    plain = mbd.MBDSystem.from_workload(box, precision=precision)
    tuned = mbd.MBDSystem.from_workload(box, precision=precision)
    c = tuned.autotune(R)
    assert c["ld"] == R + (R & 1)
    assert 1 <= c["field_atoms_per_block"] <= 64
    if precision == "mixed":
        assert c["fft_tile"] in (16, 32)
        assert c["spread_tile"] in ((16, 32) if (c["ld"] // 2) % 32 == 0 else (0,))
    else:
        assert c["fft_tile"] == 0 and c["spread_tile"] == 0
    x = torch.randn(R, 3 * box.n_atoms, dtype=torch.float64, device="cuda")
    assert torch.equal(plain.apply_C(x), tuned.apply_C(x))
    tol = 1e-12 if precision == "fp64" else 1e-10
    e0, d0 = plain.lanczos_energy(R, 12, 99, details=True)
    e1, d1 = tuned.lanczos_energy(R, 12, 99, details=True)
    assert abs(e1 - e0) <= tol * abs(e0)
    np.testing.assert_allclose(d1["a"], d0["a"], rtol=tol)
    f0 = plain.energy_forces(R, 12, 99)[1]
    f1 = tuned.energy_forces(R, 12, 99)[1]
    assert float((f1 - f0).abs().max()) <= 100 * tol * float(f0.abs().max())


def test_autotune_invalid(mbd, box):
    g = mbd.MBDSystem.from_workload(box, precision="mixed")
    with pytest.raises(mbd.MBDError):
        g.autotune(0)
