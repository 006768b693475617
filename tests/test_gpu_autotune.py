"""mbd_autotune: the chosen launch settings are valid, leave C x unchanged bit
for bit (tile widths and atoms per block do not enter the arithmetic of a
product), and leave energies unchanged up to the summation order of a_k: FP64
to 1e-12 (the Chebyshev quadrature's spectral interval is bracketed by Sturm
counts, so a last-bit change of a_k can move it and the expansion's 1e-13-level
truncation with it); with the FP32 operator a last-bit change of y_k can flip
the FP32 rounding of a few dipoles, so 1e-10 for the energy.  The per-probe
coefficients a_k of the FP32 operator get 1e-6: once a Ritz value of a probe
has converged, the recurrence amplifies such a flip over the later steps (one
probe of 64 at mesh 64^3 moved by 5e-8), while the quadrature stays within
1e-10.  mbd_set_launch_choices applies saved choices (bit-identical results)
and refuses invalid ones."""
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


@pytest.fixture(scope="module", params=[48, 64])
def box(request):
    k = request.param
    return water_system(300, 31, mesh=(k, k, k))


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
    np.testing.assert_allclose(d1["a"], d0["a"], rtol=tol if precision == "fp64" else 1e-6)
    f0 = plain.energy_forces(R, 12, 99)[1]
    f1 = tuned.energy_forces(R, 12, 99)[1]
    assert float((f1 - f0).abs().max()) <= 100 * tol * float(f0.abs().max())


def test_autotune_invalid(mbd, box):
    g = mbd.MBDSystem.from_workload(box, precision="mixed")
    with pytest.raises(mbd.MBDError):
        g.autotune(0)


def test_set_launch_choices(mbd, box):
    """A second system given the tuner's choices reproduces the tuned system's
    results bit for bit (the computation is deterministic); None returns to the
    built-in rules, whose results a fresh system reproduces."""
    R, m, seed = 64, 10, 5
    tuned = mbd.MBDSystem.from_workload(box, precision="mixed")
    c = tuned.autotune(R)
    other = mbd.MBDSystem.from_workload(box, precision="mixed")
    other.set_launch_choices(c)
    e1, d1 = tuned.lanczos_energy(R, m, seed, details=True)
    e2, d2 = other.lanczos_energy(R, m, seed, details=True)
    assert e1 == e2 and np.array_equal(d1["a"], d2["a"]) and np.array_equal(d1["b"], d2["b"])
    other.set_launch_choices(None)
    fresh = mbd.MBDSystem.from_workload(box, precision="mixed")
    assert other.lanczos_energy(R, m, seed) == fresh.lanczos_energy(R, m, seed)
    for bad in ({"ld": 7}, {"ld": -2}, {"ld": 64, "field_atoms_per_block": 65},
                {"ld": 64, "spread_tile": 8}, {"ld": 64, "fft_tile": 24}):
        with pytest.raises(mbd.MBDError):
            other.set_launch_choices(bad)
    g64 = mbd.MBDSystem.from_workload(box, precision="fp64")
    with pytest.raises(mbd.MBDError):
        g64.set_launch_choices({"ld": 8, "fft_tile": 32})
    g64.set_launch_choices({"ld": 8, "field_atoms_per_block": 3})
    for g in (tuned, other, fresh, g64):
        g.close()
