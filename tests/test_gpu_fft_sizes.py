"""Every mesh size with a compile-time FFT pass (all 2^a 3^b 5^c sizes in
[16, 256]) in every position: along k3 (narrow rows, and the spreading fused
with it), along k2, and along k1 (the pass fused with the influence function).
The FFT convolution is compared with the oracle's (NumPy FFT) at 1e-12 (FP64)
and 1e-5 (FP32 mesh), and the fused spreading through Lanczos quadratures on
identical probes (1e-8 FP64, 2e-6 FP32 mesh)."""
import numpy as np
import pytest
import torch

from oracle import spme as ospme
from oracle.lanczos import slq
from oracle.operator import Operator
from _parity import atom_max, close, rel
from workloads.systems import random_system

pytestmark = pytest.mark.gpu


def _smooth(n):
    for f in (2, 3, 5):
        while n % f == 0:
            n //= f
    return n == 1


SIZES = [k for k in range(16, 257) if _smooth(k)]


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _system(mesh):
    return random_system(6, 12.0, 99, mesh=mesh, r_cut=5.9, damp_cut=5.9)




def test_size_list():
    assert len(SIZES) == 41 and SIZES[0] == 16 and SIZES[-1] == 256


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("precision,nvecs,tol", [("fp64", (2, 32), 1e-12), ("mixed", (2, 64), 1e-5)])
def test_convolve_every_size(mbd, axis, precision, nvecs, tol):
    """nvec = 2 gives one complex column per mesh point (masked tiles); 32 or 64
    give whole tiles of 16 (FP64) or 32 (FP32) columns along k3."""
    rng = np.random.default_rng(7 + axis)
    bad = []
    for k in SIZES:
        mesh = [16, 18, 20]
        mesh[axis] = k
        mesh = tuple(mesh)
        s = _system(mesh)
        g = mbd.MBDSystem.from_workload(s, precision=precision)
        for nvec in nvecs:
            q = rng.normal(size=(nvec,) + mesh)
            phi = g.convolve(torch.tensor(q, dtype=torch.float64, device="cuda")).cpu().numpy()
            ref = ospme.convolve(s, q)
            err, err_pt = rel(phi, ref), atom_max(phi, ref, width=1)
            if not (err < tol and err_pt < 10.0 * tol):
                bad.append((mesh, nvec, err, err_pt))
        g.close()
    assert not bad, bad


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("mixed", 2e-6)])
def test_fused_spreading_every_k3(mbd, precision, tol):
    """R = 32 probes: 16 complex columns, the fused spreading + k3 pass for every
    compile-time k3 size (tiles of 16 in both precisions)."""
    R, m, seed = 32, 4, 2468
    bad = []
    for k in SIZES:
        s = _system((16, 16, k))
        g = mbd.MBDSystem.from_workload(s, precision=precision)
        _, det = g.lanczos_energy(R, m, seed, details=True)
        g.close()
        q_ref, _, _, _ = slq(Operator(s, "spme"), 3 * s.n_atoms, R, m, seed)
        err = np.max(np.abs(det["q"] - q_ref) / np.abs(q_ref))
        if not err < tol:
            bad.append((k, err))
    assert not bad, bad
