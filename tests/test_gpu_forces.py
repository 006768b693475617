"""GPU forces against the exact gradient: the oracle's dense analytic gradient
and central finite differences of the oracle's dense energy.

The force estimator F = -(1/4)(D/R) sum_l (g.w_l)^T (dT'/dR) (g.v_l), with
w_l = C^{-1/2} v_l, has expectation -(1/4) Tr(C^{-1/2} dC/dR) = -dE/dR over
Rademacher probes once the quadrature is exact (m >= 3N Lanczos steps).  The
GPU FP64 path runs it on many probes in calls whose probe streams are
disjoint (seeds 2^48 apart; the probe rule puts probe l of seed s at
s + (l << 32) + i), and each component of the mean force must lie within 5
standard errors, taken from the per-call means, of the exact value.

The finite difference of the GPU's own stochastic energy at fixed probes is
not the estimator's target: d/dR of v^T C^{1/2} v is v^T D[C^{1/2}](dC/dR) v,
which equals (1/2) v^T C^{-1/2} (dC/dR) v only under the trace.  The two agree
in expectation, not probe by probe, so both are compared with the exact
gradient instead.
"""
import numpy as np
import pytest
import torch

from oracle.dense import dense_energy, dense_gradient
from oracle.operator import Operator
from workloads.systems import random_system

pytestmark = pytest.mark.gpu

CALLS, PROBES_PER_CALL = 32, 2048


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _mean_force(mbd, s, n_steps, seed=977):
    g = mbd.MBDSystem.from_workload(s, precision="fp64")
    fs = []
    for c in range(CALLS):
        _, f = g.energy_forces(PROBES_PER_CALL, n_steps, seed + (c << 48))
        fs.append(f.cpu().numpy())
    g.close()
    fs = np.stack(fs)
    return fs.mean(axis=0), fs.std(axis=0, ddof=1) / np.sqrt(CALLS)


def test_forces_against_dense_gradient(mbd):
    """10 atoms (D = 30), m = 30, 65,536 probes: the mean GPU force within 5
    standard errors of -dE/dR from the oracle's dense gradient, per component.
    At this probe count a flipped sign or a doubled force lies far outside."""
    s = random_system(10, 10.5, 21, mesh=(16, 16, 16), r_cut=5.2, damp_cut=5.2)
    ref = -dense_gradient(Operator(s, "spme"))
    mean, se = _mean_force(mbd, s, 3 * s.n_atoms)
    assert np.all(np.abs(mean - ref) <= 5.0 * se), np.abs(mean - ref) / se
    assert np.abs((-mean - ref) / se).max() > 5.0
    assert np.abs((2.0 * mean - ref) / se).max() > 5.0


def test_forces_against_finite_differences(mbd):
    """6 atoms (D = 18), m = 18, 65,536 probes: the mean GPU force within 5
    standard errors of minus the central difference (h = 1e-4 bohr) of the
    oracle's dense energy (Eq. plasmonic, from eigh of C), every component."""
    s = random_system(6, 9.5, 17, mesh=(16, 16, 16), r_cut=4.6, damp_cut=4.6)
    h = 1e-4
    fd = np.zeros((s.n_atoms, 3))
    for i in range(s.n_atoms):
        for c in range(3):
            e = []
            for sgn in (1.0, -1.0):
                p = s.pos.copy()
                p[i, c] += sgn * h
                e.append(dense_energy(Operator(s.with_(pos=p), "spme").dense(), s.omega))
            fd[i, c] = -(e[0] - e[1]) / (2.0 * h)
    mean, se = _mean_force(mbd, s, 3 * s.n_atoms)
    assert np.all(np.abs(mean - fd) <= 5.0 * se), np.abs(mean - fd) / se
    assert np.abs((-mean - fd) / se).max() > 5.0
