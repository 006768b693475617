"""Delta_11 (the first diagonal element of the Lanczos tridiagonal for a fixed
probe, the observable of the paper's mesh-convergence study) on the GPU against
the oracle at the same mesh, for the 14.2 angstrom water and diamond boxes; and
the chooser's parameters run through the GPU path."""
import numpy as np
import pytest
import torch

from oracle.lanczos import normalised_probes
from oracle.operator import Operator
from workloads.systems import diamond_system, water_system

pytestmark = pytest.mark.gpu
SEED = 2307022781


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _box(which):
    s = water_system(96, 5) if which == "water96" else diamond_system()
    return s.with_(r_cut=12.0, damp_cut=13.0, ewald_beta=0.3)


def _delta11(mbd, s, precision):
    g = mbd.MBDSystem.from_workload(s, precision=precision)
    _, det = g.lanczos_energy(1, 2, SEED, details=True)
    g.close()
    return det["a"][0, 0]


@pytest.mark.parametrize("which", ["water96", "diamond512"])
@pytest.mark.parametrize("k", [12, 18, 27])
def test_delta11_parity(mbd, which, k):
    s = _box(which).with_(mesh=(k, k, k))
    v = normalised_probes(SEED, 1, 3 * s.n_atoms)[0]
    ref = v @ Operator(s, "spme")(v)
    assert abs(_delta11(mbd, s, "fp64") - ref) <= 1e-11 * abs(ref)
    assert abs(_delta11(mbd, s, "mixed") - ref) <= 1e-6 * abs(ref)


def test_chosen_parameters_on_gpu(mbd):
    s = water_system(96, 5)
    c = mbd.spme_params(s, 1e-4, 6)
    t = s.with_(ewald_beta=c["ewald_beta"], r_cut=c["r_cut"], damp_cut=c["damp_cut"], mesh=c["mesh"])
    v = normalised_probes(SEED, 1, 3 * t.n_atoms)[0]
    ref_exact = v @ Operator(t, "exact")(v)
    d11 = _delta11(mbd, t, "fp64")
    assert abs(d11 - v @ Operator(t, "spme")(v)) <= 1e-11 * abs(ref_exact)
    assert abs(d11 - ref_exact) <= 1e-4 * abs(ref_exact)
