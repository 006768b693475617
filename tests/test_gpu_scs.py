"""GPU parity of the screening front end (mbd_scs_screen) against the oracle
(oracle/scs.py), through the C ABI.

Tolerances, per atom (largest relative error of alpha^SCS at every
frequency, of omega^SCS, C6 and R_vdw^SCS):
- FP64 systems: the conjugate gradient stops at residual 1e-12 of the
  right-hand side; with condition numbers of a few, the solution error is of
  that order: 1e-9 leaves room for the summation order.
- mixed systems: T_SR and the search direction in FP32, each T_SR x a sum of
  about 100 FP32 pair products (relative rounding ~1e-6 of a term that is a
  fraction of the diagonal): 3e-6.
"""
import numpy as np
import pytest
import torch

from oracle import scs as oscs
from oracle.lanczos import slq_energy
from oracle.operator import Operator
from workloads.systems import System, config, random_system, water_system

pytestmark = pytest.mark.gpu

KEYS = ("alpha", "omega", "r_vdw", "c6")


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _periodic_small():
    rng = np.random.default_rng(21)
    box, n = 9.0, 6
    while True:
        pos = rng.uniform(0, box, size=(n, 3))
        diff = pos[:, None] - pos[None]
        diff -= box * np.round(diff / box)
        if (np.sqrt(np.sum(diff ** 2, -1)) + np.eye(n) * 99).min() > 2.2:
            break
    return System(name="periodic6", cell=np.eye(3) * box, pos=pos, alpha=rng.uniform(4, 12, n),
                  omega=rng.uniform(0.3, 0.7, n), r_vdw=rng.uniform(3.0, 3.8, n), r_cut=11.0, damp_cut=11.0,
                  mesh=(16, 16, 16))


def _water(n_mol=150, seed=77):
    return water_system(n_mol, seed, r_cut=9.0, damp_cut=9.0, ewald_beta=0.35)


def _systems():
    return {"c1": config(1), "periodic6": _periodic_small(), "water450": _water()}


def _worst(got, ref):
    out = {k: float(np.max(np.abs(got[k] - ref[k]) / np.abs(ref[k]))) for k in KEYS}
    out["alpha_iu"] = float(np.max(np.abs(got["alpha_iu"] - ref["alpha_iu"]) / np.abs(ref["alpha_iu"])))
    return out


@pytest.mark.parametrize("name", ["c1", "periodic6", "water450"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 3e-6)])
def test_screening_matches_oracle(mbd, name, precision, tol):
    s = _systems()[name]
    ref = oscs.scs(s, n_freq=23)
    with mbd.MBDSystem.from_workload(s, precision=precision) as g:
        got = g.scs_screen(n_freq=23, tol=1e-12, max_iter=500)
    assert got["residual"] <= 1e-12 and 0 < got["iterations"] < 500
    worst = _worst(got, ref)
    assert max(worst.values()) < tol, worst
    assert np.max(np.abs(ref["alpha"] - s.alpha) / s.alpha) > 1e-2          # the screening is not trivial


def test_water3000_screening_against_the_oracle_cg(mbd):
    s = config(2)
    ref = oscs.scs(s, n_freq=15, solver="cg")
    with mbd.MBDSystem.from_workload(s, precision="mixed") as g:
        got = g.scs_screen(n_freq=15, tol=1e-10, max_iter=500)
    worst = _worst(got, ref)
    assert max(worst.values()) < 3e-6, worst


def test_supercell_copies_agree_at_24000_atoms(mbd):
    # a property that holds at any size: every copy of an atom in a 2 x 2 x 2
    # replica of the 3000-atom box is screened like the atom itself
    s = config(2)
    L = s.cell[0, 0]
    shifts = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float) * L
    big = s.with_(cell=s.cell * 2, pos=np.concatenate([s.pos + sh for sh in shifts]), alpha=np.tile(s.alpha, 8),
                  omega=np.tile(s.omega, 8), r_vdw=np.tile(s.r_vdw, 8), mesh=(128, 128, 128))
    with mbd.MBDSystem.from_workload(s, precision="mixed") as g:
        one = g.scs_screen(n_freq=15, tol=1e-10)
    with mbd.MBDSystem.from_workload(big, precision="mixed") as g:
        eight = g.scs_screen(n_freq=15, tol=1e-10)
    for k in KEYS:
        assert np.max(np.abs(eight[k] - np.tile(one[k], 8)) / np.tile(one[k], 8)) < 3e-6, k


def test_water100002_mixed_against_fp64(mbd):
    s = config(5)
    with mbd.MBDSystem.from_workload(s, precision="mixed") as g:
        mixed = g.scs_screen(n_freq=23, tol=1e-10)
    with mbd.MBDSystem.from_workload(s, precision="fp64") as g:
        f64 = g.scs_screen(n_freq=23, tol=1e-10)
    assert mixed["residual"] <= 1e-10 and f64["residual"] <= 1e-10
    for k in KEYS:
        assert np.max(np.abs(mixed[k] - f64[k]) / np.abs(f64[k])) < 3e-6, k
    assert 0.5 < np.mean(f64["alpha"] / s.alpha) < 1.0                  # water screens its polarisabilities down


def test_screened_parameters_feed_the_mbd_energy(mbd):
    # the oracle's screened parameters and the library's give the same energy
    # on the same probes (FP64)
    s = config(1)
    ref = oscs.scs(s, n_freq=23)
    with mbd.MBDSystem.from_workload(s, precision="fp64") as g:
        got = g.scs_screen(n_freq=23, tol=1e-12)
    screened_ref = s.with_(alpha=ref["alpha"], omega=ref["omega"], r_vdw=ref["r_vdw"])
    screened_gpu = s.with_(alpha=got["alpha"], omega=got["omega"], r_vdw=got["r_vdw"])
    e_ref, _ = slq_energy(Operator(screened_ref, "spme"), s.n_probes, s.n_steps, s.probe_seed)
    with mbd.MBDSystem.from_workload(screened_gpu, precision="fp64") as g:
        e_gpu = g.lanczos_energy(s.n_probes, s.n_steps, s.probe_seed)
    assert abs(e_gpu - e_ref) < 1e-8 * abs(e_ref)
    e_unscreened, _ = slq_energy(Operator(s, "spme"), s.n_probes, s.n_steps, s.probe_seed)
    assert abs(e_ref - e_unscreened) > 1e-3 * abs(e_ref)


def test_no_iterations_returns_the_unscreened_parameters(mbd):
    s = _periodic_small()
    with mbd.MBDSystem.from_workload(s, precision="fp64") as g:
        got = g.scs_screen(n_freq=23, tol=1e-12, max_iter=0)
    assert got["iterations"] == 0
    np.testing.assert_allclose(got["alpha"], s.alpha, rtol=1e-15)
    np.testing.assert_allclose(got["omega"], s.omega, rtol=1e-9)       # the quadrature of a single pole
    np.testing.assert_allclose(got["r_vdw"], s.r_vdw, rtol=1e-15)


def test_invalid_arguments_leave_outputs_untouched(mbd):
    import ctypes
    from paper_2307_02278_gb300._abi import lib
    invalid = 1                                                          # MBD_ERR_INVALID_ARG
    s = _periodic_small()
    n = s.pos.shape[0]
    with mbd.MBDSystem.from_workload(s, precision="fp64") as g:
        a, o, r = np.full(n, 7.0), np.full(n, 7.0), np.full(n, 7.0)
        pa, po, pr = (x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in (a, o, r))
        for nf, tol, it in ((0, 1e-8, 10), (32, 1e-8, 10), (8, 0.0, 10), (8, float("nan"), 10), (8, 1e-8, -1)):
            st = lib().mbd_scs_screen(g._handle, nf, tol, it, pa, po, pr, None, None, None, None)
            assert st == invalid
        assert lib().mbd_scs_screen(g._handle, 8, 1e-8, 10, None, po, pr, None, None, None, None) == invalid
        assert np.all(a == 7.0) and np.all(o == 7.0) and np.all(r == 7.0)
