"""Batches of independent systems (mbd_create_batch / mbd_batch_lanczos_energy):
every member of a graph-replayed batch against the same system run alone and,
for the 64-atom member, against the FP64 oracle's Lanczos quadrature on the
same probes (1e-8 relative)."""
import numpy as np
import pytest
import torch

from oracle.lanczos import slq_energy
from oracle.operator import Operator
from workloads.systems import WATER_ATOM_DENSITY, config, random_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbd():
    from paper_2307_02278_gb300.build import build
    build()
    import paper_2307_02278_gb300 as m
    torch.cuda.set_device(0)
    return m


def _members():
    """Uneven members: different atom counts, cells and meshes (radix 2, 3 and 5
    sizes), one skewed cell, and the 64-atom box."""
    out = [random_system(24, 12.0, 4242, mesh=(16, 16, 16), r_cut=5.9, damp_cut=5.9),
           config(1)]
    cell = np.array([[13.0, 0.0, 0.0], [1.5, 12.5, 0.0], [-0.8, 1.2, 13.5]])
    base = random_system(40, 13.0, 77, r_cut=5.9, damp_cut=5.9)
    out.append(base.with_(cell=cell, pos=(base.pos / 13.0) @ cell, mesh=(25, 27, 30)))
    for n, seed in ((300, 5), (900, 6)):
        box = (n / WATER_ATOM_DENSITY) ** (1.0 / 3.0)
        out.append(random_system(n, box, seed))          # mesh: smooth size >= box (1 bohr spacing)
    return out


@pytest.fixture(scope="module")
def members():
    return _members()


def _single(mbd, s, precision, R, m, seed):
    return mbd.MBDSystem.from_workload(s, precision=precision).lanczos_energy(R, m, seed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_single_systems(mbd, members, precision):
    R, m = 8, 20
    seeds = np.arange(len(members), dtype=np.uint64) + 2307022784
    with mbd.MBDBatch(members, precision=precision) as b:
        e, t = b.lanczos_energy(R, m, seeds)
        info = b.info()
    assert info["n_sys"] == len(members) and info["graph_kernels"] > 0
    assert info["total_atoms"] == sum(s.n_atoms for s in members)
    for i, s in enumerate(members):
        ref = _single(mbd, s, precision, R, m, int(seeds[i]))
        # same kernels in the same order on the same data
        assert abs(e[i] - ref) <= 1e-13 * abs(ref), (i, e[i], ref)
        assert abs((0.5 * t[i] - 1.5 * s.omega.sum()) - e[i]) <= 1e-12 * abs(e[i])


def test_batch_member_against_oracle(mbd, members):
    s = config(1)
    R, m = s.n_probes, s.n_steps
    seeds = np.full(len(members), 11, dtype=np.uint64)
    seeds[1] = s.probe_seed
    with mbd.MBDBatch(members, precision="fp64") as b:
        e, _ = b.lanczos_energy(R, m, seeds)
    ref, _ = slq_energy(Operator(s, "spme"), R, m, s.probe_seed)
    assert abs(e[1] - ref) <= 1e-8 * abs(ref)


def test_batch_replay_new_seeds_and_recapture(mbd, members):
    with mbd.MBDBatch(members, precision="mixed") as b:
        s0 = np.arange(len(members), dtype=np.uint64) + 7
        e0, _ = b.lanczos_energy(6, 12, s0)
        k0 = b.info()["graph_kernels"]
        s1 = s0 + 1000
        e1, _ = b.lanczos_energy(6, 12, s1)            # replay: only the seeds change
        assert b.info()["graph_kernels"] == k0
        assert np.all(e1 != e0)
        e0b, _ = b.lanczos_energy(6, 12, s0)           # and back: replays are deterministic
        np.testing.assert_array_equal(e0b, e0)
        e2, _ = b.lanczos_energy(5, 15, s1)            # new (R, m): a new graph
        assert b.info()["graph_kernels"] != k0
    for i in (0, 3):
        ref1 = _single(mbd, members[i], "mixed", 6, 12, int(s1[i]))
        ref2 = _single(mbd, members[i], "mixed", 5, 15, int(s1[i]))
        assert abs(e1[i] - ref1) <= 1e-13 * abs(ref1)
        assert abs(e2[i] - ref2) <= 1e-13 * abs(ref2)


def test_batch_failing_member(mbd, members):
    """A member in the polarisation catastrophe (C not positive definite) is
    reported by index; the others are unaffected on the next call."""
    bad = members[0].with_(alpha=members[0].alpha * 60.0)
    batch = [members[1], members[2], bad, members[3]]
    with mbd.MBDBatch(batch, precision="fp64") as b:
        with pytest.raises(mbd.MBDError) as err:
            b.lanczos_energy(4, 20, np.arange(4, dtype=np.uint64))
    assert err.value.code == 4 and "member 2" in str(err.value)


def test_batch_rejects_mixed_precisions_and_bad_args(mbd, members):
    from paper_2307_02278_gb300._abi import SystemDesc, lib
    from paper_2307_02278_gb300.system import _make_desc, _workload_kw
    import ctypes
    descs = (SystemDesc * 2)()
    keep = []
    for i, prec in enumerate(("fp64", "mixed")):
        s = members[i]
        d, k = _make_desc(s.cell, s.pos, s.alpha, s.omega, s.r_vdw, precision=prec, **_workload_kw(s))
        descs[i] = d
        keep.append(k)
    out = ctypes.c_void_p()
    assert lib().mbd_create_batch(2, descs, None, ctypes.byref(out)) == 1
    assert lib().mbd_create_batch(0, descs, None, ctypes.byref(out)) == 1
    with mbd.MBDBatch(members[:2], precision="fp64") as b:
        with pytest.raises(mbd.MBDError):
            b.lanczos_energy(0, 10, np.zeros(2, dtype=np.uint64))
        with pytest.raises(mbd.MBDError):
            b.lanczos_energy(4, 129, np.zeros(2, dtype=np.uint64))
