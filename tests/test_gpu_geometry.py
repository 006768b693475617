"""mbd_update_positions rebuilds the neighbour list, pair tensors, splines,
bricks and spreading matrix on the device with one readback at the end.  An
updated system must give bit for bit what a system created at the new
positions gives: the lists are in a fixed order (bricks sorted by atom index,
neighbours in cell order), whether the pair list fits its buffers or outgrows
them (filled again into larger ones) or shrinks."""
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
    return water_system(300, 17, mesh=(48, 48, 48))


def _same(mbd, g, s, pos, precision, x, energy=True):
    fresh = mbd.MBDSystem.from_workload(s.with_(pos=pos), precision=precision)
    assert g.info()["n_pairs"] == fresh.info()["n_pairs"]
    assert torch.equal(g.apply_C(x), fresh.apply_C(x))
    if energy:
        e1, f1 = g.energy_forces(16, 8, 3)
        e2, f2 = fresh.energy_forces(16, 8, 3)
        assert e1 == e2 and torch.equal(f1, f2)
    fresh.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_matches_fresh(mbd, box, precision):
    g = mbd.MBDSystem.from_workload(box, precision=precision)
    x = torch.randn(8, 3 * box.n_atoms, dtype=torch.float64, device="cuda")
    pos2 = box.pos + np.random.default_rng(1).normal(scale=0.15, size=box.pos.shape)
    g.update_positions(pos2)
    _same(mbd, g, box, pos2, precision, x)
    g.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_list_growth_and_shrink(mbd, box, precision):
    """Compressing the atoms towards the cell centre grows the pair list beyond
    the buffers' quarter of headroom (the refill path); going back shrinks it."""
    g = mbd.MBDSystem.from_workload(box, precision=precision)
    n0 = g.info()["n_pairs"]
    x = torch.randn(4, 3 * box.n_atoms, dtype=torch.float64, device="cuda")
    centre = box.cell.sum(axis=0) / 2
    dense = centre + 0.8 * (np.mod(box.pos, np.diag(box.cell)) - centre)
    g.update_positions(dense)
    assert g.info()["n_pairs"] > n0 + n0 // 4 + 32   # beyond the capacity sized at creation
    _same(mbd, g, box, dense, precision, x, energy=False)   # compressed bonds: C x only
    g.update_positions(box.pos)
    assert g.info()["n_pairs"] == n0
    _same(mbd, g, box, box.pos, precision, x)
    g.close()


def test_repeated_updates_return(mbd, box):
    g = mbd.MBDSystem.from_workload(box, precision="mixed")
    x = torch.randn(4, 3 * box.n_atoms, dtype=torch.float64, device="cuda")
    y0 = g.apply_C(x)
    rng = np.random.default_rng(5)
    for _ in range(5):
        g.update_positions(box.pos + rng.normal(scale=0.1, size=box.pos.shape))
    g.update_positions(box.pos)
    assert torch.equal(g.apply_C(x), y0)
    g.close()
