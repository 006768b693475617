"""The operator bound on the water boxes: the GPU FP64 product C x with SPME
reciprocal space against the direct Ewald sum at the same split (same beta,
real-space cutoff and damping-correction truncation, converged reciprocal
sum), relative L2 error <= 1e-5, and no atom's error above 3e-5 of the RMS
atom norm (Eqs. ccd, lk3, ewalddip, fld_ewald2, spme).

3000 atoms: the whole product.  24,000 and 100,002 atoms: x is nonzero on a
seeded sample of 256 atoms and the product is read on the same atoms.  The
same-split field of dipoles carried by a subset of atoms, read on that subset,
is the field of the subsystem of those atoms in the same cell, so the oracle
evaluates it on that subsystem (the direct reciprocal sum over 10^5 atoms
would take hours).
"""
import numpy as np
import pytest
import torch

from _parity import close
from oracle.ewald import apply_T
from oracle.operator import Operator
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


def test_water3000_operator_bound(mbd):
    s = config(2)
    op = Operator(s, "spme")
    x = np.random.default_rng(40).normal(size=(2, 3 * s.n_atoms))
    d = (x * op.g).reshape(2, s.n_atoms, 3)
    y_ref = op.w2 * x + op.g * apply_T(s, d, "same_split", real_matrix=op.real).reshape(2, -1)
    y = mbd.MBDSystem.from_workload(s, precision="fp64").apply_C(_t(x)).cpu().numpy()
    close(y, y_ref, 1e-5, atom_factor=3.0)
    close(y, op(x), 1e-11)


@pytest.mark.parametrize("c", [3, 5])
def test_water_operator_bound_sampled(mbd, c):
    s = config(c)
    rng = np.random.default_rng(41 + c)
    idx = np.sort(rng.choice(s.n_atoms, size=256, replace=False))
    x = np.zeros((1, s.n_atoms, 3))
    x[0, idx] = rng.normal(size=(idx.size, 3))
    y = mbd.MBDSystem.from_workload(s, precision="fp64").apply_C(_t(x.reshape(1, -1))).cpu().numpy()
    y = y.reshape(1, s.n_atoms, 3)[:, idx]
    sub = s.with_(pos=s.pos[idx], alpha=s.alpha[idx], omega=s.omega[idx], r_vdw=s.r_vdw[idx])
    y_ref = Operator(sub, "same_split")(x[:, idx].reshape(1, -1)).reshape(1, idx.size, 3)
    close(y, y_ref, 1e-5, atom_factor=3.0)
