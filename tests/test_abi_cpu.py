"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
exports every entry point include/mbd.h declares, and rejects bad arguments
before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libmbd():
    from paper_2307_02278_gb300.build import build
    build()
    from paper_2307_02278_gb300._abi import lib
    return lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "mbd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mbd_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(libmbd):
    names = _declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(libmbd, n), f"{n} not exported"


def test_status_strings(libmbd):
    from paper_2307_02278_gb300._abi import STATUS
    for code, name in STATUS.items():
        assert libmbd.mbd_status_string(code).decode() == name


def _desc(**over):
    from paper_2307_02278_gb300._abi import SystemDesc
    n = 4
    keep = dict(pos=np.random.default_rng(0).uniform(0, 10, (n, 3)), alpha=np.full(n, 8.0),
                omega=np.full(n, 0.5), rvdw=np.full(n, 3.5))
    keep.update({k: v for k, v in over.items() if k in keep})
    d = SystemDesc()
    d.n_atoms = over.get("n_atoms", n)
    d.cell[:] = list(over.get("cell", np.eye(3).ravel() * 10.0))
    dp = ctypes.POINTER(ctypes.c_double)
    d.pos = keep["pos"].ctypes.data_as(dp)
    d.alpha = keep["alpha"].ctypes.data_as(dp)
    d.omega = keep["omega"].ctypes.data_as(dp)
    d.r_vdw = keep["rvdw"].ctypes.data_as(dp)
    d.damp_beta, d.damp_d, d.ewald_beta = 0.83, 6.0, over.get("ewald_beta", 0.35)
    d.r_cut, d.damp_cut = 4.0, 0.0
    d.mesh[:] = list(over.get("mesh", (16, 16, 16)))
    d.spline_order = over.get("p", 6)
    d.precision = over.get("precision", 0)
    d.quadrature = over.get("eigen", 0)
    return d, keep


@pytest.mark.parametrize("over", [
    dict(n_atoms=0),
    dict(cell=[10, 0, 0, 0, 10, 0, 0, 0, -10]),          # left-handed
    dict(alpha=np.array([8.0, -1.0, 8.0, 8.0])),
    dict(omega=np.array([0.5, 0.5, np.nan, 0.5])),
    dict(pos=np.array([[0, 0, 0], [1, 1, np.inf], [2, 2, 2], [3, 3, 3]], float)),
    dict(mesh=(16, 14, 16)),                              # 7 is not a smooth factor
    dict(mesh=(8, 16, 16)),                               # below 2p
    dict(p=5),                                            # odd order
    dict(p=12),
    dict(precision=3),
    dict(ewald_beta=0.0),
    dict(eigen=3),
])
def test_invalid_descriptors_rejected(libmbd, over):
    d, keep = _desc(**over)
    out = ctypes.c_void_p()
    assert libmbd.mbd_create_system(ctypes.byref(d), None, ctypes.byref(out)) == 1   # MBD_ERR_INVALID_ARG
    assert out.value is None


def test_null_arguments(libmbd):
    out = ctypes.c_void_p()
    assert libmbd.mbd_create_system(None, None, ctypes.byref(out)) == 1
    d, keep = _desc()
    assert libmbd.mbd_create_system(ctypes.byref(d), None, None) == 1
    e = ctypes.c_double()
    assert libmbd.mbd_lanczos_energy(None, 4, 4, 1, ctypes.byref(e), None, None, None) == 1
    assert libmbd.mbd_apply_C(None, 1, None, None) == 1
    q = np.zeros(1)
    dp = ctypes.POINTER(ctypes.c_double)
    assert libmbd.mbd_tridiag_quadrature(1, 0, q.ctypes.data_as(dp), q.ctypes.data_as(dp), q.ctypes.data_as(dp)) == 1
    libmbd.mbd_destroy_system(None)


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_device_reported(libmbd):
    d, keep = _desc()
    out = ctypes.c_void_p()
    assert libmbd.mbd_create_system(ctypes.byref(d), None, ctypes.byref(out)) == 8   # MBD_ERR_NO_DEVICE


def test_product_path_has_no_oracle_import():
    """The library package never imports the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2307_02278_gb300")
    for fn in os.listdir(pkg):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg, fn)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), fn
