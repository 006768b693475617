"""The allocation-free quadrature entry point, through the C ABI.

mbd_tridiag_quadrature_noalloc serves callers that cannot let the library call
cudaMalloc (their device memory belongs to another allocator, or they cannot
afford the synchronisation cudaMalloc/cudaFree imply).  It must give the same
quadratures as the allocating mbd_tridiag_quadrature on consecutive calls,
reject sizes beyond its fixed scratch, and clear its shared status word on
every call.  This file is collected last so that a run stopping at the first
failure has already run every other test; it also passes alone.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle.lanczos import lanczos, normalised_probes
from oracle.operator import Operator
from workloads.systems import random_system

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2307_02278_gb300.build import build
    build()
    from paper_2307_02278_gb300._abi import lib as load
    torch.cuda.set_device(0)
    return load()


def _tridiagonals(n_probes, n_steps, seed):
    s = random_system(16, 14.0, seed, mesh=(20, 20, 20), r_cut=6.9, damp_cut=6.9)
    v = normalised_probes(seed, n_probes, 3 * s.n_atoms)
    a, b, _, _ = lanczos(Operator(s, "spme"), v, n_steps)
    return np.ascontiguousarray(a), np.ascontiguousarray(b)


def _allocating(lib, a, b):
    dp = ctypes.POINTER(ctypes.c_double)
    q = np.zeros(a.shape[0])
    rc = lib.mbd_tridiag_quadrature(a.shape[0], a.shape[1], a.ctypes.data_as(dp), b.ctypes.data_as(dp),
                                    q.ctypes.data_as(dp))
    assert rc == 0
    return q


def _noalloc(lib, a, b):
    a_dev = torch.tensor(a, dtype=torch.float64, device="cuda")
    b_dev = torch.tensor(b, dtype=torch.float64, device="cuda")
    q_dev = torch.full((a.shape[0],), -1.0, dtype=torch.float64, device="cuda")
    rc = lib.mbd_tridiag_quadrature_noalloc(a.shape[0], a.shape[1], a_dev.data_ptr(), b_dev.data_ptr(),
                                            q_dev.data_ptr(), None)
    return rc, q_dev.cpu().numpy()


def test_noalloc_matches_allocating_entry_on_consecutive_calls(lib):
    for n_probes, n_steps, seed in [(7, 20, 11), (33, 45, 12)]:
        a, b = _tridiagonals(n_probes, n_steps, seed)
        rc, q = _noalloc(lib, a, b)
        assert rc == 0
        np.testing.assert_allclose(q, _allocating(lib, a, b), rtol=1e-13, atol=0)


def test_noalloc_limits_and_status_reset(lib):
    big = np.ones((1025, 2))
    rc, _ = _noalloc(lib, big, np.zeros((1025, 2)))
    assert rc == 1                                   # MBD_ERR_INVALID_ARG: beyond the fixed scratch
    rc, _ = _noalloc(lib, np.ones((2, 129)), np.zeros((2, 129)))
    assert rc == 1
    rc, _ = _noalloc(lib, np.array([[1.0, -3.0]]), np.array([[0.1, 0.0]]))
    assert rc == 4                                   # not positive definite
    a, b = _tridiagonals(5, 12, 13)                  # the next call starts from a clean status word
    rc, q = _noalloc(lib, a, b)
    assert rc == 0
    np.testing.assert_allclose(q, _allocating(lib, a, b), rtol=1e-13, atol=0)


def test_noalloc_many_probes_and_early_zero_coupling(lib):
    """R = 300 probes spans three blocks of the preparation kernel; some rows
    carry a zero coupling mid-way (the tridiagonal ends there), as a Lanczos
    breakdown leaves them.  Same quadratures as the allocating entry point, on
    two calls in a row."""
    a, b = _tridiagonals(300, 24, 14)
    for r, k in [(0, 3), (7, 11), (150, 1), (299, 20)]:
        b[r, k] = 0.0
    for _ in range(2):
        rc, q = _noalloc(lib, a, b)
        assert rc == 0
        np.testing.assert_allclose(q, _allocating(lib, a, b), rtol=1e-13, atol=0)
