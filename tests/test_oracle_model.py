"""Pins for oracle/model.py, the B-splines of oracle/spme.py and the probe
generator of oracle/lanczos.py against closed forms and published values."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.lanczos import rademacher_probes, splitmix64
from oracle.model import (dipole_tensor, dipole_tensor_grad, fermi_damping, fermi_damping_dr,
                          reciprocal_cell, cell_volume)
from oracle.spme import bspline_moduli, cardinal_bspline, cardinal_bspline_deriv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_dimer_closed_form():
    """Free-space two-oscillator dimer (Eq. ham with two atoms): along the axis
    T has eigenvalue -2/r^3, across it +1/r^3, so each Cartesian mode is a 2x2
    problem with lambda = (w1^2+w2^2)/2 +- sqrt((w1^2-w2^2)^2/4 + (w1 w2 sqrt(a1 a2) s t)^2)."""
    w = np.array([0.43, 0.57])
    a = np.array([7.5, 11.0])
    rv = np.array([3.1, 3.6])
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    for r in (2.5, 4.0, 7.0, 12.0):
        rvec = r * axis
        s = fermi_damping(r, rv.sum(), 0.83, 6.0)
        c = np.zeros((6, 6))
        c[:3, :3] = w[0] ** 2 * np.eye(3)
        c[3:, 3:] = w[1] ** 2 * np.eye(3)
        blk = w[0] * w[1] * np.sqrt(a[0] * a[1]) * s * dipole_tensor(rvec)
        c[:3, 3:] = blk
        c[3:, :3] = blk.T
        lam = np.sort(np.linalg.eigvalsh(c))
        ref = []
        for t in (1.0 / r ** 3, 1.0 / r ** 3, -2.0 / r ** 3):
            x = w[0] * w[1] * np.sqrt(a[0] * a[1]) * s * t
            m = 0.5 * (w[0] ** 2 + w[1] ** 2)
            dd = np.sqrt(0.25 * (w[0] ** 2 - w[1] ** 2) ** 2 + x * x)
            ref += [m - dd, m + dd]
        np.testing.assert_allclose(lam, np.sort(ref), rtol=1e-14, atol=0)
        # head-to-tail coupling softens the lowest mode (attractive dispersion)
        assert lam[0] < min(w) ** 2


def test_dipole_tensor_traceless_and_grad():
    rng = np.random.default_rng(3)
    r = rng.normal(size=(20, 3)) * 3
    t = dipole_tensor(r)
    np.testing.assert_allclose(np.trace(t, axis1=1, axis2=2), 0.0, atol=1e-15)
    h = 1e-6
    g = dipole_tensor_grad(r)
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        fd = (dipole_tensor(r + e) - dipole_tensor(r - e)) / (2 * h)
        np.testing.assert_allclose(g[..., c], fd, rtol=1e-6, atol=1e-9)


def test_fermi_damping():
    r = np.linspace(0.5, 20, 50)
    s = fermi_damping(r, 6.4, 0.83, 6.0)
    assert np.all(np.diff(s) > 0) and s[0] < 0.01 and s[-1] > 0.99
    np.testing.assert_allclose(fermi_damping(0.83 * 6.4, 6.4, 0.83, 6.0), 0.5, rtol=1e-15)
    h = 1e-6
    fd = (fermi_damping(r + h, 6.4, 0.83, 6.0) - fermi_damping(r - h, 6.4, 0.83, 6.0)) / (2 * h)
    np.testing.assert_allclose(fermi_damping_dr(r, 6.4, 0.83, 6.0), fd, rtol=1e-6, atol=1e-9)


def test_reciprocal_cell():
    cell = np.array([[10.0, 0.0, 0.0], [2.0, 9.0, 0.0], [1.0, -1.5, 11.0]])
    rec = reciprocal_cell(cell)
    np.testing.assert_allclose(rec @ cell.T, np.eye(3), atol=1e-15)
    assert abs(cell_volume(cell) - 990.0) < 1e-12


def test_bspline_integer_values_golden():
    for row in _rows("cardinal_bspline_integers.txt"):
        n = int(row[0])
        ref = [float(Fraction(x)) for x in row[1:]]
        np.testing.assert_allclose(cardinal_bspline(np.arange(1.0, n), n), ref, rtol=1e-14)


@pytest.mark.parametrize("p", [4, 6, 8])
def test_bspline_partition_of_unity(p):
    x = np.random.default_rng(p).uniform(0, 1, size=100)
    t = np.arange(p)
    vals = cardinal_bspline(x[:, None] + t[None, :], p)
    np.testing.assert_allclose(vals.sum(axis=1), 1.0, rtol=1e-14)
    for order in (1, 2):
        der = cardinal_bspline_deriv(x[:, None] + t[None, :], p, order)
        np.testing.assert_allclose(der.sum(axis=1), 0.0, atol=1e-13)
    h = 1e-6
    fd = (cardinal_bspline(x + 2 + h, p) - cardinal_bspline(x + 2 - h, p)) / (2 * h)
    np.testing.assert_allclose(cardinal_bspline_deriv(x + 2, p), fd, rtol=1e-6, atol=1e-9)
    fd2 = (cardinal_bspline_deriv(x + 2 + h, p) - cardinal_bspline_deriv(x + 2 - h, p)) / (2 * h)
    np.testing.assert_allclose(cardinal_bspline_deriv(x + 2, p, 2), fd2, rtol=1e-5, atol=1e-8)


def test_bspline_moduli():
    b = bspline_moduli(32, 6)
    assert abs(b[0] - 1.0) < 1e-14          # sum_k M_p(k+1) = 1
    np.testing.assert_allclose(b[1:], b[1:][::-1], rtol=1e-13)   # |b(m)| = |b(-m)|
    assert np.all(b >= 1.0 - 1e-14) and np.isfinite(b).all()


def test_splitmix64_golden():
    ref = [int(r[0], 16) for r in _rows("splitmix64_state0.txt")]
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % 2 ** 64], dtype=np.uint64)
    assert [int(x) for x in splitmix64(states)] == ref


def test_probe_rule():
    u = rademacher_probes(12345, 4, 1000)
    assert set(np.unique(u)) == {-1.0, 1.0}
    assert abs(u.mean()) < 0.1
    # rule: top bit of SplitMix64(seed + (l << 32) + i)
    x = np.uint64(12345) + (np.uint64(2) << np.uint64(32)) + np.uint64(17)
    top = int(splitmix64(np.array([x]))[0]) >> 63
    assert u[2, 17] == (1.0 if top == 0 else -1.0)
    np.testing.assert_array_equal(rademacher_probes(12345, 2, 1000, first=2), u[2:])
