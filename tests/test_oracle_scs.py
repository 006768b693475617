"""Pins of the screening oracle (oracle/scs.py) against facts it does not
compute itself: the symbolic Hessian of the Gaussian potential erf(r/s)/r,
Poisson's equation for its trace, the Fourier integral of two Gaussian
densities (their combined width), the self-interaction identity that defines
the Gaussian width, exact quadrature of closed-form integrals, an isolated
atom (nothing to screen), the dimer solved as two scalar 2 x 2 problems from
the symbolic derivatives, and the invariants of the periodic sum (a supercell
gives every copy of an atom the same screened values; translations and
permutations of the atoms change nothing)."""
import numpy as np
import pytest

from oracle import scs
from oracle.ewald import pair_list
from oracle.model import dipole_tensor, fermi_damping
from workloads.systems import System


def _system(pos, cell, alpha, omega, r_vdw, damp_cut=10.0):
    return System(name="scs", cell=np.asarray(cell, float), pos=np.asarray(pos, float), alpha=np.asarray(alpha, float),
                  omega=np.asarray(omega, float), r_vdw=np.asarray(r_vdw, float), damp_cut=damp_cut, r_cut=damp_cut)


def _symbolic_phi_derivatives():
    sp = pytest.importorskip("sympy")
    r, s = sp.symbols("r s", positive=True)
    phi = sp.erf(r / s) / r
    return (sp.lambdify((r, s), sp.diff(phi, r), "mpmath"), sp.lambdify((r, s), sp.diff(phi, r, 2), "mpmath"))


def test_frequency_grid_integrates_closed_forms():
    u, w = scs.frequency_grid(23)
    assert np.all(u > 0) and np.all(np.diff(u) > 0)
    assert abs(np.sum(w / (1 + u) ** 3) - 0.5) < 1e-12                  # int (1+u)^-3 = 1/2
    assert abs(np.sum(w / (1 + u * u)) - np.pi / 2) < 1e-9             # int 1/(1+u^2) = pi/2
    for om in (0.2, 0.45, 0.7, 1.5):                                    # int (1 + u^2/om^2)^-2 = pi om / 4
        assert abs(np.sum(w / (1 + (u / om) ** 2) ** 2) / (np.pi * om / 4) - 1) < 1e-9
    for a, b in ((0.3, 0.6), (0.2, 1.5)):                               # two poles: pi a b / (2 (a + b))
        assert abs(np.sum(w / ((1 + (u / a) ** 2) * (1 + (u / b) ** 2))) / (np.pi * a * b / (2 * (a + b))) - 1) < 1e-9


def test_gg_tensor_is_minus_the_symbolic_hessian():
    sp = pytest.importorskip("sympy")
    x, y, z, s = sp.symbols("x y z s", real=True)
    rr = sp.sqrt(x * x + y * y + z * z)
    phi = sp.erf(rr / s) / rr
    hess = [[sp.lambdify((x, y, z, s), -sp.diff(phi, a, b), "mpmath") for b in (x, y, z)] for a in (x, y, z)]
    rng = np.random.default_rng(3)
    for _ in range(6):
        rv = rng.normal(size=3) * rng.uniform(0.5, 4.0)
        sig = rng.uniform(0.5, 3.0)
        ref = np.array([[float(hess[a][b](*rv, sig)) for b in range(3)] for a in range(3)])
        got = scs.gg_tensor(rv, sig)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_gg_tensor_tends_to_the_point_dipole_tensor():
    rng = np.random.default_rng(4)
    rv = rng.normal(size=(20, 3)) * 3.0 + np.sign(rng.normal(size=(20, 3)))
    got = scs.gg_tensor(rv, np.full(20, 1e-3))
    assert np.max(np.abs(got - dipole_tensor(rv))) < 1e-14 * np.max(np.abs(dipole_tensor(rv)))


def test_gg_trace_is_the_gaussian_density():
    # -laplacian of erf(r/s)/r = 4 pi rho, rho = (pi s^2)^(-3/2) exp(-r^2/s^2)  (Poisson)
    rng = np.random.default_rng(5)
    rv = rng.normal(size=(30, 3)) * 1.5
    sig = rng.uniform(0.8, 2.5, size=30)
    r2 = np.sum(rv * rv, axis=1)
    rho = (np.pi * sig ** 2) ** -1.5 * np.exp(-r2 / sig ** 2)
    tr = np.trace(scs.gg_tensor(rv, sig), axis1=1, axis2=2)
    assert np.max(np.abs(tr - 4 * np.pi * rho) / (4 * np.pi * rho)) < 1e-9


def test_gaussian_width_gives_self_interaction_one_over_alpha():
    # the width is chosen so that an oscillator's density, interacting with itself
    # (combined width sqrt(2) sigma), has the coupling 1/alpha at r -> 0
    # (the r -> 0 value by Richardson extrapolation of two small separations,
    # since the closed form cancels at tiny r/sigma)
    for alpha in (0.7, 5.4, 12.0, 40.0):
        sig = scs.gaussian_width(alpha)
        t1 = scs.gg_tensor(np.array([2e-3, 0.0, 0.0]) * sig, np.sqrt(2.0) * sig)
        t2 = scs.gg_tensor(np.array([1e-3, 0.0, 0.0]) * sig, np.sqrt(2.0) * sig)
        assert np.max(np.abs((4 * t2 - t1) / 3 - np.eye(3) / alpha)) < 1e-8 / alpha


def test_pair_width_from_the_fourier_integral_of_two_gaussians():
    # the Coulomb interaction of normalised Gaussian densities of widths a and b
    # at distance r is (2/pi) int_0^inf exp(-k^2 a^2/4) exp(-k^2 b^2/4) sin(kr)/(kr) dk
    from scipy.integrate import quad
    from scipy.special import erf
    for a, b, r in ((1.1, 0.7, 2.3), (1.6, 1.6, 0.9), (0.5, 2.2, 4.0)):
        val = 2 / np.pi * quad(lambda k: np.exp(-k * k * (a * a + b * b) / 4) * np.sinc(k * r / np.pi), 0, np.inf,
                               epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        assert abs(erf(r / scs.pair_width(a, b)) / r - val) < 1e-11


def test_isolated_atom_is_not_screened():
    s = _system([[1.0, 2.0, 3.0]], np.eye(3) * 25.0, [7.3], [0.41], [3.4])
    out = scs.scs(s, n_freq=23)
    assert out["alpha"][0] == pytest.approx(7.3, rel=1e-15)
    assert out["omega"][0] == pytest.approx(0.41, rel=1e-9)               # Casimir-Polder of a single pole
    assert out["r_vdw"][0] == pytest.approx(3.4, rel=1e-15)
    assert out["c6"][0] == pytest.approx(0.75 * 7.3 ** 2 * 0.41, rel=1e-9)


def test_dimer_matches_two_scalar_problems():
    dphi, d2phi = _symbolic_phi_derivatives()
    d = np.array([0.3, -0.8, 0.52])
    d *= 4.1 / np.linalg.norm(d)
    s = _system([[5.0, 5.0, 5.0], 5.0 + np.array([0.0, 0.0, 0.0]) + d], np.eye(3) * 30.0, [6.0, 9.5], [0.5, 0.33],
                [3.1, 3.6])
    R = np.linalg.norm(d)
    one_minus_f = 1.0 - fermi_damping(R, 3.1 + 3.6, s.damp_beta, s.damp_d)
    pairs = pair_list(s.cell, s.pos, s.damp_cut)
    for u in (0.0, 0.2, 1.3):
        a = scs.dynamic_polarizability(s.alpha, s.omega, u)
        sig = float(scs.pair_width(*scs.gaussian_width(a)))
        t_par = -float(d2phi(R, sig)) * one_minus_f                       # r^ T r^ = -phi''
        t_perp = -float(dphi(R, sig)) / R * one_minus_f                   # perpendicular: -phi'/r
        expect = np.zeros(2)
        for t, mult in ((t_par, 1.0), (t_perp, 2.0)):
            m = np.array([[1 / a[0], t], [t, 1 / a[1]]])
            expect += mult * np.linalg.solve(m, np.ones(2)) / 3.0
        got = scs.screened_polarizability(s, u, pairs, s.damp_cut)
        assert np.max(np.abs(got - expect) / expect) < 1e-12


def _periodic_system(seed=11, n=6, box=9.0):
    rng = np.random.default_rng(seed)
    while True:
        pos = rng.uniform(0, box, size=(n, 3))
        diff = pos[:, None] - pos[None]
        diff -= box * np.round(diff / box)
        dist = np.sqrt(np.sum(diff ** 2, -1)) + np.eye(n) * 99
        if dist.min() > 2.2:
            break
    return _system(pos, np.eye(3) * box, rng.uniform(4, 12, n), rng.uniform(0.3, 0.7, n), rng.uniform(3.0, 3.8, n),
                   damp_cut=11.0)


def test_supercell_copies_get_the_same_screening():
    s = _periodic_system()
    out = scs.scs(s, n_freq=8)
    n = s.pos.shape[0]
    shifts = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float) * s.cell[0, 0]
    big = _system(np.concatenate([s.pos + sh for sh in shifts]), s.cell * 2, np.tile(s.alpha, 8),
                  np.tile(s.omega, 8), np.tile(s.r_vdw, 8), damp_cut=s.damp_cut)
    out2 = scs.scs(big, n_freq=8)
    for key in ("alpha", "omega", "c6", "r_vdw"):
        assert np.max(np.abs(out2[key] - np.tile(out[key], 8)) / np.abs(np.tile(out[key], 8))) < 1e-11
    assert np.max(np.abs(out["alpha"] - s.alpha) / s.alpha) > 1e-3        # the images do screen


def test_translation_and_permutation_invariance():
    s = _periodic_system(seed=12)
    out = scs.scs(s, n_freq=6)
    moved = s.with_(pos=s.pos + np.array([3.3, -1.7, 8.1]))
    assert np.allclose(scs.scs(moved, n_freq=6)["alpha"], out["alpha"], rtol=1e-12, atol=0)
    perm = np.random.default_rng(1).permutation(s.pos.shape[0])
    sp_ = s.with_(pos=s.pos[perm], alpha=s.alpha[perm], omega=s.omega[perm], r_vdw=s.r_vdw[perm])
    o2 = scs.scs(sp_, n_freq=6)
    for key in ("alpha", "omega", "r_vdw"):
        assert np.allclose(o2[key], out[key][perm], rtol=1e-12, atol=0)


def test_screened_radius_follows_the_cube_root_of_the_polarisability():
    s = _periodic_system(seed=13)
    out = scs.scs(s, n_freq=6)
    assert np.allclose(out["r_vdw"] ** 3 / out["alpha"], s.r_vdw ** 3 / s.alpha, rtol=1e-13, atol=0)


def test_sparse_cg_solve_matches_the_dense_solve():
    s = _periodic_system(seed=14, n=8, box=10.0)
    dense = scs.scs(s, n_freq=5)
    it = scs.scs(s, n_freq=5, solver="cg")
    for key in ("alpha", "omega", "c6"):
        assert np.max(np.abs(it[key] - dense[key]) / np.abs(dense[key])) < 1e-11
