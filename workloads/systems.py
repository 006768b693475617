"""Seeded synthetic periodic systems shaped like the paper's test systems.

The paper measures liquid-water boxes and a diamond crystal (Numerical results
section); their coordinates and MBD parameters are not published, so these
generators stand in for them with seeded synthetic boxes of the same shape:
water-like boxes at 1 g/cm^3 built from rigid triatomic molecules, and boxes of
random atoms with a minimum separation.

This module is shared by the tests, the benchmark and the oracle-side checks.
It samples geometry and per-atom parameters only; it holds none of the MBD
arithmetic (no damping, no dipole tensor, no Ewald or Lanczos step).
All lengths are in bohr, polarizabilities in bohr^3, frequencies in hartree.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np
from scipy.spatial import cKDTree

# Liquid water at 1 g/cm^3: 33.43 molecules/nm^3 -> 0.004954 molecules/bohr^3,
# i.e. 0.01486 atoms/bohr^3.
WATER_MOLECULE_DENSITY = 0.0049535
WATER_ATOM_DENSITY = 3 * WATER_MOLECULE_DENSITY
OH_BOND = 1.81                      # bohr
HOH_ANGLE = np.deg2rad(104.5)
MIN_SEPARATION = 2.5                # bohr, between atoms of different molecules


@dataclass
class System:
    """One periodic MBD problem: geometry, per-atom parameters, method settings."""
    name: str
    cell: np.ndarray            # (3,3) rows a1, a2, a3 (bohr)
    pos: np.ndarray             # (N,3) Cartesian (bohr)
    alpha: np.ndarray           # (N,) static polarizability (bohr^3)
    omega: np.ndarray           # (N,) characteristic frequency (Ha)
    r_vdw: np.ndarray           # (N,) vdW radius (bohr)
    damp_beta: float = 0.83     # Fermi damping range-separation parameter
    damp_d: float = 6.0         # Fermi damping steepness
    ewald_beta: float = 0.35    # Ewald splitting parameter (bohr^-1)
    r_cut: float = 10.0         # real-space erfc cutoff (bohr)
    damp_cut: float = 10.0      # cutoff of the short-range damping correction (bohr)
    mesh: tuple = (32, 32, 32)
    spline_order: int = 6
    n_probes: int = 16
    n_steps: int = 30
    probe_seed: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    def with_(self, **kw) -> "System":
        return replace(self, **kw)


def smooth_size(n: float) -> int:
    """Smallest integer >= n whose only prime factors are 2, 3 and 5."""
    k = max(1, int(np.ceil(n - 1e-9)))
    while True:
        m = k
        for f in (2, 3, 5):
            while m % f == 0:
                m //= f
        if m == 1:
            return k
        k += 1


def _resolve_close_pairs(rng, pos, box, groups, resample, max_rounds=200):
    """Re-sample groups (atoms or molecules) until no pair of atoms from
    different groups is closer than MIN_SEPARATION (periodic cubic box)."""
    for _ in range(max_rounds):
        tree = cKDTree(np.mod(pos, box), boxsize=box)
        pairs = tree.query_pairs(MIN_SEPARATION, output_type="ndarray")
        if pairs.size:
            pairs = pairs[groups[pairs[:, 0]] != groups[pairs[:, 1]]]
        if pairs.size == 0:
            return pos
        bad = np.unique(groups[pairs[:, 1]])
        pos = resample(rng, pos, bad)
    raise RuntimeError("could not reach the minimum separation")


def random_box(n_atoms: int, box: float, seed: int) -> np.ndarray:
    """Uniform random positions in a cubic box with pairwise distance >= 2.5 bohr."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(0.0, box, size=(n_atoms, 3))

    def resample(rng, pos, bad):
        pos = pos.copy()
        pos[bad] = rng.uniform(0.0, box, size=(bad.size, 3))
        return pos

    return _resolve_close_pairs(rng, pos, box, np.arange(n_atoms), resample)


def _random_rotations(rng, n):
    """Uniform random rotation matrices from unit quaternions (n,3,3)."""
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], axis=1)


def water_box(n_mol: int, seed: int, box: float | None = None) -> tuple[np.ndarray, np.ndarray, float]:
    """n_mol rigid water molecules: O on a jittered cubic lattice (+-0.5 bohr; when
    n_mol is not a cube, a seeded subset of the smallest lattice that holds it),
    random orientations, intermolecular atoms >= 2.5 bohr apart.
    Returns (positions (3M,3) ordered O,H,H per molecule, element codes 0=O 1=H, box)."""
    n_side = int(np.ceil(n_mol ** (1.0 / 3.0) - 1e-9))
    if box is None:
        box = (n_mol / WATER_MOLECULE_DENSITY) ** (1.0 / 3.0)
    rng = np.random.Generator(np.random.PCG64(seed))
    a = box / n_side
    grid = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    if grid.shape[0] > n_mol:
        grid = grid[np.sort(rng.permutation(grid.shape[0])[:n_mol])]
    oxy = (grid + 0.5) * a + rng.uniform(-0.5, 0.5, size=(n_mol, 3))
    half = 0.5 * HOH_ANGLE
    local = np.array([[0.0, 0.0, 0.0],
                      [OH_BOND * np.sin(half), 0.0, OH_BOND * np.cos(half)],
                      [-OH_BOND * np.sin(half), 0.0, OH_BOND * np.cos(half)]])

    def place(rot, o):
        return o[:, None, :] + np.einsum("mij,aj->mai", rot, local)

    mol = place(_random_rotations(rng, n_mol), oxy).reshape(-1, 3)

    def resample(rng, pos, bad):
        pos = pos.reshape(n_mol, 3, 3).copy()
        pos[bad] = place(_random_rotations(rng, bad.size), pos[bad, 0, :])
        return pos.reshape(-1, 3)

    groups = np.repeat(np.arange(n_mol), 3)
    mol = _resolve_close_pairs(rng, mol, box, groups, resample)
    elem = np.tile(np.array([0, 1, 1]), n_mol)
    return np.mod(mol, box), elem, box


def _water_params(elem, seed):
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    alpha = np.where(elem == 0, 5.4, 2.5) * rng.uniform(0.9, 1.1, size=elem.size)
    omega = np.where(elem == 0, 0.45, 0.55).astype(float)
    r_vdw = np.where(elem == 0, 3.2, 3.1).astype(float)
    return alpha, omega, r_vdw


def _random_params(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    alpha = rng.uniform(5.0, 15.0, size=n)
    omega = rng.uniform(0.3, 0.6, size=n)
    r_vdw = rng.uniform(3.0, 4.0, size=n)
    return alpha, omega, r_vdw


def random_system(n_atoms: int, box: float, seed: int, mesh=None, **kw) -> System:
    """Random-position box with the parameter distributions of the 64-atom case."""
    pos = random_box(n_atoms, box, seed)
    alpha, omega, r_vdw = _random_params(n_atoms, seed)
    if mesh is None:
        k = smooth_size(box)
        mesh = (k, k, k)
    return System(name=kw.pop("name", f"random{n_atoms}"), cell=np.eye(3) * box, pos=pos,
                  alpha=alpha, omega=omega, r_vdw=r_vdw, mesh=tuple(mesh), **kw)


def water_system(n_mol: int, seed: int, mesh=None, box=None, **kw) -> System:
    pos, elem, box = water_box(n_mol, seed, box)
    alpha, omega, r_vdw = _water_params(elem, seed)
    if mesh is None:
        k = smooth_size(box)
        mesh = (k, k, k)
    return System(name=kw.pop("name", f"water{3 * n_mol}"), cell=np.eye(3) * box, pos=pos,
                  alpha=alpha, omega=omega, r_vdw=r_vdw, mesh=tuple(mesh),
                  meta={"elements": elem}, **kw)


# Diamond: conventional cubic cell (8 atoms), lattice constant 3.567 angstrom;
# carbon free-atom polarizability, C6 and vdW radius of the Tkatchenko-Scheffler
# reference set (12.0 bohr^3, 46.6 Ha bohr^6, 3.59 bohr), omega = 4 C6 / (3 alpha^2).
ANGSTROM = 1.8897261254578281      # bohr
DIAMOND_A = 3.567 * ANGSTROM
CARBON_ALPHA, CARBON_C6, CARBON_RVDW = 12.0, 46.6, 3.59


def diamond_system(n_cells: int = 4, seed: int = 0, jitter: float = 0.0, mesh=None, **kw) -> System:
    """n_cells^3 conventional diamond cells (8 n_cells^3 atoms, 512 for n_cells = 4,
    a 14.27 angstrom box), optionally with seeded Gaussian displacements."""
    frac = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=float)
    frac = np.concatenate([frac, frac + 0.25])
    cells = np.stack(np.meshgrid(*[np.arange(n_cells)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = ((cells[:, None, :] + frac[None, :, :]).reshape(-1, 3)) * DIAMOND_A
    if jitter > 0.0:
        pos = pos + np.random.Generator(np.random.PCG64(seed)).normal(scale=jitter, size=pos.shape)
    box = n_cells * DIAMOND_A
    n = pos.shape[0]
    alpha = np.full(n, CARBON_ALPHA)
    omega = np.full(n, 4.0 * CARBON_C6 / (3.0 * CARBON_ALPHA ** 2))
    r_vdw = np.full(n, CARBON_RVDW)
    if mesh is None:
        k = smooth_size(box)
        mesh = (k, k, k)
    return System(name=kw.pop("name", f"diamond{n}"), cell=np.eye(3) * box, pos=np.mod(pos, box), alpha=alpha,
                  omega=omega, r_vdw=r_vdw, mesh=tuple(mesh), **kw)


# Ewald split of the water boxes.  The 64-atom box uses beta = 0.35 bohr^-1 and
# r_cut = 10 bohr as given; the water boxes give a mesh but no split.  With
# 0.35/10 the 64^3 mesh of the 3000-atom box leaves the SPME product C x
# 1.6e-5 (relative L2) from the same-split direct Ewald sum, above the 1e-5
# bound.  beta = 0.30 moves the mesh error to 4.1e-6 there (the error goes as
# (beta h)^p), and the 192^3 mesh of the 100,002-atom box (h = 0.98 bohr
# against 0.92) stays near 6e-6.  r_cut = 12 keeps the erfc tail
# 2 exp(-(beta r_cut)^2) at 4.7e-6; the damping correction is cut at the same
# radius (one neighbour list).
WATER_EWALD_BETA = 0.30
WATER_R_CUT = 12.0


# The five workloads.  Geometry seed 1000+c, probe seed 2307022780+c.
def config(c: int, variant: str = "") -> System:
    probe_seed = 2307022780 + c
    if c == 1:
        # 64 random atoms, L = 24 bohr, mesh 32^3, 16 probes x 30 steps, FP64
        return random_system(64, 24.0, 1001, mesh=(32, 32, 32), n_probes=16, n_steps=30,
                             probe_seed=probe_seed, name="random64_L24_mesh32")
    split = dict(ewald_beta=WATER_EWALD_BETA, r_cut=WATER_R_CUT, damp_cut=WATER_R_CUT)
    if c == 2:
        # 1000 water molecules (3000 atoms), L = 58.66 bohr, mesh 64^3, 64 probes x 50 steps
        return water_system(1000, 1002, mesh=(64, 64, 64), n_probes=64, n_steps=50,
                            probe_seed=probe_seed, name="water3000_L58.7_mesh64", **split)
    if c == 3:
        # 8000 molecules (24,000 atoms), L = 117.3 bohr, mesh 128^3, 128 probes x 60 steps
        return water_system(8000, 1003, mesh=(128, 128, 128), n_probes=128, n_steps=60,
                            probe_seed=probe_seed, name="water24000_L117.3_mesh128", **split)
    if c == 5:
        if variant == "fd":
            # 4000 molecules (12,000 atoms), L = 93.1 bohr, mesh 96^3
            return water_system(4000, 1005, mesh=(96, 96, 96), n_probes=64, n_steps=60,
                                probe_seed=probe_seed, name="water12000_L93.1_mesh96", **split)
        # 33,334 molecules (100,002 atoms) at water density, L = 188.8 bohr,
        # mesh 192^3, 64 probes x 60 steps
        return water_system(33334, 1005, mesh=(192, 192, 192), n_probes=64, n_steps=60,
                            probe_seed=probe_seed, name="water100002_L188.8_mesh192", **split)
    raise ValueError(f"unknown config {c}")


def batch_systems(n_sys: int = 64, seed: int = 1004, n_min: int = 200, n_max: int = 20000):
    """Uneven batch: N log-uniform in [n_min, n_max] random atoms at water atom
    density; mesh at ~1 bohr spacing rounded up to 2^a 3^b 5^c; 32 probes x 40 steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.round(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=n_sys))).astype(int)
    out = []
    for s, n in enumerate(ns):
        box = (n / WATER_ATOM_DENSITY) ** (1.0 / 3.0)
        k = smooth_size(box)
        out.append(random_system(int(n), box, seed * 100 + s, mesh=(k, k, k), n_probes=32,
                                 n_steps=40, probe_seed=2307022784 + s, name=f"batch{s}_N{n}"))
    return out
