"""Python binding of libmbd: the calls of include/mbd.h with the same names.

PyTorch supplies device memory and the stream; every step of the method runs
in the library's CUDA kernels.  Vectors cross the boundary as FP64 CUDA tensors
of layout [nvec][N][3] (or [nvec][3N]).
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int32, c_uint64, c_void_p

import numpy as np
import torch

from ._abi import (MBD_ERR_UNSUPPORTED, MBD_FP64, MBD_MIXED, MBD_QUAD_CHEBYSHEV, MBD_QUAD_QL, MBD_QUAD_QL_DF64,
                   MBD_TERM_ALL, STAGES, BatchInfo, Info, Profile, SystemDesc, check, lib)

PRECISIONS = {"fp64": MBD_FP64, "mixed": MBD_MIXED}
QUADRATURE = {"chebyshev": MBD_QUAD_CHEBYSHEV, "ql": MBD_QUAD_QL, "ql_df64": MBD_QUAD_QL_DF64}


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(c_double))


def _cuda_f64(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    return t.contiguous()


def _make_desc(cell, pos, alpha, omega, r_vdw, *, damp_beta=0.83, damp_d=6.0, ewald_beta=0.35, r_cut=10.0,
               damp_cut=0.0, mesh=(32, 32, 32), spline_order=6, precision="fp64", quadrature="chebyshev"):
    """An mbd_system_desc and the host arrays it points to (keep them alive while it is used)."""
    keep = [np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3),
            np.ascontiguousarray(alpha, dtype=np.float64), np.ascontiguousarray(omega, dtype=np.float64),
            np.ascontiguousarray(r_vdw, dtype=np.float64)]
    d = SystemDesc()
    d.n_atoms = int(keep[0].shape[0])
    d.cell[:] = [float(x) for x in np.asarray(cell, dtype=np.float64).ravel()]
    d.pos, d.alpha, d.omega, d.r_vdw = (_dptr(x) for x in keep)
    d.damp_beta, d.damp_d, d.ewald_beta = float(damp_beta), float(damp_d), float(ewald_beta)
    d.r_cut, d.damp_cut = float(r_cut), float(damp_cut)
    d.mesh[:] = [int(k) for k in mesh]
    d.spline_order = int(spline_order)
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    d.quadrature = QUADRATURE[quadrature] if isinstance(quadrature, str) else int(quadrature)
    return d, keep


def _workload_kw(s) -> dict:
    return dict(damp_beta=s.damp_beta, damp_d=s.damp_d, ewald_beta=s.ewald_beta, r_cut=s.r_cut,
                damp_cut=s.damp_cut, mesh=s.mesh, spline_order=s.spline_order)


def _stream(stream):
    if stream is None and torch.cuda.is_available():
        stream = torch.cuda.current_stream()
    return stream


def _stream_handle(stream):
    return c_void_p(stream.cuda_stream if stream is not None else 0)


class MBDSystem:
    """One periodic system on the GPU (mbd_create_system)."""

    def __init__(self, cell, pos, alpha, omega, r_vdw, *, damp_beta=0.83, damp_d=6.0, ewald_beta=0.35,
                 r_cut=10.0, damp_cut=0.0, mesh=(32, 32, 32), spline_order=6, precision="fp64",
                 quadrature="chebyshev", stream=None):
        self._handle = None
        d, self._keep = _make_desc(cell, pos, alpha, omega, r_vdw, damp_beta=damp_beta, damp_d=damp_d,
                                   ewald_beta=ewald_beta, r_cut=r_cut, damp_cut=damp_cut, mesh=mesh,
                                   spline_order=spline_order, precision=precision,
                                   quadrature=quadrature)
        self.n_atoms = d.n_atoms
        self._pos = self._keep[0]
        self.precision = precision
        self.stream = _stream(stream)
        out = c_void_p()
        check(lib().mbd_create_system(byref(d), _stream_handle(self.stream), byref(out)), "mbd_create_system")
        self._handle = out

    @classmethod
    def from_workload(cls, s, precision="fp64", **kw):
        """Build from a workloads.System-like object (attributes of the same names)."""
        return cls(s.cell, s.pos, s.alpha, s.omega, s.r_vdw, precision=precision, **_workload_kw(s), **kw)

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if self._handle is not None:
            lib().mbd_destroy_system(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ calls
    def update_positions(self, pos):
        self._pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
        check(lib().mbd_update_positions(self._handle, _dptr(self._pos)), "mbd_update_positions")

    def info(self) -> dict:
        inf = Info()
        check(lib().mbd_get_info(self._handle, byref(inf)), "mbd_get_info")
        return dict(n_atoms=inf.n_atoms, mesh=tuple(inf.mesh), n_pairs=inf.n_pairs,
                    device_bytes=inf.device_bytes, precision=inf.precision)

    def profile_enable(self, timing: bool = True):
        """Reset the per-stage counters; with timing, bracket stages with CUDA events."""
        check(lib().mbd_profile_enable(self._handle, 1 if timing else 0), "mbd_profile_enable")

    def profile_read(self) -> dict:
        """{stage: (launches, device ms)} plus 'total_launches'."""
        p = Profile()
        check(lib().mbd_profile_read(self._handle, byref(p)), "mbd_profile_read")
        out = {name: (int(p.launches[k]), float(p.ms[k])) for k, name in enumerate(STAGES)}
        out["total_launches"] = int(p.total_launches)
        return out

    def set_basis_storage(self, mode: str):
        """mbd_set_basis_storage: "store" (all m Lanczos vectors) or "recompute"
        (three kept; the forces rerun the recurrence)."""
        code = {"store": 0, "recompute": 1}[mode]
        check(lib().mbd_set_basis_storage(self._handle, code), "mbd_set_basis_storage")

    def set_real_space_method(self, method: str):
        """mbd_set_real_space_method: "auto", "clusters" or "pairs"."""
        code = {"auto": 0, "clusters": 1, "pairs": 2}[method]
        check(lib().mbd_set_real_space_method(self._handle, code), "mbd_set_real_space_method")

    _CHOICE_KEYS = ("ld", "field_atoms_per_block", "fft_tile", "spread_tile")

    def autotune(self, n_probes: int) -> dict:
        """mbd_autotune: time the launch choices at n_probes probes, keep the fastest."""
        out = (c_int32 * 4)()
        check(lib().mbd_autotune(self._handle, int(n_probes), out), "mbd_autotune")
        return dict(zip(self._CHOICE_KEYS, list(out)))

    def set_launch_choices(self, choices: dict | None) -> None:
        """mbd_set_launch_choices: apply choices in the form autotune returns
        (missing keys keep the built-in rule); None returns to the rules."""
        c = (c_int32 * 4)()
        if choices is not None:
            for i, k in enumerate(self._CHOICE_KEYS):
                c[i] = int(choices.get(k, 0))
        check(lib().mbd_set_launch_choices(self._handle, c), "mbd_set_launch_choices")

    def apply_C(self, x: torch.Tensor) -> torch.Tensor:
        """y = C x for x of shape [nvec, 3N] (or [3N])."""
        x = _cuda_f64(x, "x")
        one = x.dim() == 1
        xb = x.reshape(1 if one else x.shape[0], -1)
        y = torch.empty_like(xb)
        check(lib().mbd_apply_C(self._handle, xb.shape[0], xb.data_ptr(), y.data_ptr()), "mbd_apply_C")
        return y[0] if one else y

    def field(self, d: torch.Tensor, terms: int = MBD_TERM_ALL) -> torch.Tensor:
        """E = T'^pbc d restricted to `terms`, d of shape [nvec, N, 3]."""
        d = _cuda_f64(d, "d")
        e = torch.empty_like(d)
        check(lib().mbd_field(self._handle, d.shape[0], d.data_ptr(), e.data_ptr(), int(terms)), "mbd_field")
        return e

    def spread(self, d: torch.Tensor, mesh) -> torch.Tensor:
        d = _cuda_f64(d, "d")
        out = torch.empty((d.shape[0],) + tuple(mesh), dtype=torch.float64, device=d.device)
        check(lib().mbd_spread(self._handle, d.shape[0], d.data_ptr(), out.data_ptr()), "mbd_spread")
        return out

    def convolve(self, q: torch.Tensor) -> torch.Tensor:
        q = _cuda_f64(q, "mesh")
        out = torch.empty_like(q)
        check(lib().mbd_convolve(self._handle, q.shape[0], q.data_ptr(), out.data_ptr()), "mbd_convolve")
        return out

    def lanczos_energy(self, n_probes: int, n_steps: int, seed: int, details: bool = False):
        """E_MBD by stochastic Lanczos quadrature; with details also the trace,
        the per-probe quadratures q [R] and the tridiagonals a, b [R, m]."""
        e = c_double()
        tr = c_double()
        q = np.zeros(n_probes) if details else None
        ab = np.zeros((n_probes, 2, n_steps)) if details else None
        check(lib().mbd_lanczos_energy(self._handle, n_probes, n_steps, seed, byref(e), byref(tr),
                                       _dptr(q) if details else None, _dptr(ab) if details else None),
              "mbd_lanczos_energy")
        if not details:
            return e.value
        return e.value, dict(trace=tr.value, q=q, a=ab[:, 0], b=ab[:, 1])

    def energy_forces(self, n_probes: int, n_steps: int, seed: int, forces: torch.Tensor | None = None):
        """(E_MBD, F) with F = -dE/dR as a CUDA float64 tensor [N, 3]."""
        if forces is None:
            forces = torch.empty((self.n_atoms, 3), dtype=torch.float64, device="cuda")
        forces = _cuda_f64(forces, "forces")
        e = c_double()
        check(lib().mbd_energy_forces(self._handle, n_probes, n_steps, seed, byref(e), forces.data_ptr()),
              "mbd_energy_forces")
        return e.value, forces

    def scs_screen(self, n_freq: int = 23, tol: float = 1e-10, max_iter: int = 200) -> dict:
        """Screened alpha, omega, R_vdw and C6 per atom (mbd_scs_screen), with
        alpha^SCS at every frequency [n_freq + 1, N] (static first), the
        iterations taken and the largest relative residual."""
        n = self.n_atoms
        out = {k: np.zeros(n) for k in ("alpha", "omega", "r_vdw", "c6")}
        aiu = np.zeros((n_freq + 1, n))
        it = ctypes.c_int32()
        res = c_double()
        check(lib().mbd_scs_screen(self._handle, n_freq, tol, max_iter, _dptr(out["alpha"]), _dptr(out["omega"]),
                                   _dptr(out["r_vdw"]), _dptr(out["c6"]), _dptr(aiu), byref(it), byref(res)),
              "mbd_scs_screen")
        out.update(alpha_iu=aiu, iterations=it.value, residual=res.value)
        return out


class MBDBatch:
    """Independent periodic systems of uneven sizes run together (mbd_create_batch):
    every member's Lanczos run is one branch of a CUDA graph recorded on the first
    call with a given (n_probes, n_steps) and replayed afterwards."""

    def __init__(self, systems, precision="mixed", quadrature="chebyshev", stream=None):
        self._handle = None
        descs = (SystemDesc * len(systems))()
        self._keep = []
        for i, s in enumerate(systems):
            d, keep = _make_desc(s.cell, s.pos, s.alpha, s.omega, s.r_vdw, precision=precision,
                                 quadrature=quadrature, **_workload_kw(s))
            descs[i] = d
            self._keep.append(keep)
        self.n_sys = len(systems)
        self.stream = _stream(stream)
        out = c_void_p()
        check(lib().mbd_create_batch(self.n_sys, descs, _stream_handle(self.stream), byref(out)),
              "mbd_create_batch")
        self._handle = out

    def close(self):
        if self._handle is not None:
            lib().mbd_destroy_batch(self._handle)
            self._handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def info(self) -> dict:
        i = BatchInfo()
        check(lib().mbd_batch_get_info(self._handle, byref(i)), "mbd_batch_get_info")
        return dict(n_sys=i.n_sys, graph_kernels=i.graph_kernels, total_atoms=i.total_atoms)

    def lanczos_energy(self, n_probes: int, n_steps: int, seeds):
        """(energies [n_sys], traces [n_sys]) with member i on seeds[i]."""
        sd = np.ascontiguousarray(seeds, dtype=np.uint64)
        if sd.shape != (self.n_sys,):
            raise ValueError(f"seeds must have shape ({self.n_sys},)")
        e = np.zeros(self.n_sys)
        t = np.zeros(self.n_sys)
        bad = c_int32(-1)
        code = lib().mbd_batch_lanczos_energy(self._handle, n_probes, n_steps,
                                              sd.ctypes.data_as(ctypes.POINTER(c_uint64)), _dptr(e), _dptr(t),
                                              byref(bad))
        where = "mbd_batch_lanczos_energy" + (f" (member {bad.value})" if bad.value >= 0 else "")
        check(code, where)
        return e, t


def mesh_for_density(cell, points_per_bohr: float = 0.0, spline_order: int = 6) -> tuple:
    """mbd_mesh_for_density: the smooth mesh at a density of points per bohr
    along each cell vector (<= 0: the paper's 1.2 points per angstrom)."""
    c = np.ascontiguousarray(np.asarray(cell, dtype=np.float64).ravel())
    out = (c_int32 * 3)()
    check(lib().mbd_mesh_for_density(c.ctypes.data_as(ctypes.POINTER(c_double)), float(points_per_bohr),
                                     int(spline_order), out), "mbd_mesh_for_density")
    return tuple(int(k) for k in out)


def spme_params(s, tol: float, spline_order: int | None = None, r_cut_max: float = 0.0) -> dict:
    """mbd_spme_params for a workloads.System-like object: the Ewald splitting,
    cutoffs and mesh for a target relative accuracy of the field; 'ok' is False
    when the cell is too small for the damping correction to reach it."""
    kw = _workload_kw(s)
    if spline_order is not None:
        kw["spline_order"] = spline_order
    kw["r_cut"] = r_cut_max
    d, keep = _make_desc(s.cell, s.pos, s.alpha, s.omega, s.r_vdw, **kw)
    est = c_double()
    code = lib().mbd_spme_params(byref(d), float(tol), byref(est))
    if code != MBD_ERR_UNSUPPORTED:
        check(code, "mbd_spme_params")
    return dict(ewald_beta=d.ewald_beta, r_cut=d.r_cut, damp_cut=d.damp_cut, mesh=tuple(int(k) for k in d.mesh),
                spline_order=int(d.spline_order), est_err=est.value, ok=code != MBD_ERR_UNSUPPORTED)


def generate_probes(seed: int, n_probes: int, dim: int, first: int = 0) -> torch.Tensor:
    v = torch.empty((n_probes, dim), dtype=torch.float64, device="cuda")
    check(lib().mbd_generate_probes(seed, first, n_probes, dim, v.data_ptr()), "mbd_generate_probes")
    return v


def tridiag_functions(a: np.ndarray, b: np.ndarray, method: str = "chebyshev"):
    """mbd_tridiag_functions: (q [R], c [R, m]) = (e1^T Delta^{1/2} e1, Delta^{-1/2} e1) per probe."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    q = np.zeros(a.shape[0])
    c = np.zeros(a.shape)
    check(lib().mbd_tridiag_functions(a.shape[0], a.shape[1], _dptr(a), _dptr(b), QUADRATURE[method], _dptr(q),
                                      _dptr(c)), "mbd_tridiag_functions")
    return q, c


def tridiag_quadrature(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    q = np.zeros(a.shape[0])
    check(lib().mbd_tridiag_quadrature(a.shape[0], a.shape[1], _dptr(a), _dptr(b), _dptr(q)),
          "mbd_tridiag_quadrature")
    return q


def lanczos_energy_dense(c: torch.Tensor, omega_sum: float, n_probes: int, n_steps: int, seed: int):
    c = _cuda_f64(c, "C")
    e = c_double()
    q = np.zeros(n_probes)
    ab = np.zeros((n_probes, 2, n_steps))
    check(lib().mbd_lanczos_energy_dense(c.shape[0], c.data_ptr(), float(omega_sum), n_probes, n_steps, seed,
                                         byref(e), _dptr(q), _dptr(ab)), "mbd_lanczos_energy_dense")
    return e.value, dict(q=q, a=ab[:, 0], b=ab[:, 1])
