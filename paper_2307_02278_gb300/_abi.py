"""ctypes declarations of the C ABI in include/mbd.h (argument marshalling only).

The shared library is built in-tree by paper_2307_02278_gb300/build.py; loading
fails loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_uint64, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbd.so")

MBD_OK = 0
STATUS = {
    0: "MBD_OK", 1: "MBD_ERR_INVALID_ARG", 2: "MBD_ERR_OOM", 3: "MBD_ERR_CUDA",
    4: "MBD_ERR_NOT_POSITIVE_DEFINITE", 5: "MBD_ERR_NONFINITE", 6: "MBD_ERR_TIMEOUT",
    7: "MBD_ERR_UNSUPPORTED", 8: "MBD_ERR_NO_DEVICE",
}
MBD_FP64, MBD_MIXED = 0, 1
MBD_QUAD_CHEBYSHEV, MBD_QUAD_QL_DF64, MBD_QUAD_QL = 0, 1, 2
MBD_TERM_REAL, MBD_TERM_RECIP, MBD_TERM_SELF, MBD_TERM_ALL = 1, 2, 4, 7
MBD_ERR_UNSUPPORTED = 7
MBD_BASIS_STORE, MBD_BASIS_RECOMPUTE = 0, 1
MBD_DEFAULT_MESH_DENSITY = 1.2 / 1.8897261254578281     # points per bohr (1.2 per angstrom)


class SystemDesc(ctypes.Structure):
    _fields_ = [
        ("n_atoms", c_int32),
        ("cell", c_double * 9),
        ("pos", POINTER(c_double)),
        ("alpha", POINTER(c_double)),
        ("omega", POINTER(c_double)),
        ("r_vdw", POINTER(c_double)),
        ("damp_beta", c_double),
        ("damp_d", c_double),
        ("ewald_beta", c_double),
        ("r_cut", c_double),
        ("damp_cut", c_double),
        ("mesh", c_int32 * 3),
        ("spline_order", c_int32),
        ("precision", c_int32),
        ("quadrature", c_int32),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("n_atoms", c_int32),
        ("mesh", c_int32 * 3),
        ("n_pairs", c_int64),
        ("device_bytes", c_int64),
        ("precision", c_int32),
    ]


NUM_STAGES = 11
STAGES = ["prologue", "spread", "fft", "field", "quadrature", "force_prep", "force_spread", "force_fft",
          "force_gather", "other", "real"]


class Profile(ctypes.Structure):
    _fields_ = [
        ("launches", c_int64 * NUM_STAGES),
        ("ms", c_double * NUM_STAGES),
        ("total_launches", c_int64),
    ]


class BatchInfo(ctypes.Structure):
    _fields_ = [
        ("n_sys", c_int32),
        ("graph_kernels", c_int64),
        ("total_atoms", c_int64),
    ]


class MBDError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        self.name = STATUS.get(code, f"status {code}")
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


_LIB = None

PD = POINTER(c_double)
SIGNATURES = {
    "mbd_create_system": (c_int, [POINTER(SystemDesc), c_void_p, POINTER(c_void_p)]),
    "mbd_destroy_system": (None, [c_void_p]),
    "mbd_update_positions": (c_int, [c_void_p, PD]),
    "mbd_apply_C": (c_int, [c_void_p, c_int32, c_void_p, c_void_p]),
    "mbd_lanczos_energy": (c_int, [c_void_p, c_int32, c_int32, c_uint64, PD, PD, PD, PD]),
    "mbd_energy_forces": (c_int, [c_void_p, c_int32, c_int32, c_uint64, PD, c_void_p]),
    "mbd_scs_screen": (c_int, [c_void_p, c_int32, c_double, c_int32, PD, PD, PD, PD, PD, POINTER(c_int32), PD]),
    "mbd_set_basis_storage": (c_int, [c_void_p, c_int32]),
    "mbd_autotune": (c_int, [c_void_p, c_int32, POINTER(c_int32)]),
    "mbd_set_launch_choices": (c_int, [c_void_p, POINTER(c_int32)]),
    "mbd_mesh_for_density": (c_int, [POINTER(c_double), c_double, c_int32, POINTER(c_int32)]),
    "mbd_spme_params": (c_int, [POINTER(SystemDesc), c_double, PD]),
    "mbd_create_batch": (c_int, [c_int32, POINTER(SystemDesc), c_void_p, POINTER(c_void_p)]),
    "mbd_destroy_batch": (None, [c_void_p]),
    "mbd_batch_lanczos_energy": (c_int, [c_void_p, c_int32, c_int32, POINTER(c_uint64), PD, PD, POINTER(c_int32)]),
    "mbd_batch_get_info": (c_int, [c_void_p, POINTER(BatchInfo)]),
    "mbd_generate_probes": (c_int, [c_uint64, c_int32, c_int32, c_int32, c_void_p]),
    "mbd_field": (c_int, [c_void_p, c_int32, c_void_p, c_void_p, c_int32]),
    "mbd_spread": (c_int, [c_void_p, c_int32, c_void_p, c_void_p]),
    "mbd_convolve": (c_int, [c_void_p, c_int32, c_void_p, c_void_p]),
    "mbd_tridiag_quadrature": (c_int, [c_int32, c_int32, PD, PD, PD]),
    "mbd_tridiag_functions": (c_int, [c_int32, c_int32, PD, PD, c_int32, PD, PD]),
    "mbd_tridiag_quadrature_noalloc": (c_int, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    "mbd_lanczos_energy_dense": (c_int, [c_int32, c_void_p, c_double, c_int32, c_int32, c_uint64, PD, PD, PD]),
    "mbd_get_info": (c_int, [c_void_p, POINTER(Info)]),
    "mbd_profile_enable": (c_int, [c_void_p, c_int32]),
    "mbd_profile_read": (c_int, [c_void_p, POINTER(Profile)]),
    "mbd_debug_fail_allocation": (c_int, [c_int64]),
    "mbd_set_real_space_method": (c_int, [c_void_p, c_int32]),
    "mbd_status_string": (c_char_p, [c_int]),
    "mbd_last_error": (c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """The loaded libmbd; raises if the library has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2307_02278_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = handle
    return _LIB


def check(code: int, where: str) -> None:
    if code != MBD_OK:
        detail = lib().mbd_last_error().decode()
        raise MBDError(code, where, detail)
