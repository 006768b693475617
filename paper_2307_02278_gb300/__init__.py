"""GB300-native SPME stochastic-Lanczos MBD (arXiv 2307.02278).

The compute path is libmbd.so (hand-written CUDA for sm_103a, C ABI in
include/mbd.h); this package only marshals arguments to it.
"""
from ._abi import (MBD_FP64, MBD_MIXED, MBD_TERM_ALL, MBD_TERM_REAL, MBD_TERM_RECIP, MBD_TERM_SELF,  # noqa: F401
                   MBDError, lib)
from .system import (MBDBatch, MBDSystem, generate_probes, lanczos_energy_dense, mesh_for_density,  # noqa: F401
                     spme_params, tridiag_functions, tridiag_quadrature)
from .autograd import MBDEnergy, mbd_energy  # noqa: F401
