"""Plain FP64 CPU oracle for the SPME stochastic-Lanczos MBD hot path.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library
(``paper_2307_02278_gb300``) and never imports it.

Layout (each function cites the passage of arXiv 2307.02278 it follows):
  model.py     MBD quantities: damping s(R), dipole tensor T, g vector (Eqs. ham, vmbd, gvec)
  ewald.py     exact periodic dipole field T'^pbc d by direct Ewald summation, tin-foil
               boundary (Eqs. ewalddip, fld_ewald, fld_ewald1, structurefactor, fld_ewald2)
  spme.py      SPME reciprocal field: B-splines, spreading, FFT convolution, gather
               (Eqs. scaledfractional, spme, dipolarr)
  operator.py  C = Omega + Diag(g) T' Diag(g) applied matrix-free or built densely (Eqs. ccd, lk3)
  lanczos.py   Rademacher probes, Lanczos recurrence, Gauss quadrature, SLQ energy
               (Eqs. hutch, dds, recurs, tridiag1, tridiag2, sl4, plasmonic2; Algorithms 1 and 2)
  dense.py     exact energy from a full eigendecomposition (Eq. plasmonic) and its gradient
  forces.py    gradient of the bilinear form p^T T'(R) q, the stochastic force estimator
  replica.py   brute-force spherical replica sum (Eq. replica), used only to pin ewald.py
  scs.py       self-consistent screening of the polarisabilities (the rsSCS front end the
               review of the MBD model names and leaves out of the paper's scope), dense

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` against closed forms, invariants, brute force or an
independent library routine.
"""
