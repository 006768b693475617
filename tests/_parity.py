"""Comparison helpers of the GPU parity tests.

close(a, b, tol, width) is the operator-parity criterion: the relative L2 error
of the whole array below tol, and, so that a large error on one atom (or mesh
point) cannot hide in that norm, the largest error of one atom (rows of
`width` values: 3 for [.., N, 3] fields, 1 for mesh values) below
ATOM_FACTOR * tol of the RMS row norm of b.
"""
import numpy as np

ATOM_FACTOR = 10.0


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def atom_max(a, b, width=3):
    """Largest row error |a_i - b_i| over the RMS row norm of b."""
    a, b = np.asarray(a).reshape(-1, width), np.asarray(b).reshape(-1, width)
    return np.linalg.norm(a - b, axis=1).max() / np.sqrt(np.mean(np.sum(b * b, axis=1)))


def close(a, b, tol, width=3, atom_factor=ATOM_FACTOR):
    r, m = rel(a, b), atom_max(a, b, width)
    assert r < tol, f"relative L2 error {r:.3e} >= {tol:.1e}"
    assert m < atom_factor * tol, f"largest per-row error {m:.3e} >= {atom_factor * tol:.1e} of the RMS row norm"
    return r, m
