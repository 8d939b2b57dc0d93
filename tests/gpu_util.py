"""Helpers for the GPU parity tests: layout conversion and tolerances.

The oracle works in ``(nrhs, V/2, 4, 3)``; the library's canonical spinor layout
is planar ``(nrhs, 4, 3, V/2)``. Converting between them is a transpose only.
"""

import numpy as np

# relative L2 tolerances against the FP64 oracle, per storage precision
TOL = {"f64": 1e-12, "f32": 1e-5, "f16": 5e-3, "bf16": 5e-3}


def to_planar(psi):
    """(..., V/2, 4, 3) -> (..., 4, 3, V/2), contiguous."""
    return np.ascontiguousarray(np.moveaxis(np.asarray(psi), -3, -1))


def from_planar(psi):
    """(..., 4, 3, V/2) -> (..., V/2, 4, 3), contiguous."""
    return np.ascontiguousarray(np.moveaxis(np.asarray(psi), -1, -3))


def np_dtype(prec):
    return np.complex128 if prec == "f64" else np.complex64


def to_device(a, prec=None):
    import torch

    a = np.asarray(a)
    if prec is not None:
        a = a.astype(np_dtype(prec))
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
