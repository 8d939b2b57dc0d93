"""Seeded random fields in the canonical external layouts.

Canonical layouts (complex numbers interleaved re, im):

* gauge field  ``U[mu][site][a][b]``, shape ``(4, V, 3, 3)``, ``mu = 0..3`` for
  the x, y, z, t axes and ``site = ((t*Lz + z)*Ly + y)*Lx + x``;
* single-parity spinor ``psi[rhs][i][spin][colour]``, shape ``(nrhs, V/2, 4, 3)``,
  where ``i`` enumerates the sites of one parity in increasing lexicographic
  order (the caller decides what the index means; nothing here depends on it).

All generators take a ``numpy.random.Generator`` (PCG64) so that every input
of a test or benchmark is reproducible from one integer seed.
"""

from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator for ``seed``."""
    return np.random.Generator(np.random.PCG64(seed))


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def complex_gaussian(g: np.random.Generator, shape) -> np.ndarray:
    """Complex normal entries with re, im ~ N(0, 1/2), so E|z|^2 = 1."""
    s = np.sqrt(0.5)
    return (g.normal(0.0, s, shape) + 1j * g.normal(0.0, s, shape)).astype(np.complex128)


def haar_su3(g: np.random.Generator, n: int) -> np.ndarray:
    """``n`` Haar-distributed SU(3) matrices, shape ``(n, 3, 3)``.

    Recipe: QR of a complex Gaussian matrix, with the phases of R's diagonal
    moved into Q (Mezzadri, "How to generate random matrices from the classical
    compact groups", 2007), which gives Haar U(3); then division by the
    principal cube root of the determinant. That map commutes with left
    multiplication by SU(3), so the result is Haar on SU(3).
    """
    a = complex_gaussian(g, (n, 3, 3))
    q, r = np.linalg.qr(a)
    d = np.diagonal(r, axis1=1, axis2=2)
    ph = d / np.abs(d)
    q = q * ph[:, None, :]
    det = np.linalg.det(q)
    root = np.exp(1j * np.angle(det) / 3.0)
    return q / root[:, None, None]


def smooth_su3(g: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """``n`` matrices ``exp(i*eps*H)`` with ``H`` a random traceless Hermitian 3x3.

    ``H`` is the traceless part of the Hermitian part of a complex Gaussian
    matrix. The exponential is taken through the eigendecomposition of ``H``
    in FP64 and the result is re-unitarised (polar factor) and given det 1.
    """
    a = complex_gaussian(g, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    w, v = np.linalg.eigh(h)
    u = (v * np.exp(1j * eps * w)[:, None, :]) @ np.conj(np.swapaxes(v, 1, 2))
    # polar re-unitarisation and det fix (both are no-ops up to rounding)
    uu, _, vh = np.linalg.svd(u)
    u = uu @ vh
    det = np.linalg.det(u)
    return u / np.exp(1j * np.angle(det) / 3.0)[:, None, None]


def gauge_field(dims, kind: str = "haar", seed: int = 0, eps: float = 0.4) -> np.ndarray:
    """Gauge field of shape ``(4, V, 3, 3)`` complex128.

    ``kind``: ``"haar"`` (independent Haar links), ``"smooth"`` (``exp(i eps H)``)
    or ``"unit"`` (all links the identity, the free field).
    """
    v = volume(dims)
    if kind == "unit":
        return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()
    g = rng(seed)
    if kind == "haar":
        u = haar_su3(g, 4 * v)
    elif kind == "smooth":
        u = smooth_su3(g, 4 * v, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return np.ascontiguousarray(u.reshape(4, v, 3, 3))


def gaussian_spinor(dims, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """Single-parity Gaussian spinor(s), shape ``(nrhs, V/2, 4, 3)``."""
    vh = volume(dims) // 2
    return complex_gaussian(rng(seed), (nrhs, vh, 4, 3))


def point_sources(dims, site_index: int) -> np.ndarray:
    """The 12 spin-colour unit sources at one single-parity site index.

    Shape ``(12, V/2, 4, 3)``; source ``k = 3*spin + colour`` is 1 at
    ``[k, site_index, spin, colour]`` and 0 elsewhere.
    """
    vh = volume(dims) // 2
    out = np.zeros((12, vh, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            out[3 * s + c, site_index, s, c] = 1.0
    return out


def random_gauge_transform(dims, seed: int = 0) -> np.ndarray:
    """One Haar SU(3) matrix per lattice site, shape ``(V, 3, 3)``."""
    return haar_su3(rng(seed), volume(dims))
