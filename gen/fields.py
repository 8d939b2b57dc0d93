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

import concurrent.futures
import os

import numpy as np

_CHUNK = 1 << 16


def _chunked(fn, n: int, *arrays):
    """Apply ``fn`` to matching row-chunks of ``arrays`` on all host cores.

    Each matrix is transformed independently, so the result does not depend on
    the chunking; all random numbers are drawn before this is called.
    """
    if n <= _CHUNK:
        return fn(*arrays)
    out = None
    starts = list(range(0, n, _CHUNK))
    with concurrent.futures.ThreadPoolExecutor(os.cpu_count() or 1) as ex:
        parts = list(ex.map(lambda s: fn(*[a[s:s + _CHUNK] for a in arrays]), starts))
    out = np.concatenate(parts, axis=0)
    return out


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


def _unit_det(u: np.ndarray) -> np.ndarray:
    """Divide each matrix by the principal cube root of its determinant."""
    det = (u[:, 0, 0] * (u[:, 1, 1] * u[:, 2, 2] - u[:, 1, 2] * u[:, 2, 1])
           - u[:, 0, 1] * (u[:, 1, 0] * u[:, 2, 2] - u[:, 1, 2] * u[:, 2, 0])
           + u[:, 0, 2] * (u[:, 1, 0] * u[:, 2, 1] - u[:, 1, 1] * u[:, 2, 0]))
    return u / np.exp(1j * np.angle(det) / 3.0)[:, None, None]


def haar_su3(g: np.random.Generator, n: int) -> np.ndarray:
    """``n`` Haar-distributed SU(3) matrices, shape ``(n, 3, 3)``.

    Recipe: the Q factor of a complex Gaussian matrix with R's diagonal made
    positive (Mezzadri, "How to generate random matrices from the classical
    compact groups", 2007) is Haar on U(3); that Q is unique, and Gram-Schmidt
    on the columns produces exactly it (vectorised here over all matrices).
    Dividing by the principal cube root of the determinant commutes with left
    multiplication by SU(3), so the result is Haar on SU(3).
    """
    a = complex_gaussian(g, (n, 3, 3))

    def gram_schmidt(a):
        q = []
        for k in range(3):
            v = a[:, :, k]
            for j in range(k):
                v = v - np.sum(np.conj(q[j]) * v, axis=1)[:, None] * q[j]
            v = v / np.sqrt(np.sum(np.abs(v) ** 2, axis=1))[:, None]
            q.append(v)
        return _unit_det(np.stack(q, axis=2))

    return _chunked(gram_schmidt, n, a)


def smooth_su3(g: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """``n`` matrices ``exp(i*eps*H)`` with ``H`` a random traceless Hermitian 3x3.

    ``H`` is the traceless part of the Hermitian part of a complex Gaussian
    matrix. The exponential is taken in FP64 by scaling and squaring with a
    degree-16 Taylor polynomial (the scaled argument has norm <= 1/8, so the
    truncation error is far below rounding), then given det 1 (a no-op up to
    rounding since tr H = 0).
    """
    a = complex_gaussian(g, (n, 3, 3))
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h = h - tr[:, None, None] * np.eye(3)[None]
    norm = eps * np.max(np.sum(np.abs(h), axis=2), axis=1).max() if n else 0.0
    sq = max(0, int(np.ceil(np.log2(max(norm, 1e-300) * 8.0))))

    def mm(a, b):  # batched 3x3 product with ufuncs (which release the GIL)
        return (a[:, :, :, None] * b[:, None, :, :]).sum(axis=2)

    def expm(h):
        x = (1j * eps / 2.0 ** sq) * h
        eye = np.broadcast_to(np.eye(3, dtype=np.complex128), x.shape)
        u = eye.copy()
        term = eye.copy()
        for k in range(1, 17):
            term = mm(term, x) / k
            u = u + term
        for _ in range(sq):
            u = mm(u, u)
        return _unit_det(u)

    return _chunked(expm, n, h)


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
