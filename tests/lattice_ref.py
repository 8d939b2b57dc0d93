"""Test-side lattice helpers, written independently of ``oracle/``.

* the chiral gamma basis built from the Pauli matrices;
* the dense Wilson matrix written element by element from the footnote of
  Eq. 1 of arXiv:2303.08609 (brute force, small lattices only);
* site geometry, gauge transformations and plane waves for the invariance and
  closed-form pins.

Nothing here is imported by the product path.
"""

from __future__ import annotations

import itertools

import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def gammas():
    """Euclidean chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]], gamma_t = [[0,1],[1,0]]."""
    z = np.zeros((2, 2), dtype=np.complex128)
    g = []
    for s in SIGMA:
        g.append(np.block([[z, -1j * s], [1j * s, z]]))
    one = np.eye(2, dtype=np.complex128)
    g.append(np.block([[z, one], [one, z]]))
    return g


GAMMA = gammas()
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]


def lex(dims, c):
    lx, ly, lz, _ = dims
    return ((c[3] * lz + c[2]) * ly + c[1]) * lx + c[0]


def coords(dims, i):
    c = []
    for d in dims:
        c.append(i % d)
        i //= d
    return c


def all_coords(dims):
    """(V, 4) integer coordinates in lexicographic order."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel(), t.ravel()], axis=1)


def parity_sites(dims, parity):
    """Lexicographic indices of the sites of one parity, in increasing order."""
    c = all_coords(dims)
    return np.nonzero(c.sum(axis=1) % 2 == parity)[0]


def shift_index(dims, mu, step):
    """Array n with n[x] = lex(x + step * mu-hat), periodic."""
    c = all_coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % dims[mu]
    lx, ly, lz, _ = dims
    return ((c[:, 3] * lz + c[:, 2]) * ly + c[:, 1]) * lx + c[:, 0]


def dense_wilson(U, kappa, dims):
    """Dense D_W from the footnote of Eq. 1, indices (site, spin, colour).

    (D_W)_{ia,jb}(x,y) = d_ij d_ab d_xy - kappa sum_mu [ (1-g_mu)_ij U_mu(x)_ab d_{x+mu,y}
                                                    + (1+g_mu)_ij conj(U_mu(x-mu)_ba) d_{x-mu,y} ]
    """
    V = int(np.prod(dims))
    n = 12 * V
    D = np.eye(n, dtype=np.complex128)
    one = np.eye(4, dtype=np.complex128)
    for x in range(V):
        c = coords(dims, x)
        for mu in range(4):
            cf = list(c)
            cf[mu] = (cf[mu] + 1) % dims[mu]
            cb = list(c)
            cb[mu] = (cb[mu] - 1) % dims[mu]
            yf, yb = lex(dims, cf), lex(dims, cb)
            for i, j in itertools.product(range(4), range(4)):
                pm = (one - GAMMA[mu])[i, j]
                pp = (one + GAMMA[mu])[i, j]
                for a, b in itertools.product(range(3), range(3)):
                    if pm != 0:
                        D[12 * x + 3 * i + a, 12 * yf + 3 * j + b] -= kappa * pm * U[mu, x, a, b]
                    if pp != 0:
                        D[12 * x + 3 * i + a, 12 * yb + 3 * j + b] -= (
                            kappa * pp * np.conj(U[mu, yb, b, a]))
    return D


def dense_blocks(D, dims):
    """(D_ee, D_eo, D_oe, D_oo) with each parity's sites in increasing lexicographic order."""
    e = parity_sites(dims, 0)
    o = parity_sites(dims, 1)
    ie = (12 * e[:, None] + np.arange(12)[None]).ravel()
    io = (12 * o[:, None] + np.arange(12)[None]).ravel()
    return (D[np.ix_(ie, ie)], D[np.ix_(ie, io)], D[np.ix_(io, ie)], D[np.ix_(io, io)])


def gauge_transform(U, g, dims):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dag."""
    out = np.empty_like(U)
    gd = np.conj(np.swapaxes(g, 1, 2))
    for mu in range(4):
        fwd = shift_index(dims, mu, +1)
        out[mu] = g @ U[mu] @ gd[fwd]
    return out


def rotate_parity_spinor(psi, g, dims, parity):
    """psi(x) -> g(x) psi(x) on the sites of one parity; psi shape (V/2, 4, 3)."""
    sites = parity_sites(dims, parity)
    return np.einsum("nab,nsb->nsa", g[sites], psi)


def plane_wave(dims, nvec, u, parity):
    """psi(x) = exp(i p.x) u on one parity, p_mu = 2 pi n_mu / L_mu."""
    sites = parity_sites(dims, parity)
    c = all_coords(dims)[sites]
    p = 2 * np.pi * np.asarray(nvec) / np.asarray(dims)
    ph = np.exp(1j * (c @ p))
    return ph[:, None, None] * u[None]


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b.ravel())
    return float(np.linalg.norm((a - b).ravel()) / (nb if nb > 0 else 1.0))


def vdot(a, b):
    return complex(np.vdot(np.asarray(a).ravel(), np.asarray(b).ravel()))
