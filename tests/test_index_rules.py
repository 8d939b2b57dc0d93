"""Host-side checks of the index and coefficient rules the kernels use (the
GPU parity tests check that the kernels follow them):

* the x-compacted neighbour indices of a parity site (Sec. 3.3-3.4), written as
  the hopping kernels compute them, against lex/2 of x +- mu computed from the
  coordinates, for extents down to 2;
* the fused kernel's wavefront task order: each first-hop task A(t) and
  second-hop task B(t) appears once, and every B(t) comes after A(t-1), A(t),
  A(t+1), for every t extent and lookahead (this is what makes its bounded
  waits deadlock-free);
* the float-float kernel's run-time projector table: unit factors c0, c1 and
  spin indices j0, j1 with h = psi_up + c psi_j, and d2, d3, k2, k3 with
  out_dn += d chi_k, against (1 - S gamma_mu) in the chiral basis of Eq. 1.
"""

import itertools

import numpy as np
import pytest


def kernel_neighbours(dims, out_parity, i):
    """The compact neighbour indices as the hopping kernels compute them."""
    lx, ly, lz, lt = dims
    lxh = lx // 2
    xh, rem = i % lxh, i // lxh
    y, rem = rem % ly, rem // ly
    z, t = rem % lz, rem // lz
    par = (y + z + t + out_parity) & 1
    sy, sz, st = lxh, lxh * ly, lxh * ly * lz
    row = i - xh
    xp = (0 if xh + 1 == lxh else xh + 1) if par else xh
    xm = xh if par else (lxh - 1 if xh == 0 else xh - 1)
    return {
        (0, 1): row + xp, (0, -1): row + xm,
        (1, 1): i + (-(ly - 1) * sy if y + 1 == ly else sy), (1, -1): i + ((ly - 1) * sy if y == 0 else -sy),
        (2, 1): i + (-(lz - 1) * sz if z + 1 == lz else sz), (2, -1): i + ((lz - 1) * sz if z == 0 else -sz),
        (3, 1): i + (-(lt - 1) * st if t + 1 == lt else st), (3, -1): i + ((lt - 1) * st if t == 0 else -st),
    }, (2 * xh + par, y, z, t)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 2), (4, 2, 2, 8), (6, 4, 4, 2), (8, 6, 2, 4)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_compact_neighbour_indices(dims, out_parity):
    lx, ly, lz, lt = dims
    vh = lx * ly * lz * lt // 2
    for i in range(vh):
        nb, (x, y, z, t) = kernel_neighbours(dims, out_parity, i)
        assert (x + y + z + t) % 2 == out_parity
        assert ((t * lz + z) * ly + y) * lx + x == 2 * i + (x % 2)  # lex/2 == i
        c = [x, y, z, t]
        for (mu, sgn), n in nb.items():
            d = list(c)
            d[mu] = (d[mu] + sgn) % dims[mu]
            lex = ((d[3] * lz + d[2]) * ly + d[1]) * lx + d[0]
            assert n == lex // 2, (dims, out_parity, i, mu, sgn)


def fused_task(L, D, k):
    """Slice task k of the fused kernel's queue: ('A'|'B', t)."""
    if k == 0:
        return ("A", L - 1)
    if k <= D:
        return ("A", k - 1)
    kp, pairs = k - (D + 1), L - 1 - D
    if kp < 2 * pairs:
        return ("B", kp >> 1) if kp & 1 else ("A", (kp >> 1) + D)
    return ("B", pairs + (kp - 2 * pairs))


def test_fused_queue_order():
    for L in range(2, 131, 2):
        for D0 in range(1, 70):
            D = max(1, min(D0, L - 1))  # as the host clamps it
            seq = [fused_task(L, D, k) for k in range(2 * L)]
            assert sorted(seq) == sorted([("A", t) for t in range(L)] + [("B", t) for t in range(L)])
            pos = {x: n for n, x in enumerate(seq)}
            for t in range(L):
                for u in ((t - 1) % L, t, (t + 1) % L):
                    assert pos[("A", u)] < pos[("B", t)], (L, D, t, u)


def dir_coef(mu, S):
    """The float-float kernel's table: (c0, j0, c1, j1, d2, k2, d3, k3), unit
    factors as complex numbers."""
    sp = S > 0

    def unit(rot, neg):
        return (1j if rot else 1) * (-1 if neg else 1)

    rows = {
        0: (True, not sp, True, not sp, 3, 2, True, sp, True, sp, 1, 0),
        1: (False, not sp, False, sp, 3, 2, False, sp, False, not sp, 1, 0),
        2: (True, not sp, True, sp, 2, 3, True, sp, True, not sp, 0, 1),
        3: (False, sp, False, sp, 2, 3, False, sp, False, sp, 0, 1),
    }
    r0, n0, r1, n1, j0, j1, r2, n2, r3, n3, k2, k3 = rows[mu]
    return unit(r0, n0), j0, unit(r1, n1), j1, unit(r2, n2), k2, unit(r3, n3), k3


@pytest.mark.parametrize("mu,S", list(itertools.product(range(4), (1, -1))))
def test_float_float_projector_table(oracle_lib, mu, S):
    """(1 - S gamma_mu) psi has upper components h = psi_up + c psi_j and lower
    components -S A^dag h; the kernel adds d_2 chi_{k2}, d_3 chi_{k3} to the
    lower components of out for chi = U h, which must equal that lower part."""
    g = oracle_lib.gamma(mu)
    P = np.eye(4) - S * g
    rng = np.random.default_rng(10 * mu + (S > 0))
    psi = rng.normal(size=4) + 1j * rng.normal(size=4)
    full = P @ psi
    c0, j0, c1, j1, d2, k2, d3, k3 = dir_coef(mu, S)
    h = np.array([psi[0] + c0 * psi[j0], psi[1] + c1 * psi[j1]])
    assert np.allclose(full[:2], h)
    # the lower half of (1 - S gamma) psi, rebuilt from h as the kernel does
    assert np.allclose(full[2], d2 * h[k2]) and np.allclose(full[3], d3 * h[k3])
