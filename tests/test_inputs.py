"""The seeded synthetic inputs every test and the benchmark use (`gen/`): the
links are SU(3), the smooth field is close to the identity by the amount its
epsilon sets, the Gaussian spinors have E|z|^2 = 1 per component, point sources
are unit vectors at one site, the chunked multi-core generation gives the same
numbers as one chunk, and one seed always gives the same field."""

import numpy as np
import pytest

import gen
from gen import fields


def _su3_residuals(u):
    u = u.reshape(-1, 3, 3)
    eye = np.eye(3)
    unit = np.abs(np.einsum("nab,ncb->nac", u, u.conj()) - eye).max()
    det = np.abs(np.linalg.det(u) - 1.0).max()
    return unit, det


@pytest.mark.parametrize("kind", ["haar", "smooth"])
def test_links_are_su3(kind):
    u = gen.gauge_field((4, 2, 2, 4), kind, seed=5)
    assert u.shape == (4, 64, 3, 3) and u.dtype == np.complex128
    unit, det = _su3_residuals(u)
    assert unit < 1e-13 and det < 1e-13


def test_haar_links_are_spread_and_smooth_links_near_one():
    # Haar measure on SU(3): E tr U = 0 and E |tr U|^2 = 1
    tr = np.trace(gen.gauge_field((8, 8, 8, 8), "haar", seed=6), axis1=-2, axis2=-1)
    assert abs(tr.mean()) < 0.02 and abs(np.mean(np.abs(tr) ** 2) - 1.0) < 0.03
    # exp(i eps H): the distance to the identity grows with eps
    d = [np.abs(gen.gauge_field((4, 4, 4, 4), "smooth", seed=7, eps=e) - np.eye(3)).mean()
         for e in (0.05, 0.2, 0.4)]
    assert d[0] < d[1] < d[2] and d[0] < 0.05
    assert np.array_equal(gen.gauge_field((2, 2, 2, 2), "unit"),
                          np.broadcast_to(np.eye(3), (4, 16, 3, 3)))


def test_gaussian_spinor_moments():
    psi = gen.gaussian_spinor((8, 8, 8, 8), nrhs=2, seed=8)
    assert psi.shape == (2, 2048, 4, 3)
    assert abs(np.mean(np.abs(psi) ** 2) - 1.0) < 0.01
    assert abs(psi.real.var() - 0.5) < 0.01 and abs(psi.imag.var() - 0.5) < 0.01
    assert abs(psi.mean()) < 0.01


def test_point_sources_are_unit_vectors_at_one_site():
    src = gen.point_sources((4, 4, 2, 2), 5)
    assert src.shape == (12, 32, 4, 3)
    for k in range(12):
        nz = np.argwhere(src[k] != 0)
        assert nz.tolist() == [[5, k // 3, k % 3]] and src[k][5, k // 3, k % 3] == 1


def test_seeds_reproduce_and_differ():
    a = gen.gauge_field((4, 4, 2, 2), "haar", seed=9)
    assert np.array_equal(a, gen.gauge_field((4, 4, 2, 2), "haar", seed=9))
    assert not np.array_equal(a, gen.gauge_field((4, 4, 2, 2), "haar", seed=10))


def test_chunked_generation_equals_one_chunk(monkeypatch):
    """Generation split over host cores (chunks of rows) draws all random
    numbers first, so it gives bit-identical fields."""
    dims = (8, 8, 8, 4)  # 4 V = 8192 links
    ref = gen.gauge_field(dims, "smooth", seed=11)
    monkeypatch.setattr(fields, "_CHUNK", 1000)
    assert np.array_equal(ref, gen.gauge_field(dims, "smooth", seed=11))
    ref = gen.gauge_field(dims, "haar", seed=12)
    monkeypatch.setattr(fields, "_CHUNK", 1 << 16)
    assert np.array_equal(ref, gen.gauge_field(dims, "haar", seed=12))
