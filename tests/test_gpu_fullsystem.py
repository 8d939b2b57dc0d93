"""The full Wilson system D_W xi = eta through Eqs. 3-5 on the GPU.

* prepare_source / reconstruct against the oracle's hopping terms;
* solve_full against the dense LAPACK solve of the D_W built from the footnote
  of Eq. 1 at 4^4, and against the full-lattice residual |D_W xi - eta| / |eta|
  evaluated with the oracle at 8^4.
"""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar
from lattice_ref import dense_wilson, parity_sites

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_prepare_and_reconstruct(weo, oracle_lib, prec):
    import torch

    dims = (4, 6, 4, 8)
    kappa = 0.13
    U = gen.gauge_field(dims, "haar", seed=90)
    ee, eo = gen.gaussian_spinor(dims, nrhs=2, seed=91)
    op = weo.WilsonEO(dims, kappa, to_device(U), prec=prec)
    a, b = to_device(to_planar(ee), prec), to_device(to_planar(eo), prec)
    out = torch.empty_like(a)
    weo.wilson_eo_prepare_source(op.handle, out, a, b)
    want = ee + kappa * oracle_lib.hop(U, eo, dims, 0)
    assert rel_l2(from_planar(out.cpu().numpy()), want) <= TOL[prec]
    weo.wilson_eo_reconstruct(op.handle, out, b, a)
    want = eo + kappa * oracle_lib.hop(U, ee, dims, 1)
    assert rel_l2(from_planar(out.cpu().numpy()), want) <= TOL[prec]
    op.close()


@pytest.mark.parametrize("prec,mixed", [("f64", False), ("f32", True), ("f16", True)])
def test_solve_full_against_dense(weo, prec, mixed):
    import torch

    dims = (4, 4, 4, 4)
    kappa = 0.125
    U = gen.gauge_field(dims, "smooth", seed=92, eps=0.4)
    eta = gen.complex_gaussian(gen.rng(93), (256, 4, 3))
    e, o = parity_sites(dims, 0), parity_sites(dims, 1)
    xi_dense = np.linalg.solve(dense_wilson(U, kappa, dims), eta.ravel()).reshape(eta.shape)
    op = weo.WilsonEO(dims, kappa, to_device(U), prec=prec)
    ee, eo = to_device(to_planar(eta[e])), to_device(to_planar(eta[o]))
    xe, xo = torch.zeros_like(ee), torch.zeros_like(eo)
    st, it, rr = weo.wilson_eo_solve_full(op.handle, xe, xo, ee, eo, tol=1e-12, mixed=mixed)
    assert st == 0 and rr <= 1e-12
    xi = np.empty_like(eta)
    xi[e], xi[o] = from_planar(xe.cpu().numpy()), from_planar(xo.cpu().numpy())
    assert rel_l2(xi, xi_dense) <= 1e-9
    op.close()


def test_solve_full_residual_8x8x8x8(weo, oracle_lib):
    import torch

    dims = (8, 8, 8, 8)
    kappa = 0.13
    U = gen.gauge_field(dims, "smooth", seed=94, eps=0.4)
    eta_e, eta_o = gen.gaussian_spinor(dims, nrhs=2, seed=95)
    op = weo.WilsonEO(dims, kappa, to_device(U), prec="f16")
    ee, eo = to_device(to_planar(eta_e)), to_device(to_planar(eta_o))
    xe, xo = torch.zeros_like(ee), torch.zeros_like(eo)
    st, it, rr = weo.wilson_eo_solve_full(op.handle, xe, xo, ee, eo, tol=1e-10, mixed=True)
    assert st == 0
    xi_e, xi_o = from_planar(xe.cpu().numpy()), from_planar(xo.cpu().numpy())
    # D_W xi = xi - kappa H xi, parity by parity
    re = xi_e - kappa * oracle_lib.hop(U, xi_o, dims, 0) - eta_e
    ro = xi_o - kappa * oracle_lib.hop(U, xi_e, dims, 1) - eta_o
    res = np.sqrt(np.linalg.norm(re) ** 2 + np.linalg.norm(ro) ** 2)
    nrm = np.sqrt(np.linalg.norm(eta_e) ** 2 + np.linalg.norm(eta_o) ** 2)
    assert res / nrm <= 1e-8
    assert np.linalg.norm(ro) / nrm <= 1e-13  # odd equations hold by construction
    op.close()
