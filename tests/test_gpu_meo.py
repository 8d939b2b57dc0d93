"""Parity of the CUDA M_eo, M_eo^dag and hopping kernels with the FP64 oracle.

Every case calls through the C ABI (``libwilson_eo.so`` via its ctypes binding)
on seeded inputs and compares element by element with ``oracle/`` within the
relative L2 tolerance of the storage precision: 1e-12 (FP64), 1e-5 (FP32),
5e-3 (FP16/BF16 storage with FP32 arithmetic).
"""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, np_dtype, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu

PRECS = [("f64", 18), ("f64", 12), ("f32", 18), ("f32", 12), ("f16", 18), ("f16", 12),
         ("bf16", 18), ("bf16", 12)]


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def _run(weo, dims, kappa, U, psi, prec, fmt, dag=False, host=False):
    import torch

    gauge = to_device(U, "f64")
    op = weo.WilsonEO(dims, kappa, gauge, prec=prec, linkfmt=fmt)
    x = to_planar(psi).astype(np_dtype(prec))
    if host:
        out = np.empty_like(x)
        nrhs = 1 if x.ndim == 3 else x.shape[0]
        (weo.wilson_eo_apply_dag if dag else weo.wilson_eo_apply)(op.handle, out, x, nrhs)
        res = out
    else:
        res = op.apply(torch.from_numpy(x).cuda(), dag=dag).cpu().numpy()
    torch.cuda.synchronize()
    op.close()
    return from_planar(res)


@pytest.mark.parametrize("prec,fmt", PRECS)
@pytest.mark.parametrize("dag", [False, True])
def test_meo_8x8x8x8_haar(weo, oracle_lib, prec, fmt, dag):
    """8^4, kappa = 0.125, Haar links, Gaussian even source, seed 0."""
    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, "haar", seed=0)
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    want = (oracle_lib.meo_dag if dag else oracle_lib.meo)(U, 0.125, psi, dims)
    got = _run(weo, dims, 0.125, U, psi, prec, fmt, dag)
    assert rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 8), (6, 2, 4, 2), (4, 6, 2, 10),
                                  (10, 4, 4, 6)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_meo_ragged_and_degenerate_dims(weo, oracle_lib, dims, prec):
    """Extents of 2 (x+mu = x-mu), Lx = 2, non-cubic shapes, V/2 not a multiple of the block."""
    U = gen.gauge_field(dims, "smooth", seed=5, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=6)[0]
    for dag in (False, True):
        want = (oracle_lib.meo_dag if dag else oracle_lib.meo)(U, 0.13, psi, dims)
        got = _run(weo, dims, 0.13, U, psi, prec, 18, dag)
        assert rel_l2(got, want) <= TOL[prec]


@pytest.mark.parametrize("prec,fmt", [("f64", 18), ("f32", 18), ("f32", 12), ("f16", 12),
                                      ("bf16", 18)])
def test_meo_full_size_sampled(weo, oracle_lib, prec, fmt, fields_32x64):
    """32^3 x 64, kappa = 0.13, exp(i 0.4 H) links: 400 sampled output sites
    against the oracle's per-site evaluation, plus global properties."""
    import torch

    dims = (32, 32, 32, 64)
    vh = 32 * 32 * 32 * 64 // 2
    dims, U, _ = fields_32x64  # smooth links, seed 0
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U, "f64"), prec=prec, linkfmt=fmt)
    x = torch.from_numpy(to_planar(psi).astype(np_dtype(prec))).cuda()
    sites = np.sort(gen.rng(1).choice(vh, 400, replace=False))
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        got = from_planar(y[:, :, torch.from_numpy(sites).cuda()].cpu().numpy())
        want = oracle_lib.meo_sites(U, 0.13, psi, dims, sites, dag=dag)
        assert rel_l2(got, want) <= TOL[prec]
        assert torch.isfinite(torch.view_as_real(y)).all()
    op.close()


def test_meo_multi_rhs(weo, oracle_lib):
    """Several right-hand sides in one call: each matches its own oracle result."""
    dims = (8, 8, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=7)
    psi = gen.gaussian_spinor(dims, nrhs=5, seed=8)
    for prec in ("f64", "f32", "f16"):
        got = _run(weo, dims, 0.12, U, psi, prec, 18)
        for r in range(5):
            assert rel_l2(got[r], oracle_lib.meo(U, 0.12, psi[r], dims)) <= TOL[prec]


def test_meo_host_arrays(weo, oracle_lib):
    """Host (numpy) input and output go through the library's staging path."""
    dims = (4, 4, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=9)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=10)
    for dag in (False, True):
        got = _run(weo, dims, 0.13, U, psi, "f32", 18, dag=dag, host=True)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        assert rel_l2(got, f(U, 0.13, psi, dims)) <= TOL["f32"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_hop_both_parities(weo, oracle_lib, prec):
    """H_oe (even -> odd) and H_eo (odd -> even), and their adjoints (sign-swapped projectors)."""
    import torch

    dims = (4, 6, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=11)
    psi = gen.gaussian_spinor(dims, seed=12)[0]
    op = weo.WilsonEO(dims, 0.1, to_device(U, "f64"), prec=prec, linkfmt=18)
    x = torch.from_numpy(to_planar(psi).astype(np_dtype(prec))).cuda()
    for parity in (0, 1):
        for dag in (False, True):
            got = from_planar(op.hop(x, parity, dag=dag).cpu().numpy())
            f = oracle_lib.hop_adj if dag else oracle_lib.hop
            assert rel_l2(got, f(U, psi, dims, parity)) <= TOL[prec]
    op.close()


def test_kappa_zero_is_identity_and_set_kappa(weo):
    import torch

    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=13)
    psi = to_planar(gen.gaussian_spinor(dims, seed=14))
    op = weo.WilsonEO(dims, 0.0, to_device(U), prec="f64")
    x = torch.from_numpy(psi).cuda()
    assert torch.equal(op.apply(x), x)
    op.set_kappa(0.13)
    assert not torch.equal(op.apply(x), x)
    op.close()
