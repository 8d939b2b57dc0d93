"""The fused single-launch M_eo (both hops in one persistent launch, the first
hop running `lookahead` t-slices ahead of the second) against the oracle and,
bit for bit, against the two-launch path (same per-site code), for every link
format, lookaheads from 1 to beyond Lt (clamped to Lt - 1), both CTA sizes, and
t extents from 2 up."""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.mark.parametrize("dims", [(4, 4, 4, 2), (4, 4, 4, 4), (8, 4, 6, 6), (8, 8, 8, 8),
                                  (4, 6, 2, 22), (6, 4, 4, 40)])
@pytest.mark.parametrize("lookahead,threads", [(1, 128), (2, 256), (8, 128), (64, 256)])
def test_fused_matches_oracle(weo, oracle_lib, dims, lookahead, threads):
    import torch

    U = gen.gauge_field(dims, "haar", seed=100)
    psi = gen.gaussian_spinor(dims, seed=101)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(psi), "f32")
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    weo.wilson_eo_set_algorithm(op.handle, "fused", lookahead, threads)
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        assert rel_l2(from_planar(y.cpu().numpy()), f(U, 0.13, psi, dims)) <= TOL["f32"]
        assert torch.equal(y, ref[dag])
    op.close()


@pytest.mark.parametrize("prec,fmt", [("f32", 12), ("f16", 18), ("f16", 12), ("bf16", 18),
                                      ("bf16", 12)])
def test_fused_link_formats(weo, oracle_lib, prec, fmt):
    import torch

    dims = (8, 8, 8, 16)
    U = gen.gauge_field(dims, "smooth", seed=102, eps=0.4)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=103)
    op = weo.WilsonEO(dims, 0.125, to_device(U), prec=prec, linkfmt=fmt)
    x = to_device(to_planar(psi), "f32")
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    weo.wilson_eo_set_algorithm(op.handle, "fused", 4, 128)
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(2):
            assert rel_l2(from_planar(y[r].cpu().numpy()), f(U, 0.125, psi[r], dims)) <= TOL[prec]
        assert torch.equal(y, ref[dag])
    op.close()


def test_fused_full_size_sampled_and_solver(weo, oracle_lib, fields_32x64):
    """32^3 x 64 sampled sites, then a mixed solve whose inner operator is fused."""
    import torch

    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    dims, U, _ = fields_32x64  # smooth links, seed 0
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_algorithm(op.handle, "fused", 8, 128)
    x = to_device(to_planar(psi), "f32")
    sites = np.sort(gen.rng(2).choice(vh, 300, replace=False))
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        got = from_planar(y[:, :, torch.from_numpy(sites).cuda()].cpu().numpy())
        assert rel_l2(got, oracle_lib.meo_sites(U, 0.13, psi, dims, sites, dag=dag)) <= TOL["f32"]
    op.close()
    small = (8, 8, 8, 8)
    Us = gen.gauge_field(small, "smooth", seed=104, eps=0.4)
    b = gen.gaussian_spinor(small, seed=105)[0]
    op = weo.WilsonEO(small, 0.13, to_device(Us), prec="f16")
    weo.wilson_eo_set_algorithm(op.handle, "fused", 1, 128)
    xs, info = op.solve(to_device(to_planar(b)), tol=1e-10, mixed=True)
    weo.wilson_eo_check(op.handle)
    assert info["converged"]
    xg = from_planar(xs.cpu().numpy())
    ax = oracle_lib.meo_dag(Us, 0.13, oracle_lib.meo(Us, 0.13, xg, small), small)
    assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= 1.5e-10
    op.close()


def test_fused_rejected_for_fp64(weo):
    dims = (4, 4, 4, 4)
    op = weo.WilsonEO(dims, 0.1, to_device(gen.gauge_field(dims, "haar", seed=1)), prec="f64")
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_set_algorithm(op.handle, "fused")
    assert e.value.status == -3
    op.close()


def test_fused_bounded_wait_reports_timeout_and_recovers(weo, oracle_lib):
    """Failure detection without a fault: first-hop completions are never
    published, the second hop's bounded waits run out, wilson_eo_check reports
    WEO_ERR_TIMEOUT once, and the next fused apply on the same context is correct."""
    import torch

    dims = (8, 8, 8, 16)
    U = gen.gauge_field(dims, "haar", seed=106)
    psi = gen.gaussian_spinor(dims, seed=107)[0]
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    weo.wilson_eo_set_algorithm(op.handle, "fused", 4, 128)
    x = to_device(to_planar(psi), "f32")
    y = torch.empty_like(x)
    weo.wilson_eo_inject_fused_timeout(op.handle, y, x)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_check(op.handle)
    assert e.value.status == -7
    weo.wilson_eo_check(op.handle)  # the record was cleared
    y = op.apply(x)
    weo.wilson_eo_check(op.handle)
    assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U, 0.12, psi, dims)) <= TOL["f32"]
    op.close()
