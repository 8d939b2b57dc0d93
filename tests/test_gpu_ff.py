"""M_eo in float-float arithmetic (wilson_eo_apply_ff64) and the mixed solver's
float-float reliable-update residuals.

The float-float operator carries every real as hi + lo of two floats (about 48
significant bits) and must meet the FP64 bar against the FP64 oracle (relative
L2 <= 1e-12) -- it does so with a wide margin -- on small lattices in full,
ragged lattices, several right-hand sides, both adjoints, host and device
arrays, handles of every storage precision, and sampled sites of 32^3 x 64."""

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


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (2, 6, 4, 10), (8, 4, 6, 6), (4, 4, 4, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
def test_ff_matches_oracle_at_fp64_accuracy(weo, oracle_lib, dims, prec):
    U = gen.gauge_field(dims, "haar", seed=130)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=131)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec=prec)
    x = to_device(to_planar(psi), "f64")
    for dag in (False, True):
        y = op.apply_ff64(x, dag=dag)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(2):
            err = rel_l2(from_planar(y[r].cpu().numpy()), f(U, 0.13, psi[r], dims))
            assert err <= TOL["f64"], err
            assert err <= 1e-13, err  # float-float keeps ~48 bits, far below FP32's 1e-7
    op.close()


def test_ff_host_arrays_and_set_gauge(weo, oracle_lib):
    dims = (4, 6, 4, 8)
    U1 = gen.gauge_field(dims, "smooth", seed=132, eps=0.4)
    U2 = gen.gauge_field(dims, "haar", seed=133)
    psi = gen.gaussian_spinor(dims, seed=134)[0]
    op = weo.WilsonEO(dims, 0.125, to_device(U1), prec="f64")
    x = to_planar(psi)
    y = np.zeros_like(x)
    weo.wilson_eo_apply_ff64(op.handle, y, x)
    assert rel_l2(from_planar(y), oracle_lib.meo(U1, 0.125, psi, dims)) <= 1e-13
    op.set_gauge(to_device(U2))  # the float-float links follow the new field
    weo.wilson_eo_apply_ff64(op.handle, y, x, dag=True)
    assert rel_l2(from_planar(y), oracle_lib.meo_dag(U2, 0.125, psi, dims)) <= 1e-13
    op.close()


def test_ff_full_size_sampled(weo, oracle_lib, fields_32x64):
    import torch

    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    dims, U, _ = fields_32x64  # smooth links, seed 0
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f64")
    x = to_device(to_planar(psi), "f64")
    y = op.apply_ff64(x)
    y64 = op.apply(x)
    assert rel_l2(y.cpu().numpy(), y64.cpu().numpy()) <= 1e-13
    sites = np.sort(gen.rng(4).choice(vh, 200, replace=False))
    got = from_planar(y[:, :, torch.from_numpy(sites).cuda()].cpu().numpy())
    assert rel_l2(got, oracle_lib.meo_sites(U, 0.13, psi, dims, sites)) <= 1e-13
    op.close()


@pytest.mark.parametrize("prec", ["f16", "f32"])
def test_mixed_solve_with_ff_residuals(weo, oracle_lib, prec):
    """Reliable updates with float-float residuals reach the same FP64-checked
    tolerance as with native FP64 residuals, with far fewer FP64 applications."""
    import torch

    dims = (8, 8, 8, 16)
    kappa = 0.13
    U = gen.gauge_field(dims, "smooth", seed=135, eps=0.4)
    b = gen.gaussian_spinor(dims, seed=136)[0]
    bd = to_device(to_planar(b), "f64")
    res = {}
    for mode in (1, 0):
        op = weo.WilsonEO(dims, kappa, to_device(U), prec=prec)
        weo.wilson_eo_solver_residual(op.handle, mode)
        x, info = op.solve(bd, tol=1e-10, maxiter=5000, mixed=True)
        assert info["converged"], info
        xg = from_planar(x.cpu().numpy())
        ax = oracle_lib.meo_dag(U, kappa, oracle_lib.meo(U, kappa, xg, dims), dims)
        assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= 1.5e-10
        res[mode] = info
        op.close()
    # a zero initial guess starts from r = b with no operator application; every
    # reliable update then forms one true residual (float-float in mode 1, with
    # at most a native FP64 confirmation of convergence; native FP64 in mode 0)
    assert res[1]["ff_applies"] >= res[1]["reliable_updates"]
    assert res[1]["fp64_applies"] <= 2 and res[0]["ff_applies"] == 0
    assert res[0]["fp64_applies"] == res[0]["reliable_updates"]
    assert abs(res[1]["iterations"] - res[0]["iterations"]) <= 16


def test_handle_releases_float_float_fields(weo):
    """Device memory taken by the float-float gauge field, work fields and the
    solver's float-float vectors comes back when the handle is destroyed."""
    import torch

    dims = (16, 16, 16, 16)
    U = to_device(gen.gauge_field(dims, "haar", seed=137))
    b = to_device(to_planar(gen.gaussian_spinor(dims, seed=138)[0]), "f64")
    def round_trip():
        op = weo.WilsonEO(dims, 0.12, U, prec="f16")
        op.apply_ff64(b)
        x, info = op.solve(b, tol=1e-10, mixed=True)
        assert info["converged"] and info["ff_applies"] >= 1
        del x
        op.close()

    # the first round loads the kernels' modules and sizes the local-memory
    # pool, which the driver keeps; measure from there
    round_trip()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):  # a leak of the solver's float-float fields alone is 25 MB a round
        round_trip()
    torch.cuda.synchronize()
    assert free0 - torch.cuda.mem_get_info()[0] < 32 << 20


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (6, 2, 4, 2)])
def test_ff_smallest_lattices(weo, oracle_lib, dims):
    """Extents of 2 (every neighbour pair wraps onto the same site) and Lx = 2."""
    U = gen.gauge_field(dims, "haar", seed=139)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=140)
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f64")
    x = to_device(to_planar(psi), "f64")
    for dag in (False, True):
        y = op.apply_ff64(x, dag=dag)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(2):
            assert rel_l2(from_planar(y[r].cpu().numpy()), f(U, 0.12, psi[r], dims)) <= 1e-13
    op.close()
