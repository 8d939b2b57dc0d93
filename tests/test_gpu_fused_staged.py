"""The fused staged M_eo (wilson_eo_set_algorithm(h, 2)): both hops of Eq. 4 in
one persistent launch fed by TMA, first-hop tiles running ahead of second-hop
tiles in a wavefront over t-slices, links from pair blocks shared by the hops.

Against the oracle on lattices from 4^4 to tiles of 64 sites (halo rows that
wrap, Lt = 2, Lz = 2), for lookaheads 1, 2, 4, both M_eo and M_eo^dag; bitwise
against two TMA-staged hop launches (the same per-direction arithmetic and
summation order); inside the mixed solver; after set_gauge; its write set; the
failure path of its bounded waits; and the handles it refuses."""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 4), (8, 4, 6, 6), (8, 8, 8, 8), (16, 2, 4, 4), (12, 6, 4, 8), (24, 8, 2, 2),
        (32, 8, 2, 4), (8, 8, 4, 22), (32, 4, 4, 2)]


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("lookahead", [1, 2, 4])
def test_fused_staged_matches_oracle_and_staged_launches(weo, oracle_lib, dims, lookahead):
    U = gen.gauge_field(dims, "smooth", seed=600, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=601)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(psi), "f32")
    weo.wilson_eo_set_staging(op.handle, True)
    weo.wilson_eo_set_launch(op.handle, 128, 1, 0)  # second hop upward, as the fused launch
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    weo.wilson_eo_set_algorithm(op.handle, "fused_staged", lookahead)
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        assert rel_l2(from_planar(y.cpu().numpy()), f(U, 0.13, psi, dims)) <= TOL["f32"]
        assert np.array_equal(y.cpu().numpy(), ref[dag].cpu().numpy())
    op.close()


def test_fused_staged_multi_rhs_set_gauge_and_solver(weo, oracle_lib):
    dims = (8, 8, 8, 8)
    U1 = gen.gauge_field(dims, "haar", seed=602)
    U2 = gen.gauge_field(dims, "smooth", seed=603, eps=0.4)
    psi = gen.gaussian_spinor(dims, nrhs=3, seed=604)
    op = weo.WilsonEO(dims, 0.125, to_device(U1), prec="f32")
    weo.wilson_eo_set_algorithm(op.handle, "fused_staged", 2)
    x = to_device(to_planar(psi), "f32")
    for U in (U1, U2):
        if U is U2:
            op.set_gauge(to_device(U2))  # the pair blocks follow the new field
        y = op.apply(x)
        weo.wilson_eo_check(op.handle)
        got = from_planar(y.cpu().numpy())
        for r in range(3):
            assert rel_l2(got[r], oracle_lib.meo(U, 0.125, psi[r], dims)) <= TOL["f32"]
    b = gen.gaussian_spinor(dims, seed=605)[0]
    xs, info = op.solve(to_device(to_planar(b)), tol=0.99e-10, mixed=True)
    weo.wilson_eo_check(op.handle)
    assert info["converged"]
    xg = from_planar(xs.cpu().numpy())
    ax = oracle_lib.meo_dag(U2, 0.125, oracle_lib.meo(U2, 0.125, xg, dims), dims)
    assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= 1e-10
    op.close()


def test_fused_staged_write_set(weo):
    import torch

    dims = (8, 4, 6, 6)
    U = gen.gauge_field(dims, "haar", seed=606)
    psi = gen.gaussian_spinor(dims, seed=607)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_algorithm(op.handle, "fused_staged", 1)
    x = to_device(to_planar(psi), "f32")
    x0 = x.clone()
    guard, n = 4096, x.numel()
    for dag in (False, True):
        buf = torch.full((n + 2 * guard,), complex(float("nan"), 7.0), dtype=torch.complex64, device="cuda")
        y = buf[guard:guard + n].view(x.shape)
        (weo.wilson_eo_apply_dag if dag else weo.wilson_eo_apply)(op.handle, y, x, 1)
        weo.wilson_eo_check(op.handle)
        torch.cuda.synchronize()
        sentinel = torch.isnan(buf.real) & (buf.imag == 7.0)
        assert not bool(sentinel[guard:guard + n].any())
        assert bool(sentinel[:guard].all()) and bool(sentinel[guard + n:].all())
        assert torch.equal(x, x0)
    op.close()


def test_fused_staged_bounded_wait_reports_timeout_and_recovers(weo, oracle_lib):
    """First-hop tiles never publish; the producers' bounded waits give up, every
    consumer group is stopped, wilson_eo_check reports WEO_ERR_TIMEOUT once, and
    the next apply on the same context is correct."""
    import torch

    dims = (8, 8, 8, 16)
    U = gen.gauge_field(dims, "haar", seed=608)
    psi = gen.gaussian_spinor(dims, seed=609)[0]
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    weo.wilson_eo_set_algorithm(op.handle, "fused_staged", 2)
    x = to_device(to_planar(psi), "f32")
    y = op.apply(x)  # builds the pair blocks
    weo.wilson_eo_check(op.handle)
    weo.wilson_eo_inject_fused_timeout(op.handle, y, x)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_check(op.handle)
    assert e.value.status == -7
    weo.wilson_eo_check(op.handle)
    y = op.apply(x)
    weo.wilson_eo_check(op.handle)
    torch.cuda.synchronize()
    assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U, 0.12, psi, dims)) <= TOL["f32"]
    op.close()


def test_fused_staged_refuses_other_handles(weo):
    for prec, fmt, dims in (("f64", 18, (4, 4, 4, 4)), ("f16", 18, (4, 4, 4, 4)), ("f32", 12, (4, 4, 4, 4)),
                            ("f32", 18, (6, 4, 4, 4))):  # Lx/2 odd: rows cannot start on 16 B
        U = gen.gauge_field(dims, "haar", seed=610)
        op = weo.WilsonEO(dims, 0.1, to_device(U), prec=prec, linkfmt=fmt)
        with pytest.raises(weo.WilsonEOError) as e:
            weo.wilson_eo_set_algorithm(op.handle, "fused_staged")
        assert e.value.status == -3
        op.close()
