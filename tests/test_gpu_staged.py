"""The TMA-staged hopping kernel (tiles of R rows; neighbour rows, links and
the addend loaded as cp.async.bulk.tensor boxes into a three-stage ring) against
the oracle, for tile shapes from 8 to 64 sites (R = 2 .. 16 rows, halo rows that
wrap onto the tile itself when R = Ly), both parities, both projector pairings,
and both walking orders; at 32^3 x 64 on sampled sites; inside the solver and
the force; on lattices it cannot take; and on the failure path of its bounded
waits."""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu

DIMS = [(4, 4, 4, 4), (8, 4, 6, 6), (8, 8, 8, 8), (16, 2, 4, 4), (12, 6, 4, 8), (24, 8, 2, 2),
        (32, 8, 2, 4), (48, 4, 2, 2), (8, 8, 4, 22)]


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.mark.parametrize("dims", DIMS)
def test_staged_hop_matches_oracle(weo, oracle_lib, dims):
    U = gen.gauge_field(dims, "haar", seed=300)
    psi = gen.gaussian_spinor(dims, seed=301)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(psi), "f32")
    ref = {(par, dag): op.hop(x, par, dag=dag) for par in (0, 1) for dag in (False, True)}
    weo.wilson_eo_set_staging(op.handle, True)
    assert weo.wilson_eo_get_staging(op.handle)["staged"]
    for par in (0, 1):
        for dag in (False, True):
            y = op.hop(x, par, dag=dag)
            weo.wilson_eo_check(op.handle)
            want = oracle_lib.hop(U, psi, dims, par, sign=-1 if dag else 1)
            assert rel_l2(from_planar(y.cpu().numpy()), want) <= TOL["f32"]
            # same per-direction arithmetic, halves added in another order
            assert rel_l2(y.cpu().numpy(), ref[(par, dag)].cpu().numpy()) <= 1e-6
    op.close()


@pytest.mark.parametrize("dims", DIMS[:6])
@pytest.mark.parametrize("order", [0, 1])
def test_staged_meo_matches_oracle(weo, oracle_lib, dims, order):
    U = gen.gauge_field(dims, "smooth", seed=302, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=303)[0]
    op = weo.WilsonEO(dims, 0.125, to_device(U), prec="f32")
    weo.wilson_eo_set_launch(op.handle, 128, 1, order)
    weo.wilson_eo_set_staging(op.handle, True)
    x = to_device(to_planar(psi), "f32")
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        assert rel_l2(from_planar(y.cpu().numpy()), f(U, 0.125, psi, dims)) <= TOL["f32"]
    op.close()


def test_staged_full_size_sampled(weo, oracle_lib, fields_32x64):
    """32^3 x 64 (tiles of 4 rows = 64 sites, 16384 tiles over 152 CTAs)."""
    import torch

    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    dims, U, _ = fields_32x64  # smooth links, seed 0
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(psi), "f32")
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    weo.wilson_eo_set_staging(op.handle, True)
    sites = np.sort(gen.rng(3).choice(vh, 300, replace=False))
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        got = from_planar(y[:, :, torch.from_numpy(sites).cuda()].cpu().numpy())
        assert rel_l2(got, oracle_lib.meo_sites(U, 0.13, psi, dims, sites, dag=dag)) <= TOL["f32"]
        assert rel_l2(y.cpu().numpy(), ref[dag].cpu().numpy()) <= 1e-6
    op.close()


def test_staged_in_solver_and_force(weo, oracle_lib):
    """An FP64 handle's mixed solve, whose FP32 inner operator runs staged, to
    the FP64 oracle's true residual; and the force of an FP32 handle."""
    import torch

    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, "smooth", seed=304, eps=0.4)
    b = gen.gaussian_spinor(dims, seed=305)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f64")
    weo.wilson_eo_set_staging(op.handle, True)
    xs, info = op.solve(to_device(to_planar(b)), tol=1e-10, mixed=True)
    weo.wilson_eo_check(op.handle)
    assert info["converged"]
    xg = from_planar(xs.cpu().numpy())
    ax = oracle_lib.meo_dag(U, 0.13, oracle_lib.meo(U, 0.13, xg, dims), dims)
    assert np.linalg.norm(b - ax) / np.linalg.norm(b) <= 1.5e-10
    op.close()

    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    phi = to_device(to_planar(b), "f32")
    F0, _ = op.force(phi)
    weo.wilson_eo_set_staging(op.handle, True)
    F1, _ = op.force(phi)
    weo.wilson_eo_check(op.handle)
    assert float(torch.linalg.norm(F1 - F0) / torch.linalg.norm(F0)) <= 1e-5
    op.close()


@pytest.mark.parametrize("dims,prec,fmt", [((6, 4, 4, 4), "f32", 18), ((2, 4, 4, 4), "f32", 18),
                                           ((4, 6, 6, 4), "f32", 18)])
def test_staged_rejects_ineligible_lattices(weo, dims, prec, fmt):
    """Lx/2 odd (rows would start off 16-byte boundaries) is refused with
    WEO_ERR_UNSUPPORTED; Lx/2 = 2 with Ly = 6 (R = 6) is taken."""
    op = weo.WilsonEO(dims, 0.1, to_device(gen.gauge_field(dims, "haar", seed=1)), prec=prec,
                      linkfmt=fmt)
    if (dims[0] // 2) % 2:
        with pytest.raises(weo.WilsonEOError) as e:
            weo.wilson_eo_set_staging(op.handle, True)
        assert e.value.status == -3
        assert weo.wilson_eo_get_staging(op.handle) == {"staged": 0, "rows": 0, "depth": 0}
    else:
        weo.wilson_eo_set_staging(op.handle, True)
    op.close()


def test_staged_other_formats_keep_the_default_kernel(weo, oracle_lib):
    """Staging on, but 12-real links / FP16 storage / two right-hand sides
    (multi-RHS hops are staged only with staged = 2): the default kernels run
    and the results stay correct."""
    dims = (8, 8, 8, 8)
    U = gen.gauge_field(dims, "smooth", seed=306, eps=0.4)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=307)
    for prec, fmt in (("f32", 12), ("f16", 18), ("f32", 18)):
        op = weo.WilsonEO(dims, 0.125, to_device(U), prec=prec, linkfmt=fmt)
        weo.wilson_eo_set_staging(op.handle, True)
        y = op.apply(to_device(to_planar(psi), "f32"))
        weo.wilson_eo_check(op.handle)
        for r in range(2):
            assert rel_l2(from_planar(y[r].cpu().numpy()),
                          oracle_lib.meo(U, 0.125, psi[r], dims)) <= TOL[prec]
        op.close()


def test_staged_bounded_wait_reports_timeout_and_recovers(weo, oracle_lib):
    """Failure detection without a fault: the producer never loads each CTA's
    first tile, the consumers' bounded waits run out (2 ms), the producer gives
    up on the stage they never release and waits for its own loads in flight;
    wilson_eo_check reports WEO_ERR_TIMEOUT once and the next staged hop on the
    same context is correct."""
    import torch

    dims = (16, 16, 16, 16)
    U = gen.gauge_field(dims, "haar", seed=308)
    psi = gen.gaussian_spinor(dims, seed=309)[0]
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    weo.wilson_eo_set_staging(op.handle, True)
    x = to_device(to_planar(psi), "f32")
    y = torch.empty_like(x)
    weo.wilson_eo_inject_staged_timeout(op.handle, y, x)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_check(op.handle)
    assert e.value.status == -7
    weo.wilson_eo_check(op.handle)  # the record was cleared
    y = op.hop(x, 1)
    weo.wilson_eo_check(op.handle)
    assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.hop(U, psi, dims, 1)) <= TOL["f32"]
    op.close()


@pytest.mark.parametrize("rows,depth", [(2, 2), (2, 3), (2, 5), (4, 2), (4, 4), (8, 2), (8, 3)])
def test_staged_tile_and_ring_shapes(weo, oracle_lib, rows, depth):
    """16^4: tiles of 16, 32 and 64 sites (one or two teams per tile, six or
    three tiles computed at once) with rings of 2 to 5 stages."""
    dims = (16, 16, 16, 16)
    U = gen.gauge_field(dims, "smooth", seed=310, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=311)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_staging(op.handle, True, rows, depth)
    assert weo.wilson_eo_get_staging(op.handle) == {"staged": 1, "rows": rows, "depth": depth}
    x = to_device(to_planar(psi), "f32")
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        assert rel_l2(from_planar(y.cpu().numpy()), f(U, 0.13, psi, dims)) <= TOL["f32"]
    op.close()


def test_staged_rejects_shapes_that_do_not_fit(weo):
    dims = (32, 8, 4, 4)
    op = weo.WilsonEO(dims, 0.1, to_device(gen.gauge_field(dims, "haar", seed=2)), prec="f32")
    for rows, depth in ((4, 4), (3, 0), (16, 0)):  # 4 x 77 KB; 3 does not divide 8; 256 sites
        with pytest.raises(weo.WilsonEOError) as e:
            weo.wilson_eo_set_staging(op.handle, True, rows, depth)
        assert e.value.status == -3
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_set_staging(op.handle, True, 0, 6)
    assert e.value.status == -1
    assert weo.wilson_eo_get_staging(op.handle) == {"staged": 0, "rows": 4, "depth": 3}
    op.close()


def test_tuner_considers_the_staged_hop(weo, oracle_lib):
    """wilson_eo_tune with one right-hand side times the staged hop beside the
    other configurations; whichever wins, M_eo stays correct."""
    dims = (16, 16, 16, 16)
    U = gen.gauge_field(dims, "smooth", seed=312, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=313)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    threads, rb, ms = weo.wilson_eo_tune(op.handle, nrhs=1)
    assert ms > 0
    st = weo.wilson_eo_get_staging(op.handle)
    assert st["rows"] == 8 and st["depth"] == 3
    y = op.apply(to_device(to_planar(psi), "f32"))
    weo.wilson_eo_check(op.handle)
    assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U, 0.13, psi, dims)) <= TOL["f32"]
    if not st["staged"]:
        assert op.info()["device_bytes"] < 60 * 2**20  # the trial's link blocks (36 MiB) were released
    op.close()


def test_staged_is_deterministic(weo):
    """Fixed accumulation order (x/y half plus z/t half, per site): repeated
    applies and applies on another stream give identical bits."""
    import torch

    dims = (32, 8, 8, 8)
    U = to_device(gen.gauge_field(dims, "haar", seed=316))
    x = to_device(to_planar(gen.gaussian_spinor(dims, seed=317)[0]), "f32")
    op = weo.WilsonEO(dims, 0.13, U, prec="f32")
    weo.wilson_eo_set_staging(op.handle, True)
    y0 = op.apply(x)
    s = torch.cuda.Stream()
    for k in range(3):
        y = op.apply(x) if k % 2 == 0 else op.apply(x, stream=s)
        torch.cuda.synchronize()
        assert torch.equal(y, y0)
    weo.wilson_eo_check(op.handle)
    op.close()


@pytest.mark.parametrize("dims,nrhs", [((8, 8, 8, 8), 2), ((16, 16, 16, 16), 3), ((16, 8, 4, 6), 5),
                                       ((16, 16, 16, 16), 12), ((4, 4, 4, 4), 7)])
def test_staged_multi_rhs_matches_oracle(weo, oracle_lib, dims, nrhs):
    """Several right-hand sides: each tile's link block is loaded once and
    serves every right-hand side (rings of 2 or 3 spinor stages), for M_eo,
    M_eo^dag and single hops of both parities, against the oracle and the
    default multi-RHS kernels."""
    U = gen.gauge_field(dims, "haar", seed=318)
    psi = gen.gaussian_spinor(dims, nrhs=nrhs, seed=319)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(psi), "f32")
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    href = op.hop(x, 1)
    weo.wilson_eo_set_staging(op.handle, 2)
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(nrhs):
            assert rel_l2(from_planar(y[r].cpu().numpy()), f(U, 0.13, psi[r], dims)) <= TOL["f32"]
        assert rel_l2(y.cpu().numpy(), ref[dag].cpu().numpy()) <= 1e-6
    h = op.hop(x, 1)
    weo.wilson_eo_check(op.handle)
    assert rel_l2(h.cpu().numpy(), href.cpu().numpy()) <= 1e-6
    op.close()


def test_staged_multi_rhs_full_size_sampled(weo, oracle_lib, fields_32x64):
    """32^3 x 64 with 12 point-source-like right-hand sides (Gaussian here),
    sampled sites of every right-hand side against the oracle."""
    import torch

    dims = (32, 32, 32, 64)
    vh = int(np.prod(dims)) // 2
    dims, U, _ = fields_32x64  # smooth links, seed 0
    psi = gen.gaussian_spinor(dims, nrhs=12, seed=320)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_staging(op.handle, 2)
    x = to_device(to_planar(psi), "f32")
    y = op.apply(x)
    weo.wilson_eo_check(op.handle)
    sites = np.sort(gen.rng(4).choice(vh, 60, replace=False))
    got = from_planar(y[:, :, :, torch.from_numpy(sites).cuda()].cpu().numpy())
    for r in (0, 5, 11):
        want = oracle_lib.meo_sites(U, 0.13, psi[r], dims, sites)
        assert rel_l2(got[r], want) <= TOL["f32"]
    op.close()


def test_staged_link_blocks_follow_set_gauge(weo, oracle_lib):
    """The per-tile link blocks are rebuilt after wilson_eo_set_gauge (host and
    device fields), for an FP32 handle's applies and for an FP64 handle's mixed
    solve, whose FP32 inner operator is repacked; never a stale block."""
    dims = (16, 8, 8, 8)
    U0 = gen.gauge_field(dims, "haar", seed=321)
    U1 = gen.gauge_field(dims, "smooth", seed=322, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=323)[0]
    op = weo.WilsonEO(dims, 0.13, to_device(U0), prec="f32")
    weo.wilson_eo_set_staging(op.handle, True)
    x = to_device(to_planar(psi), "f32")
    y = op.apply(x)
    assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U0, 0.13, psi, dims)) <= TOL["f32"]
    for U in (U1, U0):
        op.set_gauge(to_device(U) if U is U1 else U)
        y = op.apply(x)
        weo.wilson_eo_check(op.handle)
        assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U, 0.13, psi, dims)) <= TOL["f32"]
    op.close()

    op = weo.WilsonEO(dims, 0.13, to_device(U0), prec="f64")
    weo.wilson_eo_set_staging(op.handle, True)
    b = to_device(to_planar(psi))
    for U in (U0, U1):
        op.set_gauge(to_device(U))
        xs, info = op.solve(b, tol=1e-10, mixed=True)
        weo.wilson_eo_check(op.handle)
        assert info["converged"]
        xg = from_planar(xs.cpu().numpy())
        ax = oracle_lib.meo_dag(U, 0.13, oracle_lib.meo(U, 0.13, xg, dims), dims)
        assert np.linalg.norm(psi - ax) / np.linalg.norm(psi) <= 1.5e-10
    op.close()
