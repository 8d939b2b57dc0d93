"""Multi-RHS hops over tiles whose links sit in shared memory
(wilson_eo_set_tile_links): every right-hand side against the FP64 oracle,
for 2, 4 and 8 right-hand sides per pass (tiles of 128, 64, 32 sites), FP32
and 16-bit storage, 18- and 12-real links, right-hand-side counts that do and
do not fill a pass, and lattices whose V/2 is not a multiple of the tile (the
last tile is partial) or has extents of 2; plus the write set with NaN-sentinel
guard zones, and the autotuner choosing among these configurations."""

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


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (2, 6, 4, 10), (6, 4, 2, 6), (12, 6, 4, 8)])
@pytest.mark.parametrize("nrl,rpt", [(2, 1), (4, 1), (8, 1), (2, 2), (4, 2)])
@pytest.mark.parametrize("nrhs", [2, 5, 12])
def test_tile_links_matches_oracle_fp32(weo, oracle_lib, dims, nrl, rpt, nrhs):
    """(2 RHS per thread runs when nrhs >= 2 groups; 5 with 2 groups leaves one
    thread group a single right-hand side in its last pass)"""
    U = gen.gauge_field(dims, "haar", seed=500)
    psi = gen.gaussian_spinor(dims, nrhs=nrhs, seed=501)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_tile_links(op.handle, nrl, rpt)
    assert weo.wilson_eo_get_tile_links(op.handle) == (nrl, rpt)
    x = to_device(to_planar(psi), "f32")
    for dag in (False, True):
        got = from_planar(op.apply(x, dag=dag).cpu().numpy())
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(nrhs):
            assert rel_l2(got[r], f(U, 0.13, psi[r], dims)) <= TOL["f32"], (r, dag)
    op.close()


@pytest.mark.parametrize("prec,fmt", [("f32", 12), ("f16", 18), ("f16", 12), ("bf16", 12)])
def test_tile_links_other_formats(weo, oracle_lib, prec, fmt):
    dims = (8, 6, 4, 10)
    U = gen.gauge_field(dims, "smooth", seed=502, eps=0.4)
    psi = gen.gaussian_spinor(dims, nrhs=6, seed=503)
    op = weo.WilsonEO(dims, 0.125, to_device(U), prec=prec, linkfmt=fmt)
    x = to_device(to_planar(psi), "f32")
    ref = {d: op.apply(x, dag=d) for d in (False, True)}
    for rpt in (1, 2):
        weo.wilson_eo_set_tile_links(op.handle, 2, rpt)
        for dag in (False, True):
            y = op.apply(x, dag=dag)
            got = from_planar(y.cpu().numpy())
            f = oracle_lib.meo_dag if dag else oracle_lib.meo
            for r in range(6):
                assert rel_l2(got[r], f(U, 0.125, psi[r], dims)) <= TOL[prec]
            # the same per-site arithmetic as the one-site-per-thread kernel: bitwise equal
            assert np.array_equal(y.cpu().numpy(), ref[dag].cpu().numpy())
    op.close()


@pytest.mark.parametrize("nrl,rpt", [(2, 1), (8, 1), (2, 2)])
def test_tile_links_write_set(weo, nrl, rpt):
    import torch

    dims = (6, 4, 2, 6)
    U = gen.gauge_field(dims, "haar", seed=504)
    psi = gen.gaussian_spinor(dims, nrhs=3, seed=505)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_tile_links(op.handle, nrl, rpt)
    x = to_device(to_planar(psi), "f32")
    x0 = x.clone()
    guard = 4096
    n = x.numel()
    for dag in (False, True):
        buf = torch.full((n + 2 * guard,), complex(float("nan"), 7.0), dtype=torch.complex64, device="cuda")
        y = buf[guard:guard + n].view(x.shape)
        (weo.wilson_eo_apply_dag if dag else weo.wilson_eo_apply)(op.handle, y, x, 3)
        torch.cuda.synchronize()
        sentinel = torch.isnan(buf.real) & (buf.imag == 7.0)
        assert not bool(sentinel[guard:guard + n].any())
        assert bool(sentinel[:guard].all()) and bool(sentinel[guard + n:].all())
        assert torch.equal(x, x0)
    op.close()


def test_tile_links_arguments_and_tuner(weo, oracle_lib):
    dims = (8, 8, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=506)
    psi = gen.gaussian_spinor(dims, nrhs=8, seed=507)
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    for bad, rpt in ((1, 1), (3, 1), (16, 1), (-1, 1), (4, 3), (4, 0)):
        with pytest.raises(weo.WilsonEOError):
            weo.wilson_eo_set_tile_links(op.handle, bad, rpt)
    weo.wilson_eo_tune(op.handle, nrhs=8)
    got = from_planar(op.apply(to_device(to_planar(psi), "f32")).cpu().numpy())
    for r in range(8):
        assert rel_l2(got[r], oracle_lib.meo(U, 0.12, psi[r], dims)) <= TOL["f32"]
    op.close()
    op64 = weo.WilsonEO(dims, 0.12, to_device(U), prec="f64")
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_set_tile_links(op64.handle, 4, 1)
    assert e.value.status == -3
    op64.close()
