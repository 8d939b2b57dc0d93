"""The blocked site order of the one-site-per-thread hops
(wilson_eo_set_site_blocks): CTAs of 8 Lx/2 threads over 2x2x2 blocks of rows.
The per-site arithmetic is unchanged, so every result is bitwise equal to the
default order's, and matches the FP64 oracle, for every storage precision, one
and several right-hand sides, and both walking orders of the second hop."""

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


@pytest.mark.parametrize("dims", [(16, 4, 6, 8), (32, 2, 2, 4), (24, 6, 4, 2)])
@pytest.mark.parametrize("prec,fmt", [("f64", 18), ("f32", 18), ("f32", 12), ("f16", 12), ("bf16", 18)])
def test_blocked_order_bitwise_and_oracle(weo, oracle_lib, dims, prec, fmt):
    U = gen.gauge_field(dims, "smooth", seed=700, eps=0.4)
    psi = gen.gaussian_spinor(dims, nrhs=3, seed=701)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec=prec, linkfmt=fmt)
    x = to_device(to_planar(psi), "f64" if prec == "f64" else "f32")
    for order in (0, 1):
        for rb in ((1, 2) if prec != "f64" else (1,)):
            weo.wilson_eo_set_launch(op.handle, 128, rb, order)
            weo.wilson_eo_set_site_blocks(op.handle, False)
            ref = {d: op.apply(x, dag=d).cpu().numpy() for d in (False, True)}
            weo.wilson_eo_set_site_blocks(op.handle, True)
            for dag in (False, True):
                y = op.apply(x, dag=dag).cpu().numpy()
                assert np.array_equal(y, ref[dag])
                f = oracle_lib.meo_dag if dag else oracle_lib.meo
                got = from_planar(y)
                for r in range(3):
                    assert rel_l2(got[r], f(U, 0.13, psi[r], dims)) <= TOL[prec]
    assert weo.library().wilson_eo_set_site_blocks(op.handle, 2) == -1
    op.close()
