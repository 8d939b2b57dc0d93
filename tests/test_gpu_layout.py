"""wilson_eo_spinor_layout: site-major psi[rhs][i][spin][colour] <-> the
library's planar psi[rhs][spin][colour][i], on the device.

The conversion must equal numpy's axis move element by element (a pure
reordering: bit-exact), for both element sizes, several right-hand sides and
half volumes that are not a multiple of the 128-site block; and a caller that
holds site-major spinors gets the oracle's M_eo by converting in and out."""

import numpy as np
import pytest

import gen
from gpu_util import TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("vh,nrhs", [(1, 1), (127, 3), (128, 2), (4099, 5), (8192, 12)])
def test_layout_is_the_axis_move_and_round_trips(weo, dtype, vh, nrhs):
    import torch

    g = np.random.default_rng(vh + nrhs)
    a = (g.standard_normal((nrhs, vh, 4, 3)) + 1j * g.standard_normal((nrhs, vh, 4, 3))).astype(dtype)
    src = torch.from_numpy(a).cuda()
    planar = torch.empty((nrhs, 4, 3, vh), dtype=src.dtype, device="cuda")
    weo.wilson_eo_spinor_layout(planar, src, to_planar=True)
    back = torch.empty_like(src)
    weo.wilson_eo_spinor_layout(back, planar, to_planar=False)
    torch.cuda.synchronize()
    assert np.array_equal(planar.cpu().numpy(), np.moveaxis(a, 1, -1))
    assert torch.equal(back, src)


def test_site_major_caller_gets_the_oracle_meo(weo, oracle_lib):
    import torch

    dims = (6, 4, 4, 8)
    U = gen.gauge_field(dims, "haar", seed=400)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=401)  # (2, V/2, 4, 3): site-major
    op = weo.WilsonEO(dims, 0.13, torch.from_numpy(U).cuda(), prec="f32")
    x_sm = torch.from_numpy(psi.astype(np.complex64)).cuda()
    x = torch.empty((2, 4, 3, op.vh), dtype=torch.complex64, device="cuda")
    weo.wilson_eo_spinor_layout(x, x_sm, to_planar=True)
    y = op.apply(x)
    y_sm = torch.empty_like(x_sm)
    weo.wilson_eo_spinor_layout(y_sm, y, to_planar=False)
    got = y_sm.cpu().numpy()
    for r in range(2):
        assert rel_l2(got[r], oracle_lib.meo(U, 0.13, psi[r], dims)) <= TOL["f32"]
    op.close()
