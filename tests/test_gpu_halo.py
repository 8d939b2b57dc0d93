"""The domain-decomposed hop with forced exchange (pack / exchange / bulk /
finish) equals the unsplit hop and the oracle, for 1 rank (self-exchange of
the periodic wrap), several ranks, and one t-slice per rank (both faces of a
sub-domain on the same slice)."""

import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims,ranks", [((4, 4, 4, 8), 1), ((4, 4, 4, 8), 2), ((4, 6, 2, 8), 4),
                                        ((4, 4, 2, 6), 6), ((8, 8, 8, 16), 2), ((4, 4, 4, 2), 2)])
def test_split_hop_equals_unsplit(oracle_lib, prec, dims, ranks):
    import torch

    import paper_2303_08609_gb300 as weo

    U = gen.gauge_field(dims, "haar", seed=110)
    psi = gen.gaussian_spinor(dims, seed=111)[0]
    op = weo.WilsonEO(dims, 0.1, to_device(U), prec=prec)
    x = to_device(to_planar(psi), prec)
    for parity in (0, 1):
        for dag in (False, True):
            ref = op.hop(x, parity, dag=dag)
            y = torch.empty_like(x)
            weo.wilson_eo_hop_split(op.handle, ranks, parity, dag, y, x)
            torch.cuda.synchronize()
            assert rel_l2(y.cpu().numpy(), ref.cpu().numpy()) <= (1e-14 if prec == "f64" else 1e-6)
            f = oracle_lib.hop_adj if dag else oracle_lib.hop
            assert rel_l2(from_planar(y.cpu().numpy()), f(U, psi, dims, parity)) <= TOL[prec]
    op.close()


def test_split_rejects_bad_rank_count():
    import torch

    import paper_2303_08609_gb300 as weo

    dims = (4, 4, 4, 8)
    op = weo.WilsonEO(dims, 0.1, to_device(gen.gauge_field(dims, "haar", seed=1)), prec="f32")
    x = torch.zeros((4, 3, 256), dtype=torch.complex64, device="cuda")
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_hop_split(op.handle, 3, 0, False, torch.empty_like(x), x)
    assert e.value.status == -1
    op.close()
