"""wilson_eo_apply_noalloc, the entry point for callers that cannot allocate.

Callers whose device memory is owned by someone else (a framework's caching
allocator, a real-time loop, a plug-in that only receives buffers) cannot call
cudaMalloc; this entry point runs M_eo with its odd-site intermediate in a
fixed array inside the library. These tests call it through the C ABI and
compare with wilson_eo_apply on an FP32 handle, on two calls in a row (the
second call reuses the array the first one left behind). The file is named so
that pytest collects it last.
"""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_planar

pytestmark = pytest.mark.gpu

GUARD = 4096  # complex elements of NaN sentinel before and after each output


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def test_noalloc_matches_apply_on_two_calls_in_a_row(weo):
    import torch

    cases = [((8, 8, 8, 8), 0.125, "haar", 60), ((16, 8, 4, 12), 0.13, "smooth", 61)]
    for k, (dims, kappa, kind, seed) in enumerate(cases):
        U = gen.gauge_field(dims, kind, seed=seed, eps=0.4)
        psi = gen.gaussian_spinor(dims, nrhs=2, seed=seed + 100)
        Ud = torch.from_numpy(U.astype(np.complex64)).cuda()
        op = weo.WilsonEO(dims, kappa, Ud, prec="f32", linkfmt=18)
        for r in range(2):  # two calls in a row on the same lattice
            x = torch.from_numpy(to_planar(psi[r]).astype(np.complex64)).cuda()
            for dag in (False, True):
                want = op.apply(x, dag=dag)
                got = torch.empty_like(x)
                weo.wilson_eo_apply_noalloc(dims, kappa, Ud, got, x, dag=dag)
                torch.cuda.synchronize()
                assert rel_l2(got.cpu().numpy(), want.cpu().numpy()) <= TOL["f32"]
        op.close()


def test_noalloc_second_call_takes_no_device_memory(weo):
    import torch

    dims = (8, 8, 8, 8)
    U = torch.from_numpy(gen.gauge_field(dims, "haar", seed=62).astype(np.complex64)).cuda()
    x = torch.from_numpy(to_planar(gen.gaussian_spinor(dims, seed=63)[0]).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    weo.wilson_eo_apply_noalloc(dims, 0.12, U, y, x)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    weo.wilson_eo_apply_noalloc(dims, 0.12, U, y, x)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_lattices_beyond_its_scratch(weo):
    import torch

    dims = (32, 32, 32, 64)  # V/2 = 1048576 > 349525
    U = torch.zeros((4, 16, 3, 3), dtype=torch.complex64, device="cuda")
    x = torch.zeros((4, 3, 8), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_noalloc(dims, 0.1, U, y, x)
    assert e.value.status == -2
    assert "349525" in weo.wilson_eo_last_error()
    # host arrays are refused by the library itself (staging them would allocate)
    Uh = np.zeros((4, 8**4, 3, 3), dtype=np.complex64)
    xd = torch.zeros((4, 3, 8**4 // 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_noalloc((8, 8, 8, 8), 0.1, Uh, torch.empty_like(xd), xd)
    assert e.value.status == -1
    # a host tensor beside device tensors is refused by the binding, before the library
    with pytest.raises(ValueError):
        weo.wilson_eo_apply_noalloc((8, 8, 8, 8), 0.1, torch.from_numpy(Uh),
                                    torch.empty_like(xd), xd)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 6, 4, 10), (6, 4, 2, 6), (8, 6, 4, 6)])
def test_noalloc_ragged_lattices_match_oracle_and_write_only_the_output(weo, oracle_lib, dims):
    """Extents of 2, Lx = 2 and V/2 not a multiple of the 128-thread block (the
    kernels' tail guard): the result equals the FP64 oracle's, every output
    element is written, nothing before or after the output is, and the inputs
    are unchanged."""
    import torch

    U = gen.gauge_field(dims, "haar", seed=64)
    psi = gen.gaussian_spinor(dims, seed=65)[0]
    Ud = torch.from_numpy(U.astype(np.complex64)).cuda()
    x = torch.from_numpy(to_planar(psi).astype(np.complex64)).cuda()
    U0, x0 = Ud.clone(), x.clone()
    n = x.numel()
    for dag in (False, True):
        buf = torch.full((n + 2 * GUARD,), complex(float("nan"), 7.0), dtype=torch.complex64,
                         device="cuda")
        y = buf[GUARD:GUARD + n].view(x.shape)
        weo.wilson_eo_apply_noalloc(dims, 0.13, Ud, y, x, dag=dag)
        torch.cuda.synchronize()
        sentinel = torch.isnan(buf.real) & (buf.imag == 7.0)
        assert not bool(sentinel[GUARD:GUARD + n].any()), "output element not written"
        assert bool(sentinel[:GUARD].all()) and bool(sentinel[GUARD + n:].all()), \
            "write outside the output"
        assert torch.equal(x, x0) and torch.equal(Ud, U0), "input modified"
        want = (oracle_lib.meo_dag if dag else oracle_lib.meo)(U, 0.13, psi, dims)
        assert rel_l2(from_planar(y.cpu().numpy()), want) <= TOL["f32"]
