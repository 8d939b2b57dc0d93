"""Write-set checks (compute-sanitizer is not available on the GPU pool): every
output element is written, nothing outside the output arrays is, and inputs
stay untouched. Outputs are views into larger buffers whose guard zones before
and after hold a NaN sentinel; outputs start filled with the sentinel too. Small
lattices with extents of 2, Lx = 2 and V/2 not a multiple of the CTA size."""

import numpy as np
import pytest

import gen
from gpu_util import to_device, to_planar

pytestmark = pytest.mark.gpu

GUARD = 4096  # complex elements on each side


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def guarded(shape, dtype):
    """(buffer, view): view has `shape`, buffer adds GUARD elements on each side;
    everything holds a NaN sentinel."""
    import torch

    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), complex(float("nan"), 7.0), dtype=dtype, device="cuda")
    return buf, buf[GUARD:GUARD + n].view(shape)


def sentinel_mask(t):
    import torch

    return torch.isnan(t.real) & (t.imag == 7.0)


def check_guards(buf, n):
    assert bool(sentinel_mask(buf[:GUARD]).all()), "write before the output array"
    assert bool(sentinel_mask(buf[GUARD + n:]).all()), "write after the output array"


DIMS = [(2, 2, 2, 2), (2, 6, 4, 10), (6, 4, 2, 6)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("prec,fmt,algo", [("f64", 18, 0), ("f32", 18, 0), ("f32", 12, 1),
                                           ("f16", 18, 0), ("bf16", 12, 1)])
def test_apply_writes_exactly_its_output(weo, dims, prec, fmt, algo):
    import torch

    U = gen.gauge_field(dims, "haar", seed=150)
    psi = gen.gaussian_spinor(dims, nrhs=3, seed=151)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec=prec, linkfmt=fmt)
    if algo:
        weo.wilson_eo_set_algorithm(op.handle, "fused", 1, 128)
    dt = torch.complex128 if prec == "f64" else torch.complex64
    x = to_device(to_planar(psi)).to(dt)
    x0 = x.clone()
    for dag in (False, True):
        buf, y = guarded(tuple(x.shape), dt)
        (weo.wilson_eo_apply_dag if dag else weo.wilson_eo_apply)(op.handle, y, x, 3)
        if algo:
            weo.wilson_eo_check(op.handle)
        torch.cuda.synchronize()
        assert not bool(sentinel_mask(y).any()), "output element not written"
        check_guards(buf, y.numel())
        assert torch.equal(x, x0), "input modified"
    op.close()


@pytest.mark.parametrize("dims", DIMS)
def test_ff_hop_and_batch_write_sets(weo, dims):
    import torch

    U = gen.gauge_field(dims, "haar", seed=152)
    psi = gen.gaussian_spinor(dims, nrhs=2, seed=153)
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    x64 = to_device(to_planar(psi)).to(torch.complex128)
    buf, y = guarded(tuple(x64.shape), torch.complex128)
    weo.wilson_eo_apply_ff64(op.handle, y, x64, 2)
    torch.cuda.synchronize()
    assert not bool(sentinel_mask(y).any())
    check_guards(buf, y.numel())
    x = x64.to(torch.complex64)
    for parity in (0, 1):
        buf, y = guarded(tuple(x.shape), torch.complex64)
        weo.wilson_eo_hop(op.handle, parity, False, y, x, 2)
        torch.cuda.synchronize()
        assert not bool(sentinel_mask(y).any())
        check_guards(buf, y.numel())
    buf, y = guarded(tuple(x.shape), torch.complex64)
    weo.wilson_eo_apply_batch_rhs([op.handle], [y], [x], [2])
    torch.cuda.synchronize()
    assert not bool(sentinel_mask(y).any())
    check_guards(buf, y.numel())
    op.close()


@pytest.mark.parametrize("dims", DIMS)
def test_link_gradient_writes_exactly_its_output(weo, dims):
    import torch

    U = gen.gauge_field(dims, "haar", seed=154)
    g = to_device(to_planar(gen.gaussian_spinor(dims, seed=155)[0])).to(torch.complex64)
    phi = to_device(to_planar(gen.gaussian_spinor(dims, seed=156)[0])).to(torch.complex64)
    op = weo.WilsonEO(dims, 0.12, to_device(U), prec="f32")
    V = int(np.prod(dims))
    buf, out = guarded((4, V, 3, 3), torch.complex64)
    weo.wilson_eo_link_grad(op.handle, out, g, phi)
    torch.cuda.synchronize()
    assert not bool(sentinel_mask(out).any())
    check_guards(buf, out.numel())
    op.close()


@pytest.mark.parametrize("dims", [(4, 4, 2, 6), (8, 2, 2, 2), (16, 6, 2, 4)])
@pytest.mark.parametrize("mode,nrhs", [(1, 1), (2, 3)])
def test_staged_hop_writes_exactly_its_output(weo, dims, mode, nrhs):
    """The TMA-staged hop (tiles of 8, 8 and 48 sites; one right-hand side, and
    the multi-RHS kernel): M_eo, M_eo^dag and single hops of both parities."""
    import torch

    U = gen.gauge_field(dims, "haar", seed=153)
    psi = gen.gaussian_spinor(dims, nrhs=nrhs, seed=154)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    weo.wilson_eo_set_staging(op.handle, mode)
    x = to_device(to_planar(psi), "f32")
    if nrhs == 1:
        x = x[0]
    x0 = x.clone()
    calls = [lambda y: weo.wilson_eo_apply(op.handle, y, x, nrhs),
             lambda y: weo.wilson_eo_apply_dag(op.handle, y, x, nrhs)]
    for par in (0, 1):
        calls.append(lambda y, par=par: weo.wilson_eo_hop(op.handle, par, False, y, x, nrhs))
    for call in calls:
        buf, y = guarded(tuple(x.shape), torch.complex64)
        call(y)
        weo.wilson_eo_check(op.handle)
        torch.cuda.synchronize()
        assert not bool(sentinel_mask(y).any()), "output element not written"
        check_guards(buf, y.numel())
        assert torch.equal(x, x0), "input modified"
    op.close()
