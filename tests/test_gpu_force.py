"""Link gradient, pseudofermion force and autograd of the CUDA path.

* parity with the oracle's link gradient / force / dS/dphi (FP64 1e-12, FP32 1e-5);
* central finite differences of S = |M_eo phi|^2 evaluated on the GPU in FP64 at
  16^3 x 32 (kappa = 0.13, eps = 0.3 links) on random (link, su(3) direction)
  pairs, summing per-site differences |chi+|^2 - |chi-|^2 so that the large
  unchanged part of S cancels exactly;
* torch.autograd.gradcheck of the differentiable M_eo on a 2^4 lattice.
"""

import numpy as np
import pytest
import scipy.linalg

import gen
from gpu_util import TOL, from_planar, np_dtype, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def _op(weo, dims, kappa, U, prec):
    return weo.WilsonEO(dims, kappa, to_device(U, "f64"), prec=prec, linkfmt=18)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 2, 8)])
def test_link_grad_matches_oracle(weo, oracle_lib, prec, dims):
    import torch

    U = gen.gauge_field(dims, "haar", seed=40)
    phi = gen.gaussian_spinor(dims, seed=41)[0]
    g = gen.gaussian_spinor(dims, seed=42)[0]
    op = _op(weo, dims, 0.13, U, prec)
    G = op.link_grad(to_device(to_planar(g), prec), to_device(to_planar(phi), prec))
    torch.cuda.synchronize()
    want = oracle_lib.link_grad(U, 0.13, g, phi, dims)
    assert rel_l2(G.cpu().numpy(), want) <= TOL[prec]
    op.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_force_matches_oracle(weo, oracle_lib, prec):
    """16^3 x 32, kappa = 0.13, exp(i 0.3 H) links, Gaussian phi."""
    dims = (16, 16, 16, 32)
    U = gen.gauge_field(dims, "smooth", seed=43, eps=0.3)
    phi = gen.gaussian_spinor(dims, seed=44)[0]
    op = _op(weo, dims, 0.13, U, prec)
    F, d = op.force(to_device(to_planar(phi), prec), want_dphi=True)
    F_want, d_want = oracle_lib.force(U, 0.13, phi, dims)
    assert rel_l2(F.cpu().numpy(), F_want) <= TOL[prec]
    assert rel_l2(from_planar(d.cpu().numpy()), d_want) <= TOL[prec]
    Fn = F.cpu().numpy()
    assert np.max(np.abs(Fn + np.conj(np.swapaxes(Fn, 2, 3)))) < 1e-5
    assert np.max(np.abs(np.trace(Fn, axis1=2, axis2=3))) < 1e-5
    op.close()


def test_force_finite_differences_on_gpu(weo):
    """dS/d eps along U_mu(x) -> exp(eps X) U_mu(x) against Re tr(X^dag F): 64
    random (link, X) pairs, FP64, step 1e-6, relative error <= 1e-6."""
    import torch

    dims = (16, 16, 16, 32)
    kappa = 0.13
    U = gen.gauge_field(dims, "smooth", seed=45, eps=0.3)
    phi = gen.gaussian_spinor(dims, seed=46)[0]
    Ud = to_device(U, "f64")
    x = to_device(to_planar(phi), "f64")
    op = weo.WilsonEO(dims, kappa, Ud, prec="f64")
    F, _ = op.force(x)
    Fn = F.cpu().numpy()
    r = gen.rng(47)
    V = int(np.prod(dims))
    h = 1e-6
    worst = 0.0
    for _ in range(64):
        mu, site = int(r.integers(4)), int(r.integers(V))
        a = gen.complex_gaussian(r, (3, 3))
        X = 0.5 * (a - a.conj().T)
        X -= np.trace(X) / 3 * np.eye(3)
        chis = []
        for sgn in (+1, -1):
            Up = Ud.clone()
            Up[mu, site] = torch.from_numpy(scipy.linalg.expm(sgn * h * X) @ U[mu, site]).cuda()
            op.set_gauge(Up)
            chis.append(op.apply(x))
        dS = torch.sum(chis[0].abs() ** 2 - chis[1].abs() ** 2).item()
        fd = dS / (2 * h)
        want = np.trace(X.conj().T @ Fn[mu, site]).real
        worst = max(worst, abs(fd - want) / max(1.0, abs(want)))
    assert worst <= 1e-6
    op.close()


def test_autograd_gradcheck_2x2x2x2(weo):
    import torch

    from paper_2303_08609_gb300.autograd import meo

    dims = (2, 2, 2, 2)
    U = torch.from_numpy(gen.gauge_field(dims, "haar", seed=48)).cuda().requires_grad_(True)
    phi = torch.from_numpy(to_planar(gen.gaussian_spinor(dims, seed=49)[0])).cuda()
    phi.requires_grad_(True)
    op = weo.WilsonEO(dims, 0.13, U.detach(), prec="f64")
    # gradcheck perturbs U through .data, which the version counter does not see
    assert torch.autograd.gradcheck(lambda p, u: meo(p, u, op, refresh=True), (phi, U),
                                    eps=1e-6, atol=1e-8, rtol=1e-6)
    op.close()


def test_autograd_action_gradients_are_the_force(weo):
    """For S = |M_eo phi|^2: dS/dphi = 2 M^dag M phi and TA(dS/dU U^dag) = force."""
    import torch

    from paper_2303_08609_gb300.autograd import pseudofermion_action

    dims = (8, 8, 4, 8)
    U = torch.from_numpy(gen.gauge_field(dims, "smooth", seed=50, eps=0.3)).cuda()
    U.requires_grad_(True)
    phi = torch.from_numpy(to_planar(gen.gaussian_spinor(dims, seed=51)[0])).cuda()
    phi.requires_grad_(True)
    op = weo.WilsonEO(dims, 0.13, U.detach(), prec="f64")
    S = pseudofermion_action(phi, U, op)
    S.backward()
    F, dphi = op.force(phi.detach(), want_dphi=True)
    assert torch.allclose(phi.grad, dphi, rtol=1e-12, atol=1e-12)
    W = U.grad @ U.detach().conj().transpose(-1, -2)
    TA = 0.5 * (W - W.conj().transpose(-1, -2))
    TA = TA - torch.diagonal(TA, dim1=-2, dim2=-1).sum(-1)[..., None, None] / 3 * torch.eye(
        3, dtype=TA.dtype, device=TA.device)
    assert torch.allclose(TA, F, rtol=1e-10, atol=1e-12)
    op.close()


def test_force_rejects_16bit_handles(weo):
    import torch

    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=52)
    op = weo.WilsonEO(dims, 0.1, to_device(U), prec="f16")
    phi = torch.zeros((4, 3, 128), dtype=torch.complex64, device="cuda")
    with pytest.raises(weo.WilsonEOError) as e:
        op.force(phi)
    assert e.value.status == -3
    op.close()
