"""GPU solvers for M_eo^dag M_eo x = b against the FP64 oracle.

Plain FP64 CG and mixed-precision CG with reliable updates (FP32, FP16 and
BF16 inner operators). The oracle checks each returned x by recomputing the
true residual |b - M^dag M x| / |b| with its own FP64 operator, and at small
volume compares x with the oracle's own CG solution.
"""

import numpy as np
import pytest

import gen
from gpu_util import from_planar, rel_l2, to_planar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def _true_relres(oracle_lib, U, kappa, x, b, dims):
    ax = oracle_lib.meo_dag(U, kappa, oracle_lib.meo(U, kappa, x, dims), dims)
    return float(np.linalg.norm(b - ax) / np.linalg.norm(b))


def _setup(weo, dims, kappa, kind, seed, prec, fmt=18, eps=0.4):
    import torch

    U = gen.gauge_field(dims, kind, seed=seed, eps=eps)
    b = gen.gaussian_spinor(dims, seed=seed + 1)[0]
    op = weo.WilsonEO(dims, kappa, torch.from_numpy(U).cuda(), prec=prec, linkfmt=fmt)
    bd = torch.from_numpy(to_planar(b)).cuda()
    return U, b, op, bd


@pytest.mark.parametrize("prec,mixed,fmt", [("f64", False, 18), ("f64", True, 18),
                                            ("f32", True, 18), ("f32", True, 12),
                                            ("f16", True, 18), ("bf16", True, 12)])
def test_solve_matches_oracle_cg(weo, oracle_lib, prec, mixed, fmt):
    """8^4, kappa = 0.13, exp(i 0.4 H) links: true residual <= 1e-10 and agreement
    with the oracle's CG solution."""
    dims = (8, 8, 8, 8)
    U, b, op, bd = _setup(weo, dims, 0.13, "smooth", 70, prec, fmt)
    x, info = op.solve(bd, tol=1e-10, maxiter=5000, mixed=mixed)
    assert info["converged"], info
    assert info["true_relres"] <= 1e-10
    xg = from_planar(x.cpu().numpy())
    rr = _true_relres(oracle_lib, U, 0.13, xg, b, dims)
    assert rr <= 1.5e-10, rr
    xo, it_o, rr_o, ok = oracle_lib.cg(U, 0.13, b, dims, tol=1e-12, maxiter=5000)
    assert ok
    assert rel_l2(xg, xo) <= 1e-8
    if mixed:
        assert info["reliable_updates"] >= 1
    op.close()


def test_solve_16x16x16x16_mixed_vs_plain(weo, oracle_lib):
    """16^4, kappa = 0.135: FP16-storage mixed solve and plain FP64 solve both reach
    1e-10 (checked by the oracle) with comparable iteration counts."""
    import torch

    dims = (16, 16, 16, 16)
    U, b, op16, bd = _setup(weo, dims, 0.135, "smooth", 71, "f16")
    op64 = weo.WilsonEO(dims, 0.135, torch.from_numpy(U).cuda(), prec="f64")
    x16, i16 = op16.solve(bd, tol=1e-10, maxiter=20000, mixed=True)
    x64, i64 = op64.solve(bd, tol=1e-10, maxiter=20000, mixed=False)
    assert i16["converged"] and i64["converged"]
    for x in (x16, x64):
        assert _true_relres(oracle_lib, U, 0.135, from_planar(x.cpu().numpy()), b, dims) <= 1.5e-10
    assert i16["iterations"] <= 2.0 * i64["iterations"] + 64
    op16.close()
    op64.close()


def test_solve_not_converged_and_edge_cases(weo):
    import torch

    dims = (4, 4, 4, 8)
    U, b, op, bd = _setup(weo, dims, 0.13, "haar", 72, "f32")
    # maxiter reached
    x = torch.zeros_like(bd)
    st, it, rr = weo.wilson_eo_solve(op.handle, x, bd, 1e-12, 5, True)
    assert st == -5 and it == 5 and 0 < rr < 1
    # zero right-hand side: x = 0 exactly, no iterations
    z = torch.zeros_like(bd)
    x = torch.ones_like(bd)
    st, it, rr = weo.wilson_eo_solve(op.handle, x, z, 1e-10, 100, True)
    assert st == 0 and it == 0 and torch.count_nonzero(x) == 0
    # NaN in b
    bn = bd.clone()
    bn[0, 0, 3] = float("nan")
    x = torch.zeros_like(bd)
    st, it, rr = weo.wilson_eo_solve(op.handle, x, bn, 1e-10, 100, True, raise_on_error=False)
    assert st == -6
    # bad arguments
    for tol in (0.0, -1.0, 2.0):
        st, _, _ = weo.wilson_eo_solve(op.handle, x, bd, tol, 100, True, raise_on_error=False)
        assert st == -1
    # exact initial guess converges with no iterations
    xs, info = op.solve(bd, tol=1e-10, mixed=True)
    st, it, rr = weo.wilson_eo_solve(op.handle, xs.clone(), bd, 1e-9, 100, True)
    assert st == 0 and it == 0
    op.close()


def test_solve_graphs_match_eager_bitwise(weo):
    """Chunks replayed from a captured CUDA graph give bit-identical results to the
    same launches issued one by one (reductions are deterministic)."""
    import torch

    dims = (8, 8, 4, 8)
    U, b, op, bd = _setup(weo, dims, 0.12, "haar", 73, "f16")
    xg, ig = op.solve(bd, tol=1e-10, mixed=True)
    weo.wilson_eo_solver_config(op.handle, use_graphs=0)
    xe, ie = op.solve(bd, tol=1e-10, mixed=True)
    assert ig["iterations"] == ie["iterations"]
    assert torch.equal(xg, xe)
    op.close()


def test_solve_host_arrays(weo, oracle_lib):
    dims = (4, 4, 8, 8)
    U, b, op, bd = _setup(weo, dims, 0.13, "smooth", 74, "f32")
    x = np.zeros_like(to_planar(b))
    st, it, rr = weo.wilson_eo_solve(op.handle, x, to_planar(b), 1e-10, 5000, True)
    assert st == 0 and rr <= 1e-10
    assert _true_relres(oracle_lib, U, 0.13, from_planar(x), b, dims) <= 1.5e-10
    op.close()


@pytest.mark.parametrize("prec,mixed", [("f16", True), ("f32", True), ("f64", False)])
def test_solve_multi_rhs_point_sources(weo, oracle_lib, prec, mixed):
    """12 spin-colour point sources at a random even site plus 4 Gaussian vectors
    and one zero vector, solved in lockstep; each system is checked by the oracle
    and against a single-system solve."""
    import torch

    dims = (8, 8, 8, 8)
    kappa = 0.13
    vh = int(np.prod(dims)) // 2
    U = gen.gauge_field(dims, "smooth", seed=75, eps=0.4)
    site = int(gen.rng(76).integers(vh))
    b = np.concatenate([gen.point_sources(dims, site), gen.gaussian_spinor(dims, nrhs=4, seed=77),
                        np.zeros((1, vh, 4, 3), dtype=np.complex128)])
    nrhs = b.shape[0]
    op = weo.WilsonEO(dims, kappa, torch.from_numpy(U).cuda(), prec=prec)
    if prec != "f64":
        weo.wilson_eo_set_launch(op.handle, 128, 4)  # four right-hand sides per link load
    bd = torch.from_numpy(to_planar(b)).cuda()
    x, info = op.solve(bd, tol=1e-10, maxiter=5000, mixed=mixed)
    assert info["converged"], info
    assert info["rhs_iterations"][-1] == 0 and torch.count_nonzero(x[-1]) == 0
    xg = from_planar(x.cpu().numpy())
    for r in range(nrhs - 1):
        assert info["true_relres"][r] <= 1e-10
        assert _true_relres(oracle_lib, U, kappa, xg[r], b[r], dims) <= 1.5e-10
    x1, i1 = op.solve(bd[14], tol=1e-10, maxiter=5000, mixed=mixed)
    assert rel_l2(xg[14], from_planar(x1.cpu().numpy())) <= 1e-8
    op.close()


@pytest.mark.parametrize("dims,kappa,fmt", [((8, 8, 4, 8), 0.125, 18), ((8, 8, 4, 8), 0.125, 12),
                                            ((16, 16, 16, 16), 0.135, 18)])
def test_bf16_solve_restarts_directions_and_converges(weo, oracle_lib, dims, kappa, fmt):
    """BF16-storage inner operator: by default (restart mode 2) every reliable
    update restarts the search direction, and the solve reaches true residual
    1e-10 as recomputed by the oracle. With the directions kept (mode 0) the
    solver either converges -- checked by the oracle the same way -- or says
    WEO_ERR_NOT_CONVERGED; it never reports a convergence that is not there."""
    U, b, op, bd = _setup(weo, dims, kappa, "smooth", 78, "bf16", fmt)
    x, info = op.solve(bd, tol=0.99e-10, maxiter=20000, mixed=True)
    assert info["converged"], info
    assert _true_relres(oracle_lib, U, kappa, from_planar(x.cpu().numpy()), b, dims) <= 1e-10
    weo.wilson_eo_solver_restart(op.handle, 0)
    x, info = op.solve(bd, tol=0.99e-10, maxiter=20000, mixed=True)
    assert info["status"] in ("WEO_OK", "WEO_ERR_NOT_CONVERGED"), info
    if info["converged"]:
        assert _true_relres(oracle_lib, U, kappa, from_planar(x.cpu().numpy()), b, dims) <= 1e-10
    weo.wilson_eo_solver_restart(op.handle, 1)  # forced restarts: FP16-style keep not needed
    x, info = op.solve(bd, tol=0.99e-10, maxiter=20000, mixed=True)
    assert info["converged"], info
    with pytest.raises(weo.WilsonEOError):
        weo.wilson_eo_solver_restart(op.handle, 3)
    op.close()
