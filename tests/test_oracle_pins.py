"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle (``oracle/``) against something other than itself:
the dense Wilson matrix written element by element from the footnote of Eq. 1,
the even-odd (Schur) identities of Eqs. 3-5, exact symmetries of Eq. 1
(adjoint, gamma_5-hermiticity, gauge covariance, sign convention), the
free-field plane-wave closed form, and central finite differences. A dropped
term, a wrong sign, a transposed link or a wrong neighbour index in the oracle
fails at least one of them.
"""

import numpy as np
import pytest
import scipy.linalg

import gen
from lattice_ref import (
    GAMMA,
    GAMMA5,
    dense_blocks,
    dense_wilson,
    gauge_transform,
    parity_sites,
    plane_wave,
    rel_l2,
    rotate_parity_spinor,
    shift_index,
    vdot,
)

pytestmark = pytest.mark.usefixtures("oracle_lib")


def g5(psi):
    """gamma_5 on a spinor array (..., 4, 3)."""
    return np.einsum("ij,...jc->...ic", GAMMA5, psi)


# ----------------------------------------------------------- gamma basis --


def test_gamma_basis_algebra(oracle_lib):
    """The oracle's table is the stated chiral basis and obeys the Clifford algebra.

    Sec. 2 (after Eq. 1): gamma_mu has one non-zero +-1/+-i per row, squares to 1,
    and (1 +- gamma_mu) is twice a projector.
    """
    one = np.eye(4)
    for mu in range(4):
        g = oracle_lib.gamma(mu)
        np.testing.assert_array_equal(g, GAMMA[mu])
        assert np.allclose(g, g.conj().T)
        assert np.allclose(g @ g, one)
        assert np.all((np.abs(g) > 0).sum(axis=1) == 1)
        for s in (+1, -1):
            P = one + s * g
            assert np.allclose(P @ P, 2 * P)
            assert np.linalg.matrix_rank(P) == 2
        for nu in range(4):
            if nu != mu:
                h = oracle_lib.gamma(nu)
                assert np.allclose(g @ h + h @ g, 0)
    g5 = oracle_lib.gamma(0) @ oracle_lib.gamma(1) @ oracle_lib.gamma(2) @ oracle_lib.gamma(3)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# ------------------------------------------------------- dense brute force --


@pytest.mark.parametrize("dims,kind", [((4, 4, 4, 4), "haar"), ((2, 2, 2, 2), "haar"),
                                       ((2, 4, 2, 6), "smooth")])
def test_dense_blocks_and_meo(oracle_lib, dims, kind):
    """M_eo and M_eo^dag against the dense D_W built from the footnote of Eq. 1.

    Eqs. 3-4 with D_ee = D_oo = 1 (stated after Eq. 5): M_eo = 1 - D_eo D_oe.
    The 2^4 case has x+mu = x-mu in every direction (both terms hit one site).
    """
    kappa = 0.13
    U = gen.gauge_field(dims, kind, seed=3)
    D = dense_wilson(U, kappa, dims)
    Dee, Deo, Doe, Doo = dense_blocks(D, dims)
    np.testing.assert_array_equal(Dee, np.eye(Dee.shape[0]))
    np.testing.assert_array_equal(Doo, np.eye(Doo.shape[0]))
    M = np.eye(Dee.shape[0]) - Deo @ Doe
    psi = gen.gaussian_spinor(dims, seed=4)[0]
    want = (M @ psi.ravel()).reshape(psi.shape)
    got = oracle_lib.meo(U, kappa, psi, dims)
    assert rel_l2(got, want) < 1e-14
    want_dag = (M.conj().T @ psi.ravel()).reshape(psi.shape)
    got_dag = oracle_lib.meo_dag(U, kappa, psi, dims)
    assert rel_l2(got_dag, want_dag) < 1e-14
    # hopping blocks: D_oe = -kappa H_oe
    hoe = oracle_lib.hop(U, psi, dims, out_parity=1)
    assert rel_l2(-kappa * hoe.ravel(), Doe @ psi.ravel()) < 1e-14


def test_schur_solve_matches_dense(oracle_lib):
    """Eqs. 3-5: solving the even system then reconstructing xi_o solves D_W xi = eta."""
    dims = (4, 4, 4, 4)
    kappa = 0.12
    U = gen.gauge_field(dims, "haar", seed=11)
    D = dense_wilson(U, kappa, dims)
    V = 256
    eta = gen.complex_gaussian(gen.rng(12), (V, 4, 3))
    e, o = parity_sites(dims, 0), parity_sites(dims, 1)
    eta_e, eta_o = eta[e], eta[o]
    # Eq. 4 right-hand side: eta_e - D_eo eta_o, D_eo = -kappa H_eo
    rhs = eta_e + kappa * oracle_lib.hop(U, eta_o, dims, out_parity=0)
    # solve M_eo xi_e = rhs through the normal equations M^dag M xi_e = M^dag rhs
    b = oracle_lib.meo_dag(U, kappa, rhs, dims)
    xi_e, iters, relres, ok = oracle_lib.cg(U, kappa, b, dims, tol=1e-13, maxiter=2000)
    assert ok and relres <= 1e-13
    # Eq. 5: xi_o = eta_o - D_oe xi_e
    xi_o = eta_o + kappa * oracle_lib.hop(U, xi_e, dims, out_parity=1)
    xi = np.empty_like(eta)
    xi[e], xi[o] = xi_e, xi_o
    assert rel_l2(D @ xi.ravel(), eta.ravel()) < 1e-11
    xi_dense = np.linalg.solve(D, eta.ravel()).reshape(eta.shape)
    assert rel_l2(xi, xi_dense) < 1e-10


# ------------------------------------------------------------ symmetries --


DIMS_RAGGED = (4, 6, 2, 8)


def test_adjoint_identity(oracle_lib):
    """<chi, M psi> = <M^dag chi, psi> (M^dag built from conjugate-transposed blocks)."""
    U = gen.gauge_field(DIMS_RAGGED, "haar", seed=5)
    psi = gen.gaussian_spinor(DIMS_RAGGED, seed=6)[0]
    chi = gen.gaussian_spinor(DIMS_RAGGED, seed=7)[0]
    kappa = 0.135
    lhs = vdot(chi, oracle_lib.meo(U, kappa, psi, DIMS_RAGGED))
    rhs = vdot(oracle_lib.meo_dag(U, kappa, chi, DIMS_RAGGED), psi)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gamma5_hermiticity(oracle_lib):
    """gamma_5 M gamma_5 = M^dag, a consequence of Eq. 1 (gamma_5 anticommutes with gamma_mu)."""
    U = gen.gauge_field(DIMS_RAGGED, "smooth", seed=8, eps=0.4)
    psi = gen.gaussian_spinor(DIMS_RAGGED, seed=9)[0]
    kappa = 0.13
    a = g5(oracle_lib.meo(U, kappa, g5(psi), DIMS_RAGGED))
    b = oracle_lib.meo_dag(U, kappa, psi, DIMS_RAGGED)
    assert rel_l2(a, b) < 1e-14


def test_sign_convention_identity(oracle_lib):
    """Eq. 1 and Fig. 2 pair the projectors oppositely: M[-gamma] = gamma_5 M[gamma] gamma_5."""
    U = gen.gauge_field(DIMS_RAGGED, "haar", seed=10)
    psi = gen.gaussian_spinor(DIMS_RAGGED, seed=11)[0]
    kappa = 0.125
    a = oracle_lib.meo_sign(U, kappa, psi, DIMS_RAGGED, -1)
    b = g5(oracle_lib.meo(U, kappa, g5(psi), DIMS_RAGGED))
    assert rel_l2(a, b) < 1e-14
    c = oracle_lib.meo_sign(U, kappa, psi, DIMS_RAGGED, +1)
    assert rel_l2(c, oracle_lib.meo(U, kappa, psi, DIMS_RAGGED)) == 0.0
    # and the two conventions really differ
    assert rel_l2(a, c) > 1e-3


def test_gauge_covariance(oracle_lib):
    """M[U^g](g psi) = g (M[U] psi) with U_mu(x) -> g(x) U_mu(x) g(x+mu)^dag."""
    dims = (4, 4, 6, 4)
    U = gen.gauge_field(dims, "haar", seed=13)
    g = gen.random_gauge_transform(dims, seed=14)
    psi = gen.gaussian_spinor(dims, seed=15)[0]
    kappa = 0.13
    Ug = gauge_transform(U, g, dims)
    lhs = oracle_lib.meo(Ug, kappa, rotate_parity_spinor(psi, g, dims, 0), dims)
    rhs = rotate_parity_spinor(oracle_lib.meo(U, kappa, psi, dims), g, dims, 0)
    assert rel_l2(lhs, rhs) < 1e-13
    # M^dag too
    lhs = oracle_lib.meo_dag(Ug, kappa, rotate_parity_spinor(psi, g, dims, 0), dims)
    rhs = rotate_parity_spinor(oracle_lib.meo_dag(U, kappa, psi, dims), g, dims, 0)
    assert rel_l2(lhs, rhs) < 1e-13


@pytest.mark.parametrize("nvec", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0),
                                  (0, 0, 0, 1), (1, 2, 1, 3), (2, 1, 3, 5)])
def test_free_field_plane_wave(oracle_lib, nvec):
    """Unit links: H e^{ipx} u = e^{ipx} K(p) u with K = a - i b.gamma,
    a = 2 sum cos p_mu, b_mu = 2 sin p_mu (Eq. 1 with U = 1), hence
    M_eo psi_e = [1 - kappa^2 (a^2 - |b|^2) + 2 i kappa^2 a b.gamma] psi_e."""
    dims = (4, 6, 4, 8)
    U = gen.gauge_field(dims, "unit")
    u = gen.complex_gaussian(gen.rng(16), (4, 3))
    p = 2 * np.pi * np.asarray(nvec) / np.asarray(dims)
    a = 2 * np.cos(p).sum()
    b = 2 * np.sin(p)
    bg = sum(b[m] * GAMMA[m] for m in range(4))
    for kappa in (0.0, 0.1, 0.125, 0.1350):
        C = (1 - kappa**2 * (a * a - b @ b)) * np.eye(4) + 2j * kappa**2 * a * bg
        psi = plane_wave(dims, nvec, u, 0)
        want = plane_wave(dims, nvec, C @ u, 0)
        got = oracle_lib.meo(U, kappa, psi, dims)
        assert np.max(np.abs(got - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))
        # odd intermediate: H_oe psi_e = K psi on the odd sites
        K = a * np.eye(4) - 1j * bg
        assert np.max(np.abs(oracle_lib.hop(U, psi, dims, 1)
                             - plane_wave(dims, nvec, K @ u, 1))) < 1e-13


def test_free_field_critical_kappa(oracle_lib):
    """p = 0 at kappa = 1/8 (free critical point, kappa = 1/(8+2m) at m = 0): M_eo psi = 0."""
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "unit")
    u = gen.complex_gaussian(gen.rng(17), (4, 3))
    psi = plane_wave(dims, (0, 0, 0, 0), u, 0)
    assert np.max(np.abs(oracle_lib.meo(U, 0.125, psi, dims))) < 1e-14
    # kappa = 0 is the identity for any field
    U = gen.gauge_field(dims, "haar", seed=1)
    psi = gen.gaussian_spinor(dims, seed=2)[0]
    np.testing.assert_array_equal(oracle_lib.meo(U, 0.0, psi, dims), psi)


def test_meo_sites_matches_full(oracle_lib):
    """The per-site evaluation used at full size equals the whole-lattice M_eo, M_eo^dag."""
    dims = (4, 6, 4, 6)
    U = gen.gauge_field(dims, "haar", seed=18)
    psi = gen.gaussian_spinor(dims, seed=19)[0]
    kappa = 0.13
    sites = np.arange(0, 288, 7)
    full = oracle_lib.meo(U, kappa, psi, dims)
    np.testing.assert_allclose(oracle_lib.meo_sites(U, kappa, psi, dims, sites), full[sites],
                               rtol=0, atol=1e-14)
    full = oracle_lib.meo_dag(U, kappa, psi, dims)
    np.testing.assert_allclose(oracle_lib.meo_sites(U, kappa, psi, dims, sites, dag=True),
                               full[sites], rtol=0, atol=1e-14)


# ------------------------------------------------------------------ solver --


def test_cg_against_dense_normal_equations(oracle_lib):
    """Oracle CG on M^dag M x = b agrees with a dense LAPACK solve (4^4)."""
    dims = (4, 4, 4, 4)
    kappa = 0.13
    U = gen.gauge_field(dims, "smooth", seed=20, eps=0.4)
    D = dense_wilson(U, kappa, dims)
    _, Deo, Doe, _ = dense_blocks(D, dims)
    M = np.eye(Deo.shape[0]) - Deo @ Doe
    b = gen.gaussian_spinor(dims, seed=21)[0]
    x, iters, relres, ok = oracle_lib.cg(U, kappa, b, dims, tol=1e-12, maxiter=5000)
    assert ok and relres <= 1e-12 and iters > 0
    x_dense = np.linalg.solve(M.conj().T @ M, b.ravel())
    assert rel_l2(x.ravel(), x_dense) < 1e-9


def test_cg_maxiter_reports_not_converged(oracle_lib):
    dims = (4, 4, 4, 4)
    U = gen.gauge_field(dims, "haar", seed=22)
    b = gen.gaussian_spinor(dims, seed=23)[0]
    x, iters, relres, ok = oracle_lib.cg(U, 0.13, b, dims, tol=1e-14, maxiter=3)
    assert not ok and iters == 3 and relres > 1e-14


# ------------------------------------------------------------- gradients --


def _su3_direction(rng):
    a = gen.complex_gaussian(rng, (3, 3))
    x = 0.5 * (a - a.conj().T)
    return x - np.trace(x) / 3 * np.eye(3)


def _action(oracle_lib, U, kappa, phi, dims):
    chi = oracle_lib.meo(U, kappa, phi, dims)
    return float(np.vdot(chi.ravel(), chi.ravel()).real)


def test_link_grad_finite_differences(oracle_lib):
    """G = dL/dRe U + i dL/dIm U for L = Re<g, M_eo phi>; M_eo is quadratic in U so
    central differences are exact up to rounding."""
    dims = (4, 4, 4, 4)
    kappa = 0.13
    U = gen.gauge_field(dims, "haar", seed=24)
    phi = gen.gaussian_spinor(dims, seed=25)[0]
    g = gen.gaussian_spinor(dims, seed=26)[0]
    G = oracle_lib.link_grad(U, kappa, g, phi, dims)
    r = gen.rng(27)
    h = 1e-4
    for _ in range(12):
        mu, x, a, b = int(r.integers(4)), int(r.integers(256)), int(r.integers(3)), int(r.integers(3))
        for unit in (1.0, 1j):
            Up, Um = U.copy(), U.copy()
            Up[mu, x, a, b] += h * unit
            Um[mu, x, a, b] -= h * unit
            lp = vdot(g, oracle_lib.meo(Up, kappa, phi, dims)).real
            lm = vdot(g, oracle_lib.meo(Um, kappa, phi, dims)).real
            fd = (lp - lm) / (2 * h)
            want = G[mu, x, a, b].real if unit == 1.0 else G[mu, x, a, b].imag
            assert abs(fd - want) <= 1e-8 * max(1.0, abs(want))


def test_force_finite_differences(oracle_lib):
    """F: dS/d eps = Re tr(X^dag F) for S = |M_eo phi|^2, U -> exp(eps X) U
    (central differences, step 1e-6, FP64, 64 random link/direction pairs)."""
    dims = (4, 4, 4, 4)
    kappa = 0.13
    U = gen.gauge_field(dims, "smooth", seed=28, eps=0.3)
    phi = gen.gaussian_spinor(dims, seed=29)[0]
    F, dphi = oracle_lib.force(U, kappa, phi, dims)
    # F is traceless anti-Hermitian
    assert np.max(np.abs(F + np.conj(np.swapaxes(F, 2, 3)))) < 1e-13
    assert np.max(np.abs(np.trace(F, axis1=2, axis2=3))) < 1e-13
    r = gen.rng(30)
    h = 1e-6
    worst = 0.0
    for _ in range(64):
        mu, x = int(r.integers(4)), int(r.integers(256))
        X = _su3_direction(r)
        Up, Um = U.copy(), U.copy()
        Up[mu, x] = scipy.linalg.expm(h * X) @ U[mu, x]
        Um[mu, x] = scipy.linalg.expm(-h * X) @ U[mu, x]
        fd = (_action(oracle_lib, Up, kappa, phi, dims)
              - _action(oracle_lib, Um, kappa, phi, dims)) / (2 * h)
        want = np.trace(X.conj().T @ F[mu, x]).real
        worst = max(worst, abs(fd - want) / max(1.0, abs(want)))
    assert worst < 1e-6
    # dS/dphi = 2 M^dag M phi, against differences in phi
    k = (int(r.integers(128)), 2, 1)
    for unit in (1.0, 1j):
        pp, pm = phi.copy(), phi.copy()
        pp[k] += h * unit
        pm[k] -= h * unit
        fd = (_action(oracle_lib, U, kappa, pp, dims) - _action(oracle_lib, U, kappa, pm, dims)) / (2 * h)
        want = dphi[k].real if unit == 1.0 else dphi[k].imag
        assert abs(fd - want) <= 1e-6 * max(1.0, abs(want))


def test_force_ward_identity(oracle_lib):
    """A gauge rotation at one even site x0, applied to U and phi, leaves S unchanged
    (gauge covariance of Eq. 1); to first order the link force and dS/dphi cancel:
    sum_mu <X, F_mu(x0)> + <-U X U^dag, F_mu(x0-mu)> + Re<dS/dphi(x0), X phi(x0)> = 0."""
    dims = (4, 4, 4, 4)
    kappa = 0.125
    U = gen.gauge_field(dims, "haar", seed=31)
    phi = gen.gaussian_spinor(dims, seed=32)[0]
    F, dphi = oracle_lib.force(U, kappa, phi, dims)
    r = gen.rng(33)
    even = parity_sites(dims, 0)
    for trial in range(4):
        i0 = int(r.integers(len(even)))
        x0 = int(even[i0])
        X = _su3_direction(r)
        total = 0.0
        for mu in range(4):
            xb = int(shift_index(dims, mu, -1)[x0])
            total += np.trace(X.conj().T @ F[mu, x0]).real
            Xp = -U[mu, xb] @ X @ U[mu, xb].conj().T
            total += np.trace(Xp.conj().T @ F[mu, xb]).real
        total += np.vdot(dphi[i0].ravel(), (phi[i0] @ X.T).ravel()).real
        scale = np.abs(F).max() + np.abs(dphi).max()
        assert abs(total) < 1e-12 * scale


# ------------------------------------------------------------ accounting --


def test_flop_and_footprint_identities():
    """Sec. 2: 1368 flop per site and B/F 1.12; Sec. 4: 18 MiB gauge / 6 MiB spinor at 16^4 FP32.

    Per hopping direction: 12 (projection) + 2*66 (two 3x3 complex mat-vecs)
    + 24 (accumulate) = 168; eight directions minus the first accumulate = 1320;
    the full D_W adds 48 (kappa scale and the unit term) = 1368. Bytes in FP32
    per site: 8 neighbour spinors (24 reals) + 8 links (18 reals) + in + out.
    """
    assert 8 * (12 + 2 * 66 + 24) - 24 == 1320
    assert 1320 + 48 == 1368
    bf = (8 * 24 + 8 * 18 + 24 + 24) * 4 / 1368
    assert abs(bf - 1.12) < 0.005
    V = 16**4
    assert 4 * V * 18 * 4 == 18 * 2**20
    assert V * 24 * 4 == 6 * 2**20
