"""Whole-lattice parity at the benchmark size: every output site of M_eo and
M_eo^dag on 32^3 x 64 (1,048,576 even sites) against the FP64 oracle.

The inputs are those the benchmark times (kappa = 0.13, exp(i 0.4 H) links,
seed 0; Gaussian even source, seed 0), in the launch configuration each path
runs there. Each case checks

* the relative L2 error over the whole output against the tolerance of its
  storage precision (1e-12 FP64 and float-float, 1e-5 FP32, 5e-3 16-bit), and
* the worst single site, |got_i - want_i| / rms_i |want_i| <= 10 x that
  tolerance, so that an error confined to a few sites (a tile edge, a halo row,
  the periodic wrap in t) cannot hide in the global norm.

The oracle evaluates the whole lattice once per module (OpenMP over the host
cores), then every path is compared with the same arrays.
"""

import os

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, rel_l2, to_device, to_planar

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

KAPPA = 0.13

# (name, handle precision, link format, path)
#   staged: two TMA-staged hop launches (the benchmark's main line)
#   plain : two one-site-per-thread hop launches
#   fused : one persistent launch over a wavefront of t-slices
#   fused_staged: the same wavefront through the TMA-staged pipeline
#   ff    : float-float arithmetic on an FP64 handle
PATHS = [
    ("f32_l18_staged", "f32", 18, "staged"),
    ("f32_l18_two_launch", "f32", 18, "plain"),
    ("f32_l12_two_launch", "f32", 12, "plain"),
    ("f32_l18_fused", "f32", 18, "fused"),
    ("f32_l18_fused_staged", "f32", 18, "fused_staged"),
    ("f32_l12_fused", "f32", 12, "fused"),
    ("f16_l18_two_launch", "f16", 18, "plain"),
    ("f16_l12_two_launch", "f16", 12, "plain"),
    ("f16_l12_fused", "f16", 12, "fused"),
    ("bf16_l18_two_launch", "bf16", 18, "plain"),
    ("bf16_l12_two_launch", "bf16", 12, "plain"),
    ("f64_l18_two_launch", "f64", 18, "plain"),
    ("f64_l12_two_launch", "f64", 12, "plain"),
    ("ff64_l18", "f64", 18, "ff"),
]


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


@pytest.fixture(scope="module")
def reference(oracle_lib, fields_32x64):
    """Oracle M_eo psi and M_eo^dag psi on the whole lattice."""
    dims, U, psi = fields_32x64
    oracle_lib.set_threads(os.cpu_count() or 1)
    return {False: oracle_lib.meo(U, KAPPA, psi, dims),
            True: oracle_lib.meo_dag(U, KAPPA, psi, dims)}


def site_error(got, want):
    """Largest per-site error, relative to the RMS norm of the sites where
    ``want`` is nonzero (all of them for a Gaussian source, the few within two
    hops for a point source); with the index of that site. Arrays are
    (..., V/2, 4, 3)."""
    n = want.shape[-3]
    d = np.linalg.norm((got - want).reshape(-1, n, 12), axis=-1).max(axis=0)
    w = np.linalg.norm(want.reshape(-1, n, 12), axis=-1).ravel()
    rms = float(np.sqrt(np.mean(w[w > 0] ** 2)))
    return float(d.max() / rms), int(d.argmax())


def check_whole(got, want, prec, what):
    tol = TOL[prec]
    err = rel_l2(got, want)
    worst, at = site_error(got, want)
    assert err <= tol, f"{what}: rel. L2 error {err:.3e} > {tol:g}"
    assert worst <= 10 * tol, f"{what}: site {at} error {worst:.3e} > {10 * tol:g}"
    return err, worst


@pytest.mark.parametrize("name,prec,fmt,path", PATHS, ids=[p[0] for p in PATHS])
def test_meo_whole_lattice(weo, fields_32x64, reference, name, prec, fmt, path):
    import torch

    dims, U, psi = fields_32x64
    op = weo.WilsonEO(dims, KAPPA, to_device(U), prec=prec, linkfmt=fmt)
    if path == "staged":
        weo.wilson_eo_set_staging(op.handle, True)
        assert weo.wilson_eo_get_staging(op.handle)["staged"]
    elif path == "fused":
        weo.wilson_eo_set_algorithm(op.handle, "fused", 4, 128)
    elif path == "fused_staged":
        weo.wilson_eo_set_algorithm(op.handle, "fused_staged", 2)
    spin = "f64" if prec == "f64" else "f32"
    x = to_device(to_planar(psi), spin)
    for dag in (False, True):
        y = op.apply_ff64(x, dag=dag) if path == "ff" else op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        torch.cuda.synchronize()
        got = from_planar(y.cpu().numpy())
        check_whole(got, reference[dag], "f64" if path == "ff" else prec,
                    f"{name} M_eo{'^dag' if dag else ''}")
        del y
    op.close()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_twelve_point_sources_whole_lattice(weo, oracle_lib, fields_32x64, prec):
    """The batched workload: 12 spin-colour point sources at one even site in one
    call, in the launch configuration the autotuner picks for 12 right-hand
    sides; every right-hand side on every site against the oracle."""
    import torch

    dims, U, _ = fields_32x64
    vh = int(np.prod(dims)) // 2
    site = int(gen.rng(3).integers(vh))
    src = gen.point_sources(dims, site)
    op = weo.WilsonEO(dims, KAPPA, to_device(U), prec=prec)
    weo.wilson_eo_tune(op.handle, nrhs=12)
    x = to_device(to_planar(src), "f32")
    oracle_lib.set_threads(os.cpu_count() or 1)
    for dag in (False, True):
        y = op.apply(x, dag=dag)
        weo.wilson_eo_check(op.handle)
        got = from_planar(y.cpu().numpy())
        f = oracle_lib.meo_dag if dag else oracle_lib.meo
        for r in range(12):
            check_whole(got[r], f(U, KAPPA, src[r], dims), prec,
                        f"point source {r} M_eo{'^dag' if dag else ''}")
    op.close()
    torch.cuda.empty_cache()
