"""Batching: several right-hand sides per launch, several lattices per launch,
the autotuner, and CUDA-graph capture of M_eo.

* multi-RHS: the 12 spin-colour point sources at a random even site plus 4
  Gaussian vectors, with 1, 2 and 4 right-hand sides sharing each link load;
* one persistent cooperative launch over lattices of different extents, kappa
  and independent Haar links (16^4, 24^3 x 48, 32^3 x 64 sampled; and small
  ragged lattices checked in full), each against the oracle;
* the autotuner picks a valid configuration, caches it, and never changes the
  result bits; an apply captured in a CUDA graph replays to the same bits.
"""

import numpy as np
import pytest

import gen
from gpu_util import TOL, from_planar, np_dtype, rel_l2, to_device, to_planar

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def weo():
    import paper_2303_08609_gb300 as weo

    weo.library()
    return weo


def test_multi_rhs_blocks_point_sources(weo, oracle_lib):
    import torch

    dims = (8, 8, 8, 16)
    vh = int(np.prod(dims)) // 2
    U = gen.gauge_field(dims, "haar", seed=80)
    site = int(gen.rng(81).integers(vh))
    src = np.concatenate([gen.point_sources(dims, site), gen.gaussian_spinor(dims, nrhs=4, seed=82)])
    want = oracle_lib.meo(U, 0.13, src, dims)
    op = weo.WilsonEO(dims, 0.13, to_device(U), prec="f32")
    x = to_device(to_planar(src), "f32")
    outs = {}
    for r, lanes in ((1, 1), (2, 1), (4, 1), (1, 2), (1, 4), (1, 8)):
        weo.wilson_eo_set_launch(op.handle, 128, r)
        weo.wilson_eo_set_rhs_lanes(op.handle, lanes)
        y = op.apply(x)
        for k in range(16):
            assert rel_l2(from_planar(y[k].cpu().numpy()), want[k]) <= TOL["f32"]
        outs[(r, lanes)] = y
    # right-hand sides per thread or per lane group: the same arithmetic per site
    for key, y in outs.items():
        assert torch.equal(outs[(1, 1)], y), key
    op.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_small_lattices_full_check(weo, oracle_lib, prec):
    import torch

    specs = [((4, 4, 4, 4), 0.12, 1), ((8, 4, 6, 2), 0.125, 2), ((2, 6, 4, 8), 0.135, 3),
             ((8, 8, 8, 8), 0.13, 4)]
    ops, xs, ys, wants = [], [], [], []
    for dims, kappa, seed in specs:
        U = gen.gauge_field(dims, "haar", seed=seed)
        psi = gen.gaussian_spinor(dims, seed=seed + 10)[0]
        ops.append(weo.WilsonEO(dims, kappa, to_device(U), prec=prec))
        xs.append(to_device(to_planar(psi), prec))
        ys.append(torch.empty_like(xs[-1]))
        wants.append((U, kappa, psi, dims))
    for dag in (False, True):
        weo.wilson_eo_apply_batch([o.handle for o in ops], ys, xs, dag=dag)
        torch.cuda.synchronize()
        for (U, kappa, psi, dims), y, op, x in zip(wants, ys, ops, xs):
            f = oracle_lib.meo_dag if dag else oracle_lib.meo
            assert rel_l2(from_planar(y.cpu().numpy()), f(U, kappa, psi, dims)) <= TOL[prec]
            # the batch equals the single-lattice call bit for bit
            assert torch.equal(y, op.apply(x, dag=dag))
    for o in ops:
        o.close()


def test_batch_mixed_sizes_16_24_32(weo, oracle_lib):
    """16^4, 24^3 x 48, 32^3 x 64 with independent Haar links (seeds 1, 2, 3) and
    kappa drawn in [0.12, 0.135], FP32, one launch; 200 sampled sites per lattice."""
    import torch

    r = gen.rng(5)
    specs = [((16, 16, 16, 16), 1), ((24, 24, 24, 48), 2), ((32, 32, 32, 64), 3)]
    ops, xs, ys, data = [], [], [], []
    for dims, seed in specs:
        kappa = float(r.uniform(0.12, 0.135))
        U = gen.gauge_field(dims, "haar", seed=seed)
        psi = gen.gaussian_spinor(dims, seed=seed + 20)[0]
        ops.append(weo.WilsonEO(dims, kappa, to_device(U), prec="f32"))
        xs.append(to_device(to_planar(psi), "f32"))
        ys.append(torch.empty_like(xs[-1]))
        data.append((U, kappa, psi, dims))
    weo.wilson_eo_apply_batch([o.handle for o in ops], ys, xs)
    torch.cuda.synchronize()
    for (U, kappa, psi, dims), y in zip(data, ys):
        vh = int(np.prod(dims)) // 2
        sites = np.sort(gen.rng(6).choice(vh, 200, replace=False))
        got = from_planar(y[:, :, torch.from_numpy(sites).cuda()].cpu().numpy())
        assert rel_l2(got, oracle_lib.meo_sites(U, kappa, psi, dims, sites)) <= TOL["f32"]
    for o in ops:
        o.close()


def test_batch_rejects_mixed_precision_and_duplicates(weo):
    import torch

    dims = (4, 4, 4, 4)
    U = to_device(gen.gauge_field(dims, "haar", seed=7))
    a = weo.WilsonEO(dims, 0.1, U, prec="f32")
    b = weo.WilsonEO(dims, 0.1, U, prec="f64")
    x32 = torch.zeros((4, 3, 128), dtype=torch.complex64, device="cuda")
    x64 = torch.zeros((4, 3, 128), dtype=torch.complex128, device="cuda")
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_batch([a.handle, b.handle], [torch.empty_like(x32), torch.empty_like(x64)],
                                  [x32, x64])
    assert e.value.status == -3
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_batch([a.handle, a.handle], [torch.empty_like(x32)] * 2, [x32, x32])
    assert e.value.status == -1
    a.close()
    b.close()


def test_autotuner_caches_and_keeps_results(weo):
    import time

    import torch

    dims = (16, 16, 16, 16)
    U = to_device(gen.gauge_field(dims, "smooth", seed=8, eps=0.4))
    x = to_device(to_planar(gen.gaussian_spinor(dims, nrhs=4, seed=9)), "f32")
    op = weo.WilsonEO(dims, 0.13, U, prec="f32")
    y0 = op.apply(x)
    threads, rb, ms = weo.wilson_eo_tune(op.handle, nrhs=4)
    assert threads in (64, 128, 192, 256) and rb in (1, 2, 4) and ms > 0
    algo = weo.wilson_eo_get_algorithm(op.handle)
    if algo["algo"] == 0:
        assert weo.wilson_eo_get_launch(op.handle)[:2] == (threads, rb)
        assert torch.equal(op.apply(x), y0)  # same arithmetic per site
    else:
        assert algo["threads"] == threads and algo["lookahead"] in (4, 8)
        y = op.apply(x)
        weo.wilson_eo_check(op.handle)
        assert torch.equal(y, y0)  # the fused kernel runs the same per-site code
    op2 = weo.WilsonEO(dims, 0.13, U, prec="f32")
    t0 = time.perf_counter()
    assert weo.wilson_eo_tune(op2.handle, nrhs=4) == (threads, rb, ms)  # cache hit
    assert time.perf_counter() - t0 < 0.5
    op.close()
    op2.close()


def test_apply_captured_in_cuda_graph(weo):
    import torch

    dims = (8, 8, 8, 8)
    U = to_device(gen.gauge_field(dims, "haar", seed=10))
    x = to_device(to_planar(gen.gaussian_spinor(dims, seed=11)), "f32")
    op = weo.WilsonEO(dims, 0.125, U, prec="f32")
    y, z = torch.empty_like(x), torch.empty_like(x)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):  # first call outside the capture sizes the buffers
        weo.wilson_eo_apply(op.handle, y, x, 1, s)
        weo.wilson_eo_apply_dag(op.handle, z, y, 1, s)
    torch.cuda.synchronize()
    ref = z.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        weo.wilson_eo_apply(op.handle, y, x, 1, s)
        weo.wilson_eo_apply_dag(op.handle, z, y, 1, s)
    z.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(z, ref)
    op.close()


def test_batch_launch_captured_in_cuda_graph(weo, oracle_lib):
    """The cooperative mixed-lattice launch replays from a CUDA graph."""
    import torch

    specs = [((8, 8, 8, 8), 0.12, 21), ((4, 6, 4, 8), 0.13, 22)]
    ops, xs, ys, data = [], [], [], []
    for dims, kappa, seed in specs:
        U = gen.gauge_field(dims, "haar", seed=seed)
        psi = gen.gaussian_spinor(dims, seed=seed + 1)[0]
        ops.append(weo.WilsonEO(dims, kappa, to_device(U), prec="f32"))
        xs.append(to_device(to_planar(psi), "f32"))
        ys.append(torch.empty_like(xs[-1]))
        data.append((U, kappa, psi, dims))
    hs = [o.handle for o in ops]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        weo.wilson_eo_apply_batch(hs, ys, xs, False, s)  # sizes the buffers
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        weo.wilson_eo_apply_batch(hs, ys, xs, False, s)
    for y in ys:
        y.zero_()
    g.replay()
    torch.cuda.synchronize()
    for (U, kappa, psi, dims), y in zip(data, ys):
        assert rel_l2(from_planar(y.cpu().numpy()), oracle_lib.meo(U, kappa, psi, dims)) <= TOL["f32"]
    for o in ops:
        o.close()


def test_footprint_16x16x16x16_fp32(weo):
    """Sec. 4 quotes 18 MiB of FP32 links and 6 MiB per FP32 spinor at 16^4: the
    handle holds the packed 18-real FP32 links (18 MiB) next to its FP64 copy of
    the canonical field (2 x 18 MiB), and one apply adds one FP32 odd field
    (half a 6 MiB full-lattice spinor)."""
    import torch

    dims = (16, 16, 16, 16)
    op = weo.WilsonEO(dims, 0.1, to_device(gen.gauge_field(dims, "haar", seed=23)), prec="f32")
    mib = 2**20
    assert op.info()["device_bytes"] == 18 * mib + 36 * mib
    x = torch.zeros((4, 3, op.vh), dtype=torch.complex64, device="cuda")
    op.apply(x)
    assert op.info()["device_bytes"] == 18 * mib + 36 * mib + 3 * mib
    op.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_batch_multi_rhs_mixed_lattices(weo, oracle_lib, prec):
    """Lattices with 3, 1 and 4 right-hand sides in one persistent launch."""
    import torch

    specs = [((8, 8, 4, 8), 0.12, 31, 3), ((4, 6, 4, 8), 0.13, 32, 1), ((8, 8, 8, 8), 0.125, 33, 4)]
    ops, xs, ys, data = [], [], [], []
    for dims, kappa, seed, nr in specs:
        U = gen.gauge_field(dims, "haar", seed=seed)
        psi = gen.gaussian_spinor(dims, nrhs=nr, seed=seed + 1)
        ops.append(weo.WilsonEO(dims, kappa, to_device(U), prec=prec))
        xs.append(to_device(to_planar(psi), prec))
        ys.append(torch.empty_like(xs[-1]))
        data.append((U, kappa, psi, dims))
    for dag in (False, True):
        weo.wilson_eo_apply_batch_rhs([o.handle for o in ops], ys, xs, [3, 1, 4], dag=dag)
        torch.cuda.synchronize()
        for (U, kappa, psi, dims), y in zip(data, ys):
            f = oracle_lib.meo_dag if dag else oracle_lib.meo
            want = f(U, kappa, psi, dims)
            got = from_planar(y.cpu().numpy())
            for r in range(psi.shape[0]):
                assert rel_l2(got[r], want[r]) <= TOL[prec]
    for o in ops:
        o.close()


def test_batch_rhs_rejects_bad_counts(weo):
    """nrhs per lattice outside 1..1024 is refused by the library before any launch
    (called through the raw C ABI: the binding would refuse 1025 on array size)."""
    import ctypes

    import torch

    dims = (4, 4, 4, 4)
    U = to_device(gen.gauge_field(dims, "haar", seed=34))
    op = weo.WilsonEO(dims, 0.12, U, prec="f32")
    x = torch.zeros((2, 4, 3, op.vh), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    P = ctypes.c_void_p
    hs = (P * 1)(op.handle.value if isinstance(op.handle, ctypes.c_void_p) else op.handle)
    outs = (P * 1)(y.data_ptr())
    ins = (P * 1)(x.data_ptr())
    for bad in (0, 1025, -1):
        rs = (ctypes.c_int * 1)(bad)
        assert weo.library().wilson_eo_apply_batch_rhs(1, hs, outs, ins, rs, 0, None) == -1
        assert "nrhs" in weo.wilson_eo_last_error()
    op.close()
