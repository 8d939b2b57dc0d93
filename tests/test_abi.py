"""The C ABI library loads and exports every function ``include/*.h`` declares,
and argument errors come back as status codes (no GPU needed for either)."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(wilson_eo_\w+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2303_08609_gb300 as weo

    if not os.path.exists(weo.LIB_PATH):
        from paper_2303_08609_gb300 import build

        build.build()
    return weo.library()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for n in ("wilson_eo_create", "wilson_eo_apply", "wilson_eo_apply_dag", "wilson_eo_destroy",
              "wilson_eo_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_strerror_and_destroy_null(lib):
    import paper_2303_08609_gb300 as weo

    assert weo.wilson_eo_strerror(0) == "success"
    assert "dimensions" in weo.wilson_eo_strerror(-2)
    assert weo.wilson_eo_strerror(12345) == "unknown status"
    weo.wilson_eo_destroy(None)  # no-op


@pytest.mark.parametrize("dims", [(3, 4, 4, 4), (4, 4, 4, 0), (4, 1, 4, 4), (4, 4, 5, 4)])
def test_create_rejects_bad_dims_before_touching_the_device(lib, dims):
    import paper_2303_08609_gb300 as weo

    U = np.zeros((4, 1, 3, 3), dtype=np.complex128)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_create(dims, 0.1, "f32", 18, U)
    assert e.value.status == -2
    assert "even" in weo.wilson_eo_last_error()


def test_create_rejects_bad_enums_and_nulls(lib):
    import paper_2303_08609_gb300 as weo

    U = np.zeros((4, 16, 3, 3), dtype=np.complex128)
    h = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(2, 2, 2, 2)
    assert lib.wilson_eo_create(ctypes.byref(h), d, 0.1, 7, 0, U.ctypes.data, 1, None) == -1
    assert lib.wilson_eo_create(ctypes.byref(h), d, 0.1, 1, 5, U.ctypes.data, 1, None) == -1
    assert lib.wilson_eo_create(ctypes.byref(h), d, 0.1, 1, 0, None, 1, None) == -1
    assert lib.wilson_eo_create(None, d, 0.1, 1, 0, U.ctypes.data, 1, None) == -1
    assert lib.wilson_eo_apply(None, None, None, 1, None) == -1
    assert lib.wilson_eo_info(None, None, None, None, None, None, None) == -1
    assert weo.STATUS[-1] == "WEO_ERR_ARG"


def test_create_rejects_half_volume_beyond_int32(lib):
    """Site indices are 32-bit inside the kernels: V/2 >= 2^31 is refused up front."""
    import paper_2303_08609_gb300 as weo

    U = np.zeros((4, 1, 3, 3), dtype=np.complex128)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_create((2048, 2048, 1024, 2), 0.1, "f32", 18, U)
    assert e.value.status == -2 and "large" in weo.wilson_eo_last_error()


def test_noalloc_rejects_bad_arguments_before_the_device(lib):
    import paper_2303_08609_gb300 as weo

    z = np.zeros(8, dtype=np.complex64)
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_noalloc((4, 4, 3, 4), 0.1, z, z.copy(), z)
    assert e.value.status == -2
    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_apply_noalloc((64, 64, 64, 64), 0.1, z, z.copy(), z)
    assert e.value.status == -2 and "349525" in weo.wilson_eo_last_error()


def test_alu_peak_rejects_other_precisions(lib):
    import paper_2303_08609_gb300 as weo

    with pytest.raises(weo.WilsonEOError) as e:
        weo.wilson_eo_alu_peak("f16")
    assert e.value.status == -1


def test_rhs_lanes_rejects_bad_values(lib):
    assert lib.wilson_eo_set_rhs_lanes(None, 2) == -1


def test_ff_and_residual_mode_reject_null(lib):
    assert lib.wilson_eo_apply_ff64(None, None, None, 1, 0, None) == -1
    assert lib.wilson_eo_solver_residual(None, 1) == -1


def test_staging_rejects_null_and_bad_values(lib):
    assert lib.wilson_eo_set_staging(None, 1, 0, 0) == -1
    assert lib.wilson_eo_get_staging(None, None, None, None) == -1
    assert lib.wilson_eo_inject_staged_timeout(None, None, None, None) == -1


def test_noalloc_refuses_tensors_off_the_gpu_before_the_library(lib):
    """Torch tensors that are not CUDA arrays (here on the meta and CPU devices)
    are refused by the binding before any library call, as are arrays on
    different GPUs."""
    import torch

    import paper_2303_08609_gb300 as weo

    for device in ("meta", "cpu"):
        z = torch.empty(8, dtype=torch.complex64, device=device)
        with pytest.raises(ValueError, match="CUDA device arrays only"):
            weo.wilson_eo_apply_noalloc((4, 4, 4, 4), 0.1, z, z.clone(), z)
    assert weo._noalloc_device((np.zeros(2), None, 5)) is None

    class OnGpu:  # stands in for a CUDA tensor: only its device is looked at
        is_cuda = True

        def __init__(self, index):
            self.device = torch.device("cuda", index)

        def data_ptr(self):
            return 0

    assert weo._noalloc_device((OnGpu(1), OnGpu(1), None)) == 1
    with pytest.raises(ValueError, match="different devices"):
        weo.wilson_eo_apply_noalloc((4, 4, 4, 4), 0.1, OnGpu(0), OnGpu(1), OnGpu(0))


def test_spinor_layout_rejects_bad_arguments_before_the_device(lib):
    n = 8
    a = np.zeros(12 * n, dtype=np.complex64)
    b = np.zeros(12 * n, dtype=np.complex64)
    P = a.ctypes.data
    Q = b.ctypes.data
    assert lib.wilson_eo_spinor_layout(n, 1, 8, 1, None, Q, None) == -1
    assert lib.wilson_eo_spinor_layout(0, 1, 8, 1, P, Q, None) == -1
    assert lib.wilson_eo_spinor_layout(n, 0, 8, 1, P, Q, None) == -1
    assert lib.wilson_eo_spinor_layout(n, 1, 4, 1, P, Q, None) == -1
    assert lib.wilson_eo_spinor_layout(n, 1, 8, 2, P, Q, None) == -1
    assert lib.wilson_eo_spinor_layout(n, 1, 8, 1, P, P + 8, None) == -1  # overlapping
    assert lib.wilson_eo_spinor_layout(n, 1, 8, 1, P, Q, None) == -1      # host arrays


def test_tile_links_rejects_null(lib):
    assert lib.wilson_eo_set_tile_links(None, 4, 1) == -1
    assert lib.wilson_eo_get_tile_links(None, None, None) == -1


def test_l2_peak_rejects_null(lib):
    assert lib.wilson_eo_l2_peak(None, None) == -1


def test_site_blocks_rejects_null_and_bad_values(lib):
    assert lib.wilson_eo_set_site_blocks(None, 1) == -1
