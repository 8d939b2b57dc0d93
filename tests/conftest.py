import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def pytest_collection_modifyitems(config, items):
    # GPU tests fail loudly (rather than skip) when CUDA is missing but they were
    # selected explicitly with -m gpu; otherwise they are skipped on CPU-only hosts.
    try:
        import torch

        has_cuda = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_cuda = False
    markexpr = config.getoption("-m") or ""
    if has_cuda or markexpr.strip() == "gpu":
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def fields_32x64():
    """The benchmark workload's inputs, generated once per session:
    32^3 x 64, exp(i 0.4 H) links (seed 0), Gaussian even source (seed 0)."""
    import gen

    dims = (32, 32, 32, 64)
    U = gen.gauge_field(dims, "smooth", seed=0, eps=0.4)
    psi = gen.gaussian_spinor(dims, seed=0)[0]
    return dims, U, psi
