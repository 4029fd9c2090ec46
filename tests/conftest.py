import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU on this machine")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def bench_lattice():
    """The benchmark lattice: 32^4, eps = 0.3, seed 3202."""
    from paper_1301_3460_gb300 import inputs

    L = (32, 32, 32, 32)
    return L, inputs.rough_gauge_field(L, 0.3, 3202)


@pytest.fixture(scope="session")
def bench_lattice_fixed(bench_lattice):
    """The oracle's whole fix of the benchmark lattice (alpha = 0.08, theta < 1e-15),
    shared by the full-size FP64 and mixed-precision tests."""
    from oracle import oracle as orc

    L, U = bench_lattice
    return orc.fix(L, U, alpha=0.08, tol=1e-15, max_iter=500, history=True)
