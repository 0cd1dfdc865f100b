import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def ism():
    """The CUDA library binding; GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2104_13347_gb300 as pkg
    pkg.load()
    return pkg


@pytest.fixture(scope="session", autouse=True)
def bounds_checked_build_reports_nothing():
    """With the bounds-checked library (ISM_LIB=libism_checked.so), the
    kernels of the whole session must have recorded no out-of-range index."""
    yield
    if "checked" not in os.environ.get("ISM_LIB", ""):
        return
    import torch
    if not torch.cuda.is_available():
        return
    from paper_2104_13347_gb300 import _lib
    flags = _lib.debug_bounds()
    assert flags is not None, "ISM_LIB names a library that is not bounds-checked"
    assert flags == 0, f"kernels recorded out-of-range indices: flags {flags:#x}"
