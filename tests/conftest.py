import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libfovea.so")


import pytest


@pytest.fixture(autouse=True)
def _no_bounds_faults(request):
    """With the bounds-checked library (FOVEA_LIBRARY naming
    libfovea_bounds.so), a GPU test fails if any kernel it ran stored outside
    its buffer (the store is skipped and recorded in a context's fault word)."""
    yield
    if "gpu" not in request.keywords or not os.environ.get("FOVEA_LIBRARY"):
        return
    import gc
    from paper_2012_08655_gb300 import fovea
    if not fovea.BOUNDS_BUILD:
        return
    gc.collect()  # contexts the test dropped close (and report) now
    faults = fovea.take_bounds_faults()
    assert not faults, f"out-of-bounds stores recorded: {faults}"
