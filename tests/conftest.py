import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True)
def _device_index_checks(request):
    """With the bounds-checked library (built with build(checked=True)) every GPU test ends by
    reading the device-side index checks: a violation anywhere in the test fails it."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    import paper_2305_06482_gb300 as cs
    if cs._lib is not None and b"bounds-checked" in cs.lib().cs_version():
        cs.device_status()
