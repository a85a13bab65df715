import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libdrr")


@pytest.fixture(scope="session")
def golden():
    import json
    with open(os.path.join(ROOT, "tests", "golden", "worked_examples.json")) as f:
        return json.load(f)


@pytest.fixture(autouse=True)
def _bounds_checked_library(request):
    """With DRR_LIBRARY naming another build of the library, every GPU test ends by
    checking that no kernel reported a device error during it; with
    DRR_EXPECT_CHECKED=1 (the bounds-checked run) the build must be the checked one,
    so that a failed bounds check could not go unseen."""
    yield
    if not os.environ.get("DRR_LIBRARY") or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2208_12737_gb300 import drr
    lib = drr.load()
    if os.environ.get("DRR_EXPECT_CHECKED") == "1":
        assert lib.drr_bounds_checked() == 1
    st = lib.drr_stream_check(None)
    assert st == 0, lib.drr_last_error().decode()
