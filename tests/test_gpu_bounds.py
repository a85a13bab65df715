"""The zero padding of the volume keeps every voxel gather of the walks in
bounds, and every live back-projection add lands inside the gradient volume:
the forward, Jacobian, back-projection, split-walk and serving tests run again,
in a child process, against the bounds-checked build of the library (every gather and add
checked, a failed check recorded in a device fault word that drr_stream_check
reports), which must report no failure."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_workloads_stay_in_bounds():
    from paper_2208_12737_gb300 import build
    lib = build.build(checked=True)
    env = dict(os.environ, DRR_LIBRARY=lib, DRR_EXPECT_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
                        "tests/test_gpu_render.py", "tests/test_gpu_grad.py", "tests/test_gpu_limits.py",
                        "tests/test_gpu_split.py", "tests/test_gpu_server.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert " passed" in r.stdout
