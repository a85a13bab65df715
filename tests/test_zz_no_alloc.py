"""GPU test of drr_pose_grad_noalloc, the entry point for callers that may not
allocate device memory (a fixed device-memory footprint, or a host framework
that owns every allocation): its pose gradient must match the allocating
drr_render_backward on two calls in a row.  Kept last in collection order so a
failure here cannot hide another test's result."""
import ctypes

import numpy as np
import pytest

from paper_2208_12737_gb300 import inputs
from tests._parity import GRAD_TOL, grad_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _call(drr, det, g, J, out):
    lib = drr.load()
    d = drr.detector(det)
    st = lib.drr_pose_grad_noalloc(ctypes.byref(d), g.shape[0], ctypes.c_void_p(g.data_ptr()),
                                   ctypes.c_void_p(J.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def test_noalloc_pose_grad_matches_allocating_path(drr):
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    vol = drr.Volume(inputs.ct_phantom_hu(shape, sp, seed=51), sp, hu=True)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    poses = torch.from_numpy(inputs.random_poses(3, seed=52)).cuda()
    _, J = drr.render(vol, det, poses, jacobian=True)
    for call in range(2):
        g = torch.from_numpy(inputs.upstream_grad((3, 45, 61), seed=53 + call)).cuda()
        ref = drr.render_backward(vol, det, poses, g, jac=J).cpu().numpy()
        out = torch.full((3, 6), float("nan"), device="cuda")
        assert _call(drr, det, g, J, out) == 0, drr.load().drr_last_error()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert grad_err(got, ref).max() < GRAD_TOL


def test_noalloc_rejects_batches_beyond_its_scratch(drr):
    det = inputs.Detector(300.0, 512, 512, 1.0, 1.0)  # 128 blocks per pose -> B <= 341
    B = 400
    g = torch.zeros((1,), device="cuda")
    st = _call(drr, det, g.expand(B), g, g)
    assert st == 1  # DRR_ERR_INVALID
    assert b"scratch" in drr.load().drr_last_error()
