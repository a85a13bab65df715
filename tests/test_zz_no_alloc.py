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


def _ref_grad(g, J):
    """sum over pixels of g * J per pose and parameter, in float64 (torch on the GPU)."""
    return (g.double().unsqueeze(1) * J.double()).sum(dim=(2, 3)).cpu().numpy()


@pytest.mark.parametrize("B,H,W,shift", [
    (65535, 8, 8, 0),     # the largest batch; float4 path (H*W % 4 == 0, aligned)
    (5, 37, 53, 0),       # H*W odd: scalar path
    (3, 64, 64, 1),       # planes offset by one float: not 16-byte aligned, scalar path
    (2, 1024, 1024, 0),   # one cluster per pose over 1 M pixels
])
def test_stored_jacobian_reduction_against_float64(drr, B, H, W, shift):
    gen = torch.Generator(device="cuda").manual_seed(B * 7 + H)
    n = B * H * W
    gbuf = torch.rand(n + shift, device="cuda", generator=gen) * 2 - 1
    jbuf = torch.randn(6 * n + shift, device="cuda", generator=gen)
    g = gbuf[shift:].view(B, H, W)
    J = jbuf[shift:].view(B, 6, H, W)
    out = torch.full((B, 6), float("nan"), device="cuda")
    det = inputs.Detector(300.0, H, W, 1.0, 1.0)
    assert _call(drr, det, g, J, out) == 0, drr.load().drr_last_error()
    ref = _ref_grad(g, J)
    got = out.cpu().numpy().astype(np.float64)
    # FP32 products summed in FP32 by each thread (n terms at most), then a
    # 10-level FP32 tree over the block's 512 threads (two 5-level butterflies),
    # FP64 across blocks: the error is below (n + 11) * 2^-24 * sum |g J|
    # (recursive-summation bound)
    n_per_thread = -(-(H * W) // (8 * 512)) + 4
    scale = (g.double().abs().unsqueeze(1) * J.double().abs()).sum(dim=(2, 3)).cpu().numpy()
    assert np.all(np.abs(got - ref) <= (n_per_thread + 11) * 2.0**-24 * scale + 1e-30)
    # bitwise reproducible
    out2 = torch.empty_like(out)
    assert _call(drr, det, g, J, out2) == 0
    assert torch.equal(out, out2)
