"""Maximum sizes and their limits through the C ABI: the largest pose batch, a large
detector (over half a million warp tiles), a long thin volume (rays of thousands of
segments), and the host checks that reject what the kernels' index arithmetic does
not cover."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import FP32_TOL, GRAD_TOL, grad_err, odet, osp, ovol, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def test_largest_pose_batch(drr):
    rng = np.random.default_rng(80)
    vol_np = rng.uniform(0, 0.05, (12, 10, 14)).astype(np.float32)
    sp = (1.1, 1.3, 0.9)
    vol = drr.Volume(vol_np, sp)
    det = inputs.Detector(80.0, 2, 3, 1.5, 1.5)
    B = 65535
    poses_np = inputs.random_poses(B, seed=81, max_angle_deg=40, max_trans_mm=3)
    E = drr.render(vol, det, torch.from_numpy(poses_np).cuda()).cpu().numpy()
    idx = np.array([0, 1, 4097, 32768, B - 2, B - 1])
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np[idx])
    assert rel_err(E[idx], E_ref).max() < FP32_TOL
    # gradient reduction over the largest batch
    g = torch.from_numpy(inputs.upstream_grad((B, 2, 3), seed=82)).cuda()
    G = drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), g).cpu().numpy()
    G_ref = oracle.pose_grad(ovol(vol_np, sp), odet(det), poses_np[idx], g.cpu().numpy()[idx].astype(np.float64))
    assert grad_err(G[idx], G_ref).max() < GRAD_TOL, grad_err(G[idx], G_ref)
    # back-projection of the largest batch (its own 4x8 warp tiles): a non-negative
    # upstream gradient, so the ~10^4 FP32 adds per voxel do not cancel
    g_pos = np.random.default_rng(88).uniform(0.0, 1.0, (B, 2, 3))
    gv = torch.zeros(vol_np.shape, device="cuda")
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_pos.astype(np.float32)).cuda(),
                        pose_grad=False, grad_volume=gv)
    ref = oracle.backproject(vol_np.shape, osp(sp), odet(det), poses_np, g_pos.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(gv.cpu().numpy(), ref, rtol=1e-4, atol=1e-6 * np.abs(ref).max())
    with pytest.raises(drr.DrrError):
        drr.render(vol, det, torch.zeros((65536, 6), device="cuda"))


def test_large_detector(drr):
    rng = np.random.default_rng(83)
    vol_np = rng.uniform(0, 0.05, (20, 24, 28)).astype(np.float32)
    sp = (1.0, 1.0, 1.0)
    vol = drr.Volume(vol_np, sp)
    det = inputs.Detector(200.0, 4100, 4097, 0.02, 0.02)  # 16.8 M rays, ragged tiles
    poses_np = inputs.random_poses(1, seed=84, max_angle_deg=20, max_trans_mm=2)
    E = drr.render(vol, det, torch.from_numpy(poses_np).cuda()).cpu().numpy()
    pix = np.random.default_rng(85).choice(det.height * det.width, size=3000, replace=False)
    pix = np.concatenate([pix, [0, det.width - 1, det.height * det.width - 1]])
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np, pixels=pix)
    assert rel_err(E.reshape(1, -1)[:, pix], E_ref).max() < FP32_TOL
    # back-projection over all 16.8 M rays: <g, A V> = <A^T g, V>, with g >= 0 so
    # that the ~10^5 FP32 atomic adds per voxel do not cancel
    g = torch.rand((1, det.height, det.width), device="cuda", generator=torch.Generator("cuda").manual_seed(89))
    gv = torch.zeros(vol_np.shape, device="cuda")
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), g, pose_grad=False, grad_volume=gv)
    lhs = float((g.double() * torch.from_numpy(E).cuda().double()).sum())
    rhs = float((gv.double() * torch.from_numpy(vol_np).cuda().double()).sum())
    assert abs(lhs - rhs) <= 1e-4 * lhs, (lhs, rhs)


def test_long_rays(drr):
    # 3000 voxels along x: rays of thousands of segments and many re-anchored chunks
    rng = np.random.default_rng(86)
    vol_np = rng.uniform(0, 0.01, (3, 5, 3000)).astype(np.float32)
    sp = (0.1, 0.7, 0.8)
    vol = drr.Volume(vol_np, sp)
    det = inputs.Detector(600.0, 5, 6, 0.2, 0.3)
    poses_np = np.array([[0.0, 0.0, 0.0, 0.01, -0.02, 0.03], [0.002, -0.001, 0.5, 0.0, 0.01, 0.0]], np.float32)
    P = torch.from_numpy(poses_np).cuda()
    E, J = drr.render(vol, det, P, jacobian=True)
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np)
    assert rel_err(E.cpu().numpy(), E_ref).max() < FP32_TOL
    g_np = inputs.upstream_grad((2, 5, 6), seed=87)
    g = torch.from_numpy(g_np).cuda()
    G_ref = oracle.pose_grad(ovol(vol_np, sp), odet(det), poses_np, g_np.astype(np.float64))
    for G in (drr.render_backward(vol, det, P, g, jac=J), drr.render_backward(vol, det, P, g)):
        G = G.cpu().numpy()
        assert grad_err(G, G_ref).max() < GRAD_TOL, grad_err(G, G_ref)
    n = drr.count_segments(vol, det, P).cpu().numpy()
    assert n.max() == oracle.count_segments((3, 5, 3000), osp(sp), odet(det), poses_np).max() > 3000


def test_geometry_just_inside_the_length_limit(drr):
    # longest ray / smallest voxel = 0.95 * 2^20: micrometre voxels seen from ~1 m.
    # The clipped span is ~4e-6 of alpha, so the clip's face choice and the pose
    # chain rule (lever arms of 500 mm against a 5 um volume) are at their
    # least forgiving here.
    rng = np.random.default_rng(88)
    vol_np = rng.uniform(0.0, 50.0, (4, 5, 6)).astype(np.float32)
    sp = (1e-3, 1.2e-3, 1.1e-3)
    vol = drr.Volume(vol_np, sp)
    det = inputs.Detector(999.0, 6, 7, 1.5e-3, 1.4e-3)
    # (no pose with all rays along an axis: there every ray stays inside one voxel
    # column, the gradient is zero and a relative error has no scale)
    poses_np = np.array([[0.3, -0.2, 0.1, 1e-4, -2e-4, 1e-4], [1.2, 0.4, -0.7, 0, 0, 0],
                         [-0.5, 0.9, 0.25, 2e-4, 0, -1e-4]], np.float32)
    P = torch.from_numpy(poses_np).cuda()
    E, J = drr.render(vol, det, P, jacobian=True)
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np)
    assert (E_ref > 0).mean() > 0.5
    assert rel_err(E.cpu().numpy(), E_ref).max() < FP32_TOL
    g_np = inputs.upstream_grad((3, 6, 7), seed=89)
    G = drr.render_backward(vol, det, P, torch.from_numpy(g_np).cuda(), jac=J).cpu().numpy()
    G_ref = oracle.pose_grad(ovol(vol_np, sp), odet(det), poses_np, g_np.astype(np.float64))
    assert grad_err(G, G_ref).max() < GRAD_TOL, grad_err(G, G_ref)


def test_size_limits_are_rejected(drr):
    vol = drr.Volume(np.ones((4, 4, 4), np.float32), (1.0, 1.0, 1.0))
    P = torch.zeros((1, 6), device="cuda")
    out = torch.zeros(16, device="cuda")
    # the detector is checked before anything is written, so a small buffer suffices here
    lib = drr.load()
    big = drr.detector(inputs.Detector(100.0, 32769, 32769, 0.01, 0.01))
    st = lib.drr_render(vol.handle, ctypes.byref(big), ctypes.c_void_p(P.data_ptr()), 1,
                        ctypes.c_void_p(out.data_ptr()), None, None)
    assert st != 0 and b"too many pixels" in lib.drr_last_error()
    torch.cuda.synchronize()
    assert not out.any()
    # rays too long for the walk's fixed-point and FP32 local positions
    tiny = drr.Volume(np.ones((4, 4, 4), np.float32), (1e-4, 1e-4, 1e-4))
    with pytest.raises(drr.DrrError, match="2\\^20"):
        drr.render(tiny, inputs.Detector(500.0, 4, 4, 1.0, 1.0), P)
