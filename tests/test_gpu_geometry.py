"""GPU parity of the gradient with respect to the detector parameters
(source-to-detector distance and pixel spacing, Sec. 3.2) against the FP64
oracle.  Tolerance as for the pose gradient: 1e-4 per pose, relative to the
largest of the three components."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import GRAD_TOL, odet, ovol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _geo_err(G, G_ref):
    G, G_ref = np.asarray(G, np.float64), np.asarray(G_ref, np.float64)
    return np.abs(G - G_ref).max(axis=1) / np.maximum(np.abs(G_ref).max(axis=1), 1e-30)


def test_geometry_gradient_vs_oracle(drr):
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    hu = inputs.ct_phantom_hu(shape, sp, seed=61)
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    poses_np = inputs.random_poses(3, seed=62)
    g_np = inputs.upstream_grad((3, det.height, det.width), seed=63)
    vol = drr.Volume(mu, sp)
    G = drr.geometry_grad(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda()).cpu().numpy()
    G_ref = oracle.geometry_grad(ovol(mu, sp), odet(det), poses_np, g_np)
    assert _geo_err(G, G_ref).max() < GRAD_TOL, (G, G_ref)
    # deterministic: the same bits twice
    G2 = drr.geometry_grad(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda()).cpu().numpy()
    np.testing.assert_array_equal(G, G2)


def test_geometry_gradient_ct_full_size(drr):
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    poses_np = inputs.random_poses(cfg["batch"], seed=cfg["pose_seed"])[:2]
    g_np = inputs.upstream_grad((2, det.height, det.width), seed=64)
    G = drr.geometry_grad(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda()).cpu().numpy()
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    G_ref = oracle.geometry_grad(ovol(mu, cfg["spacing"]), odet(det), poses_np, g_np)
    assert _geo_err(G, G_ref).max() < GRAD_TOL, (G, G_ref)


def test_geometry_fd_on_gpu_matches_oracle_fd(drr):
    # as for the pose: FP32 central differences of the GPU forward against the same
    # differences of the FP64 oracle, at a step where E is kinked at the voxel scale
    cfg = inputs.TINY
    vol_np = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    vol = drr.Volume(vol_np, cfg["spacing"])
    ov = ovol(vol_np, cfg["spacing"])
    poses_np = inputs.random_poses(1, seed=cfg["pose_seed"])
    P = torch.from_numpy(poses_np).cuda()
    g_np = inputs.upstream_grad((1, det.height, det.width), seed=65)
    base = det.as_tuple()
    fd_gpu, fd_ref = np.zeros(3), np.zeros(3)
    for k, idx in enumerate((0, 3, 4)):  # sdr, dh, dw in the detector tuple
        h = 0.5 if idx == 0 else 2e-3
        dp, dm = list(base), list(base)
        dp[idx] += h
        dm[idx] -= h
        dp, dm = odet(tuple(dp)), odet(tuple(dm))
        den = dp[idx] - dm[idx]
        Ep = drr.render(vol, inputs.Detector(*dp), P).cpu().numpy().astype(np.float64)
        Em = drr.render(vol, inputs.Detector(*dm), P).cpu().numpy().astype(np.float64)
        fd_gpu[k] = np.sum(g_np * (Ep - Em)) / den
        fd_ref[k] = np.sum(g_np * (oracle.render(ov, dp, poses_np) - oracle.render(ov, dm, poses_np))) / den
    assert np.abs(fd_gpu - fd_ref).max() < 1e-3 * np.abs(fd_ref).max(), (fd_gpu, fd_ref)


def test_geometry_gradient_argument_errors(drr):
    vol = drr.Volume(np.ones((8, 8, 8), np.float32), (1.0, 1.0, 1.0))
    det = inputs.Detector(100.0, 8, 8, 1.0, 1.0)
    with pytest.raises(Exception):
        drr.geometry_grad(vol, det, torch.zeros((2, 6), device="cuda"), torch.zeros((2, 7, 8), device="cuda"))
