"""GPU parity of the reverse path: fused per-ray pose Jacobian, the
deterministic pose-gradient reduction (stored-Jacobian and re-trace variants)
and the volume back-projection, against the FP64 oracle.
Tolerance: pose gradient within 1e-4 of the oracle's analytic gradient, per
pose and per parameter group (rotations, translations), relative to the
group's largest component."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import odet, osp, ovol, FP32_TOL, GRAD_TOL, grad_err, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _case_small_ct():
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    hu = inputs.ct_phantom_hu(shape, sp, seed=51)
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    poses_np = inputs.random_poses(3, seed=52)
    return mu, sp, det, poses_np


def test_pose_gradient_vs_oracle(drr):
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    poses = torch.from_numpy(poses_np).cuda()
    g_np = inputs.upstream_grad((3, det.height, det.width), seed=53)
    g = torch.from_numpy(g_np).cuda()
    E, J = drr.render(vol, det, poses, jacobian=True)
    G_jac = drr.render_backward(vol, det, poses, g, jac=J).cpu().numpy()
    G_walk = drr.render_backward(vol, det, poses, g).cpu().numpy()
    ov = ovol(mu, sp)
    G_ref = oracle.pose_grad(ov, odet(det), poses_np, g_np.astype(np.float64))
    assert grad_err(G_jac, G_ref).max() < GRAD_TOL, grad_err(G_jac, G_ref)
    assert grad_err(G_walk, G_ref).max() < GRAD_TOL, grad_err(G_walk, G_ref)
    E_ref = oracle.render(ov, odet(det), poses_np)
    assert rel_err(E.cpu().numpy(), E_ref).max() < FP32_TOL


def test_per_ray_jacobian_vs_oracle(drr):
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    _, J = drr.render(vol, det, torch.from_numpy(poses_np).cuda(), jacobian=True)
    J = J.cpu().numpy()  # (B, 6, H, W)
    _, J_ref = oracle.render(ovol(mu, sp), odet(det), poses_np, jacobian=True)
    J_ref = np.moveaxis(J_ref, -1, 1)
    for grp in (slice(0, 3), slice(3, 6)):
        scale = np.abs(J_ref[:, grp]).max()
        err = np.abs(J[:, grp] - J_ref[:, grp]) / scale
        # every ray: the crossing order is exact, so no ray sits on the other side
        # of a kink from the oracle (measured worst 5e-7 of the group's largest entry)
        assert err.max() < GRAD_TOL, np.sort(err.ravel())[-10:]
        assert np.median(err) < 1e-6


def test_jacobian_through_near_coincident_crossings(drr):
    # cubic voxels seen at 45 degrees plus a few 1e-5 rad: pairs of x / y (and
    # x / y / z) crossings lie closer than the FP32 walk resolves, so most
    # chunks take the exact re-walk; the voxel between two near-coincident
    # crossings, hence both crossings' weights, must follow the exact order
    vol_np = inputs.ellipsoid_phantom((32, 32, 32), (1.0, 1.0, 1.0), seed=61)
    vol = drr.Volume(vol_np, (1.0, 1.0, 1.0))
    det = inputs.Detector(200.0, 24, 24, 1.0, 1.0)
    q = np.pi / 4
    c = np.arctan(1.0 / np.sqrt(2.0))  # with rz = 45 deg: the cube's body diagonal
    poses_np = np.array([[q + 1e-5, 0, 0, 0.13, 0.07, 0.02], [q - 3e-5, 0, 0, -0.2, 0.1, 0.3],
                         [0, q + 2e-5, 0, 0.05, -0.1, 0.2], [q + 1e-5, c + 2e-5, 0, 0.1, 0.05, -0.07]], np.float32)
    P = torch.from_numpy(poses_np).cuda()
    E, J = drr.render(vol, det, P, jacobian=True)
    ov = ovol(vol_np, (1.0, 1.0, 1.0))
    E_ref, J_ref = oracle.render(ov, odet(det), poses_np, jacobian=True)
    assert rel_err(E.cpu().numpy(), E_ref).max() < FP32_TOL
    J = J.cpu().numpy()
    J_ref = np.moveaxis(J_ref, -1, 1)
    for grp in (slice(0, 3), slice(3, 6)):
        err = np.abs(J[:, grp] - J_ref[:, grp]) / np.abs(J_ref[:, grp]).max()
        assert err.max() < GRAD_TOL, np.sort(err.ravel())[-10:]  # every ray (measured worst 2.3e-7)
    g_np = inputs.upstream_grad((4, 24, 24), seed=62)
    G_ref = oracle.pose_grad(ov, odet(det), poses_np, g_np.astype(np.float64))
    g = torch.from_numpy(g_np).cuda()
    for G in (drr.render_backward(vol, det, P, g, jac=J_t) for J_t in (torch.from_numpy(np.ascontiguousarray(J)).cuda(), None)):
        G = G.cpu().numpy()
        assert grad_err(G, G_ref).max() < GRAD_TOL, grad_err(G, G_ref)


def test_ct_full_size_pose_gradient(drr):
    # the benchmarked workload (512x512x133, 200x200, 16 poses): the pose gradient of
    # every pose, from the stored Jacobian and from the re-walk, against the oracle's
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    poses_np = inputs.random_poses(cfg["batch"], seed=cfg["pose_seed"])
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    poses = torch.from_numpy(poses_np).cuda()
    g_np = inputs.upstream_grad((cfg["batch"], det.height, det.width), seed=54)
    g = torch.from_numpy(g_np).cuda()
    E, J = drr.render(vol, det, poses, jacobian=True)
    G = drr.render_backward(vol, det, poses, g, jac=J).cpu().numpy()
    G_walk = drr.render_backward(vol, det, poses, g).cpu().numpy()
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    ov = ovol(mu, cfg["spacing"])
    G_ref = oracle.pose_grad(ov, odet(det), poses_np, g_np.astype(np.float64))
    assert G_ref.shape == (cfg["batch"], 6)
    assert grad_err(G, G_ref).max() < GRAD_TOL, grad_err(G, G_ref)
    assert grad_err(G_walk, G_ref).max() < GRAD_TOL, grad_err(G_walk, G_ref)
    # and the stored per-ray Jacobian of all 640,000 rays, element by element
    E_ref, J_ref = oracle.render(ov, odet(det), poses_np, jacobian=True)
    assert rel_err(E.cpu().numpy(), E_ref).max() < FP32_TOL
    J = J.cpu().numpy()
    J_ref = np.moveaxis(J_ref, -1, 1)
    for grp in (slice(0, 3), slice(3, 6)):
        err = np.abs(J[:, grp] - J_ref[:, grp]) / np.abs(J_ref[:, grp]).max()
        assert err.max() < GRAD_TOL, np.sort(err.ravel())[-10:]  # measured worst 2.8e-6


def test_pose_gradient_is_deterministic(drr):
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    poses = torch.from_numpy(poses_np).cuda()
    g = torch.from_numpy(inputs.upstream_grad((3, det.height, det.width), seed=55)).cuda()
    a = drr.render_backward(vol, det, poses, g).cpu().numpy()
    b = drr.render_backward(vol, det, poses, g).cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_autograd_function(drr):
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    poses = torch.from_numpy(poses_np).cuda().requires_grad_(True)
    g_np = inputs.upstream_grad((3, det.height, det.width), seed=56)
    E = drr.DRR(vol, det)(poses)
    (E * torch.from_numpy(g_np).cuda()).sum().backward()
    G_ref = oracle.pose_grad(ovol(mu, sp), odet(det), poses_np, g_np.astype(np.float64))
    assert grad_err(poses.grad.cpu().numpy(), G_ref).max() < GRAD_TOL


def test_central_fd_on_gpu_matches_oracle_fd(drr):
    # FP32 central differences of the GPU forward at h = 1e-3 rad / 1e-2 mm against the same
    # differences of the FP64 oracle.  At this step E is kinked at the voxel scale, so both
    # differ from the point derivative (the oracle pins show that FD with h = 1e-7 matches
    # it); what must agree is the GPU forward under perturbation.  The analytic gradient is
    # checked against the oracle's elsewhere.
    cfg = inputs.TINY
    vol_np = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    vol = drr.Volume(vol_np, cfg["spacing"])
    ov = ovol(vol_np, cfg["spacing"])
    poses_np = inputs.random_poses(1, seed=cfg["pose_seed"])
    g_np = inputs.upstream_grad((1, det.height, det.width), seed=57)
    p0 = poses_np.astype(np.float64)
    fd_gpu, fd_ref = np.zeros(6), np.zeros(6)
    for k in range(6):
        h = 1e-3 if k < 3 else 1e-2
        pp, pm = p0.copy(), p0.copy()
        pp[0, k] += h
        pm[0, k] -= h
        pp, pm = pp.astype(np.float32), pm.astype(np.float32)
        den = np.float64(pp[0, k]) - np.float64(pm[0, k])
        Ep = drr.render(vol, det, torch.from_numpy(pp).cuda()).cpu().numpy().astype(np.float64)
        Em = drr.render(vol, det, torch.from_numpy(pm).cuda()).cpu().numpy().astype(np.float64)
        fd_gpu[k] = np.sum(g_np * (Ep - Em)) / den
        fd_ref[k] = np.sum(g_np * (oracle.render(ov, odet(det), pp) - oracle.render(ov, odet(det), pm))) / den
    for grp in (slice(0, 3), slice(3, 6)):
        assert np.abs(fd_gpu[grp] - fd_ref[grp]).max() < 1e-3 * np.abs(fd_ref[grp]).max(), (fd_gpu, fd_ref)


def test_ct_full_size_central_fd(drr):
    # the benchmarked workload (512x512x133, 200x200, 16 poses): central differences of
    # g . E for every pose and parameter, GPU forward against the oracle's forward under the
    # same perturbations, per pose and parameter group.  Steps: 1e-3 rad, which moves the
    # volume's points by 0.1-0.5 mm at this geometry, and 0.1 mm, the same displacement
    # scale for the translations (at 1e-2 mm the difference of two FP32 DRRs is only ~100x
    # their rounding, and the translation group's FD differs by up to 3e-3 on that noise)
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    B = cfg["batch"]
    p0 = inputs.random_poses(B, seed=cfg["pose_seed"]).astype(np.float64)
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    ov = ovol(oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32), cfg["spacing"])
    g_np = inputs.upstream_grad((B, det.height, det.width), seed=59).astype(np.float64)
    fd_gpu, fd_ref = np.zeros((B, 6)), np.zeros((B, 6))
    for k in range(6):
        h = 1e-3 if k < 3 else 1e-1
        pp, pm = p0.copy(), p0.copy()
        pp[:, k] += h
        pm[:, k] -= h
        pp, pm = pp.astype(np.float32), pm.astype(np.float32)
        den = pp[:, k].astype(np.float64) - pm[:, k].astype(np.float64)
        Ep = drr.render(vol, det, torch.from_numpy(pp).cuda()).cpu().numpy().astype(np.float64)
        Em = drr.render(vol, det, torch.from_numpy(pm).cuda()).cpu().numpy().astype(np.float64)
        fd_gpu[:, k] = np.sum(g_np * (Ep - Em), axis=(1, 2)) / den
        dref = oracle.render(ov, odet(det), pp) - oracle.render(ov, odet(det), pm)
        fd_ref[:, k] = np.sum(g_np * dref, axis=(1, 2)) / den
    assert grad_err(fd_gpu, fd_ref).max() < 1e-3, grad_err(fd_gpu, fd_ref)


def test_backprojection_adjoint_identity(drr):
    # <g, A V> = <A^T g, V> between the GPU forward and the GPU back-projection
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    poses = torch.from_numpy(poses_np).cuda()
    g_np = inputs.upstream_grad((3, det.height, det.width), seed=58)
    E = drr.render(vol, det, poses).cpu().numpy().astype(np.float64)
    gv = torch.zeros(mu.shape, device="cuda", dtype=torch.float32)
    drr.render_backward(vol, det, poses, torch.from_numpy(g_np).cuda(), pose_grad=False, grad_volume=gv)
    lhs = np.sum(g_np * E)
    rhs = np.sum(gv.cpu().numpy().astype(np.float64) * mu)
    assert abs(lhs - rhs) < 1e-5 * np.sum(np.abs(g_np) * E)


def test_backprojection_vs_oracle(drr):
    rng = np.random.default_rng(59)
    shape, sp = (9, 11, 13), (1.0, 0.8, 1.3)
    det = inputs.Detector(60.0, 12, 10, 1.3, 1.4)
    poses_np = inputs.random_poses(2, seed=60)
    g_np = inputs.upstream_grad((2, 12, 10), seed=61)
    vol = drr.Volume(rng.uniform(0, 1, shape).astype(np.float32), sp)
    gv = torch.zeros(shape, device="cuda", dtype=torch.float32)
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda(), pose_grad=False,
                        grad_volume=gv)
    ref = oracle.backproject(shape, osp(sp), odet(det), poses_np, g_np.astype(np.float64))
    np.testing.assert_allclose(gv.cpu().numpy(), ref, atol=2e-5 * np.abs(ref).max())


@pytest.mark.parametrize("offset", [0, 1])
def test_backprojection_odd_volume_and_alignment(drr, offset):
    # an odd voxel count, the last voxel reached, and a gradient volume 8-byte or
    # only 4-byte aligned: nothing is added outside it
    rng = np.random.default_rng(69)
    shape, sp = (7, 9, 11), (0.9, 1.1, 1.2)
    det = inputs.Detector(50.0, 13, 11, 1.2, 1.3)
    poses_np = inputs.random_poses(2, seed=79, max_angle_deg=40)  # reaches the last voxel
    g_np = inputs.upstream_grad((2, 13, 11), seed=71)
    vol = drr.Volume(rng.uniform(0, 1, shape).astype(np.float32), sp)
    n = int(np.prod(shape))
    buf = torch.zeros(n + 1, device="cuda", dtype=torch.float32)
    gv = buf[offset:offset + n].view(shape)
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda(), pose_grad=False,
                        grad_volume=gv)
    ref = oracle.backproject(shape, osp(sp), odet(det), poses_np, g_np.astype(np.float64))
    np.testing.assert_allclose(gv.cpu().numpy(), ref, atol=2e-5 * np.abs(ref).max())
    assert float(buf[n if offset == 0 else 0]) == 0.0  # nothing added outside the volume
    assert ref.reshape(-1)[-1] != 0  # the odd last voxel is reached


def test_backprojection_with_shared_voxels_and_gaps(drr):
    # Thick slices along z, so that rays a pixel apart along h cross the same
    # voxels and the warp merges their adds; zero upstream gradients and rays
    # that miss the volume leave gaps inside the merged pixel columns; the
    # detector is ragged against the warp tiles in both directions.
    rng = np.random.default_rng(62)
    shape, sp = (6, 20, 22), (0.5, 0.5, 4.0)
    det = inputs.Detector(90.0, 19, 13, 0.9, 0.35)
    poses_np = inputs.random_poses(3, seed=63, max_angle_deg=25, max_trans_mm=2)
    poses_np[2, 3:] = (0.0, 0.0, 13.0)  # shifted along z: the top rows miss the volume
    g_np = inputs.upstream_grad((3, 19, 13), seed=64)
    g_np[rng.uniform(size=g_np.shape) < 0.25] = 0.0
    vol = drr.Volume(rng.uniform(0, 1, shape).astype(np.float32), sp)
    gv = torch.zeros(shape, device="cuda", dtype=torch.float32)
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda(), pose_grad=False,
                        grad_volume=gv)
    ref = oracle.backproject(shape, osp(sp), odet(det), poses_np, g_np.astype(np.float64))
    assert np.abs(ref).max() > 0
    np.testing.assert_allclose(gv.cpu().numpy(), ref, atol=2e-5 * np.abs(ref).max())


def test_backprojection_ct_full_size_sampled_voxels(drr):
    # The volume adjoint in the launch the bench times (512x512x133 CT, 200x200
    # detector, 16 poses, upstream gradient on every pixel), checked at sampled
    # voxels against the oracle's adjoint by definition (every ray's clipped
    # chord through the voxel), within 2e-5 of the |g|-weighted sum per voxel.
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    B = cfg["batch"]
    poses_np = inputs.random_poses(B, seed=cfg["pose_seed"])
    g_np = inputs.upstream_grad((B, det.height, det.width), seed=3)
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    gv = torch.zeros(hu.shape, device="cuda", dtype=torch.float32)
    drr.render_backward(vol, det, torch.from_numpy(poses_np).cuda(), torch.from_numpy(g_np).cuda(), pose_grad=False,
                        grad_volume=gv)
    nz, ny, nx = hu.shape
    rng = np.random.default_rng(65)
    # mostly inside the field of view around the isocentre, some anywhere, and the corners
    k = rng.integers(nz // 2 - 30, nz // 2 + 30, 160)
    j = rng.integers(ny // 2 - 110, ny // 2 + 110, 160)
    i = rng.integers(0, nx, 160)
    vox = np.concatenate([(k * ny + j) * nx + i, rng.integers(0, nz * ny * nx, 40),
                          [0, nx - 1, nz * ny * nx - 1, (nz // 2 * ny + ny // 2) * nx + nx // 2]])
    ref, ref_abs = oracle.voxel_adjoint(hu.shape, osp(cfg["spacing"]), odet(det), poses_np, g_np.astype(np.float64),
                                        vox)
    got = gv.reshape(-1)[torch.from_numpy(vox).cuda()].cpu().numpy().astype(np.float64)
    assert (ref_abs > 0).sum() > 120
    err = np.abs(got - ref)
    assert np.all(err <= 2e-5 * ref_abs + 1e-30), (err / np.maximum(ref_abs, 1e-30)).max()
    assert np.all(got[ref_abs == 0] == 0)


def test_autograd_through_volume_and_poses(drr):
    # drr_volume: a volume held as a tensor; a linear loss sum(w * E) has dL/d mu = A^T w
    # (the oracle's back-projector) and dL/d poses = sum(w * dE/d eta) (its analytic gradient)
    rng = np.random.default_rng(66)
    shape, sp = (10, 12, 14), (1.1, 0.9, 1.3)
    det = inputs.Detector(70.0, 11, 9, 1.4, 1.5)
    poses_np = inputs.random_poses(2, seed=67)
    mu_np = rng.uniform(0, 0.05, shape).astype(np.float32)
    w_np = inputs.upstream_grad((2, 11, 9), seed=68)
    w = torch.from_numpy(w_np).cuda()
    mu = torch.from_numpy(mu_np).cuda().requires_grad_(True)
    P = torch.from_numpy(poses_np).cuda().requires_grad_(True)
    E = drr.drr_volume(mu, sp, det, P)
    E_ref = oracle.render(ovol(mu_np, sp), odet(det), poses_np)
    assert rel_err(E.detach().cpu().numpy(), E_ref).max() < FP32_TOL
    (E * w).sum().backward()
    ref_mu = oracle.backproject(shape, osp(sp), odet(det), poses_np, w_np.astype(np.float64))
    np.testing.assert_allclose(mu.grad.cpu().numpy(), ref_mu, atol=2e-5 * np.abs(ref_mu).max())
    G_ref = oracle.pose_grad(ovol(mu_np, sp), odet(det), poses_np, w_np.astype(np.float64))
    assert grad_err(P.grad.cpu().numpy(), G_ref).max() < GRAD_TOL
    # the volume alone (poses without grad): the forward walk, then the back-projection
    mu2 = torch.from_numpy(mu_np).cuda().requires_grad_(True)
    (drr.drr_volume(mu2, sp, det, torch.from_numpy(poses_np).cuda()) * w).sum().backward()
    np.testing.assert_allclose(mu2.grad.cpu().numpy(), ref_mu, atol=2e-5 * np.abs(ref_mu).max())
    # the poses alone (a constant volume tensor): no back-projection
    P3 = torch.from_numpy(poses_np).cuda().requires_grad_(True)
    (drr.drr_volume(torch.from_numpy(mu_np).cuda(), sp, det, P3) * w).sum().backward()
    assert torch.equal(P3.grad, P.grad)


def test_non_finite_poses(drr):
    # a pose with a NaN or infinite parameter gives NaN for every pixel of its DRR, its
    # Jacobian and its pose gradient, zero segments, and no back-projection adds; the other
    # poses of the batch keep their bits
    mu, sp, det, poses_np = _case_small_ct()
    vol = drr.Volume(mu, sp)
    bad = poses_np.copy()
    bad[1, 0] = np.nan
    bad[2, 4] = np.inf
    poses = torch.from_numpy(bad).cuda()
    g_np = inputs.upstream_grad((3, det.height, det.width), seed=60)
    g = torch.from_numpy(g_np).cuda()
    E, J = drr.render(vol, det, poses, jacobian=True)
    F = drr.render(vol, det, poses)
    G = drr.render_backward(vol, det, poses, g, jac=J).cpu().numpy()
    G_walk = drr.render_backward(vol, det, poses, g).cpu().numpy()
    gv = torch.zeros(mu.shape, device="cuda")
    drr.render_backward(vol, det, poses, g, pose_grad=False, grad_volume=gv)
    n = drr.count_segments(vol, det, poses).cpu().numpy()
    E, J, F = E.cpu().numpy(), J.cpu().numpy(), F.cpu().numpy()
    for b in (1, 2):
        assert np.isnan(E[b]).all() and np.isnan(J[b]).all() and np.isnan(F[b]).all()
        assert np.isnan(G[b]).all() and np.isnan(G_walk[b]).all()
        assert (n[b] == 0).all()
    one = torch.from_numpy(poses_np[:1]).cuda()
    E1, J1 = drr.render(vol, det, one, jacobian=True)
    np.testing.assert_array_equal(F[0], drr.render(vol, det, one).cpu().numpy()[0])
    np.testing.assert_array_equal(G_walk[0], drr.render_backward(vol, det, one, g[:1]).cpu().numpy()[0])
    np.testing.assert_array_equal(n[0], drr.count_segments(vol, det, one).cpu().numpy()[0])
    gv1 = torch.zeros(mu.shape, device="cuda")
    drr.render_backward(vol, det, one, g[:1], pose_grad=False, grad_volume=gv1)
    gv, gv1 = gv.cpu().numpy(), gv1.cpu().numpy()
    assert np.isfinite(gv).all()
    np.testing.assert_allclose(gv, gv1, rtol=1e-5, atol=1e-6 * np.abs(gv1).max())
