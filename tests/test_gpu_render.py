"""GPU parity of the forward path (ray setup, clip, Siddon walk) against the
FP64 oracle, through the C ABI.  Tolerance: 2e-5 max per-pixel relative error
for FP32 volumes (floor 1e-3 of the image maximum), exact zeros for misses."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import odet, osp, ovol, FP32_TOL, HALF_TOL, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _render(drr, vol_np, spacing, det, poses_np, storage="f32", hu=False):
    vol = drr.Volume(vol_np, spacing, storage=storage, hu=hu)
    poses = torch.from_numpy(np.ascontiguousarray(poses_np, np.float32)).cuda()
    E = drr.render(vol, det, poses)
    drr.stream_check()
    return E.cpu().numpy()


def test_ray_setup_matches_oracle(drr):
    det = inputs.Detector(510.0, 7, 9, 1.4, 1.3)
    poses_np = inputs.random_poses(3, seed=41)
    rays = drr.ray_setup(det, torch.from_numpy(poses_np).cuda()).cpu().numpy()
    for b in range(3):
        for h in range(7):
            for w in range(9):
                s, p = oracle.ray_endpoints(poses_np[b].astype(np.float64), *odet(det), h, w)
                np.testing.assert_allclose(rays[b, h, w, :3], s, atol=4e-5)
                np.testing.assert_allclose(rays[b, h, w, 3:], p, atol=4e-5)


def test_tiny_config_all_pixels(drr):
    cfg = inputs.TINY
    vol_np = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    poses_np = np.concatenate([inputs.random_poses(1, seed=cfg["pose_seed"]), inputs.random_poses(3, seed=42)])
    E = _render(drr, vol_np, cfg["spacing"], det, poses_np)
    E_ref = oracle.render(ovol(vol_np, cfg["spacing"]), odet(det), poses_np)
    r = rel_err(E, E_ref)
    assert r.max() < FP32_TOL, r.max()
    assert np.all(E[E_ref == 0] == 0)


def test_small_ct_ragged_tiles(drr):
    # CT-like anisotropic volume, detector not a multiple of the 32x8 block tile
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    hu = inputs.ct_phantom_hu(shape, sp, seed=43)
    det = inputs.Detector(420.0, 75, 90, 1.9, 1.7)
    poses_np = inputs.random_poses(3, seed=44)
    E = _render(drr, hu, sp, det, poses_np, hu=True)
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    E_ref = oracle.render(ovol(mu, sp), odet(det), poses_np)
    r = rel_err(E, E_ref)
    assert r.max() < FP32_TOL, r.max()


def test_ct_full_size_all_pixels(drr):
    # 512x512x133 HU phantom, 200x200 detector, 16 poses, as benchmarked: every pixel of
    # every pose against the oracle (the whole 640,000-ray batch)
    cfg = inputs.CT
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    poses_np = inputs.random_poses(cfg["batch"], seed=cfg["pose_seed"])
    E = _render(drr, hu, cfg["spacing"], det, poses_np, hu=True)
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    E_ref = oracle.render(ovol(mu, cfg["spacing"]), odet(det), poses_np)
    assert E.shape == E_ref.shape == (cfg["batch"], det.height, det.width)
    r = rel_err(E, E_ref)
    assert r.max() < FP32_TOL, r.max()
    assert np.all(E[E_ref == 0] == 0)


def test_uniform_cube_closed_form(drr):
    # every ray's E is c * chord, including rays that graze edges and corners
    n, dl, c = 24, 1.5, 0.25
    vol_np = np.full((n, n, n), c, np.float32)
    det = inputs.Detector(120.0, 64, 64, 1.2, 1.2)
    poses_np = np.concatenate([inputs.random_poses(4, seed=46, max_angle_deg=60, max_trans_mm=8),
                               np.zeros((1, 6), np.float32)])
    E = _render(drr, vol_np, (dl, dl, dl), det, poses_np)
    E_ref = oracle.render(ovol(vol_np, (dl, dl, dl)), odet(det), poses_np)
    r = rel_err(E, E_ref)
    assert r.max() < FP32_TOL, r.max()


def test_source_and_detector_inside_volume(drr):
    # SDR shorter than the box: both endpoints inside for central rays (alpha clamp to [0, 1])
    rng = np.random.default_rng(47)
    vol_np = rng.uniform(0.0, 0.05, (30, 34, 38)).astype(np.float32)
    sp = (1.0, 1.0, 1.0)
    det = inputs.Detector(20.0, 16, 16, 0.9, 0.9)
    poses_np = np.concatenate([inputs.random_poses(3, seed=48, max_angle_deg=90, max_trans_mm=5),
                               np.zeros((1, 6), np.float32)])
    E = _render(drr, vol_np, sp, det, poses_np)
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np)
    assert rel_err(E, E_ref).max() < FP32_TOL


def test_axis_aligned_and_right_angle_poses(drr):
    # rays parallel to voxel planes (d_a == 0) and exact quarter turns
    rng = np.random.default_rng(49)
    vol_np = rng.uniform(0.0, 0.05, (20, 22, 24)).astype(np.float32)
    sp = (1.1, 0.9, 1.3)
    det = inputs.Detector(200.0, 9, 11, 1.0, 1.0)
    q = np.pi / 2
    poses_np = np.array([[0, 0, 0, 0, 0, 0], [q, 0, 0, 0.3, 0.1, 0], [0, q, 0, 0, 0.2, 0.4],
                         [0, 0, q, 0.25, 0, 0], [q, q, q, 0.1, 0.2, 0.3], [0, 0, 0, 0.55, 0.45, 0.35]], np.float32)
    E = _render(drr, vol_np, sp, det, poses_np)
    E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np)
    assert rel_err(E, E_ref).max() < FP32_TOL


def test_rays_missing_the_volume_are_exact_zero(drr):
    vol_np = np.full((8, 8, 8), 1.0, np.float32)
    det = inputs.Detector(100.0, 16, 16, 2.0, 2.0)
    poses_np = np.array([[0, 0, 0, 0, 60.0, 0], [0.5, 0.2, 0.1, 0, 0, -70.0]], np.float32)
    E = _render(drr, vol_np, (1.0, 1.0, 1.0), det, poses_np)
    assert np.all(E == 0)


def test_degenerate_sizes(drr):
    # 1x1x1 volume and a 1x1 detector
    vol_np = np.full((1, 1, 1), 0.7, np.float32)
    det = inputs.Detector(50.0, 1, 1, 1.0, 1.0)
    poses_np = np.array([[0.1, 0.2, 0.3, 0.1, -0.2, 0.05], [0, 0, 0, 0, 0, 0]], np.float32)
    E = _render(drr, vol_np, (2.0, 3.0, 4.0), det, poses_np)
    E_ref = oracle.render(ovol(vol_np, (2.0, 3.0, 4.0)), odet(det), poses_np)
    assert rel_err(E, E_ref).max() < FP32_TOL
    assert abs(E[1, 0, 0] - 0.7 * 2.0) < 1e-6


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_half_storage(drr, storage):
    cfg = inputs.TINY
    vol_np = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    poses_np = inputs.random_poses(2, seed=50)
    E = _render(drr, vol_np, cfg["spacing"], det, poses_np, storage=storage)
    ov = ovol(vol_np, cfg["spacing"])
    E_ref = oracle.render(ov, odet(det), poses_np)
    assert rel_err(E, E_ref).max() < HALF_TOL
    # against the oracle on the de-quantised volume the kernel error alone must meet the FP32 bound
    if storage == "bf16":
        deq = oracle.round_bf16(vol_np)
    else:
        sc = oracle.f16_scale(float(np.abs(vol_np).max()))
        deq = (oracle.round_f16(vol_np * np.float32(sc)).astype(np.float64) / sc).astype(np.float32)
    E_deq = oracle.render(ovol(deq, cfg["spacing"]), odet(det), poses_np)
    assert rel_err(E, E_deq).max() < FP32_TOL


def test_argument_errors(drr):
    vol = drr.Volume(np.ones((4, 4, 4), np.float32), (1, 1, 1))
    poses = torch.zeros((1, 6), device="cuda")
    with pytest.raises(drr.DrrError):
        drr.render(vol, (100.0, 0, 4, 1.0, 1.0), poses)
    with pytest.raises(drr.DrrError):
        drr.render(vol, (-1.0, 4, 4, 1.0, 1.0), poses)
    with pytest.raises(ValueError):
        drr.render(vol, (100.0, 4, 4, 1.0, 1.0), torch.zeros((1, 5), device="cuda"))
    with pytest.raises(drr.DrrError):
        drr.Volume(np.ones((4, 4, 4), np.float32), (1, 0, 1))


def test_segment_counts_exact(drr):
    # integer work is bit-exact: segments per ray vs the oracle's sorted-crossing count (Eq. 4)
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    det = inputs.Detector(420.0, 33, 41, 2.2, 1.9)
    poses_np = inputs.random_poses(3, seed=62)
    vol = drr.Volume(np.zeros(shape, np.float32), sp)
    got = drr.count_segments(vol, det, torch.from_numpy(poses_np).cuda()).cpu().numpy()
    ref = oracle.count_segments(shape, osp(sp), odet(det), poses_np)
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("layout", ["y", "z"])
def test_layouts_give_the_same_bits(drr, layout):
    # the storage layouts change only which voxels share a cache sector: the DRR,
    # the per-ray Jacobian, the pose gradient and the back-projection are the
    # same bits as with the x-fastest layout
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    hu = inputs.ct_phantom_hu(shape, sp, seed=43)
    det = inputs.Detector(420.0, 37, 54, 1.9, 1.7)
    poses = torch.from_numpy(inputs.random_poses(3, seed=44)).cuda()
    g = torch.from_numpy(inputs.upstream_grad((3, 37, 54), seed=45)).cuda()
    out = {}
    for lay in ("x", layout):
        vol = drr.Volume(hu, sp, hu=True, layout=lay)
        E, J = drr.render(vol, det, poses, jacobian=True)
        G = drr.render_backward(vol, det, poses, g)
        gv = torch.zeros(shape, device="cuda")
        drr.render_backward(vol, det, poses, g, pose_grad=False, grad_volume=gv)
        out[lay] = (E.cpu().numpy(), J.cpu().numpy(), G.cpu().numpy(), gv.cpu().numpy())
    for a, b in zip(out["x"], out[layout][:3]):
        np.testing.assert_array_equal(a, b)
    # back-projection: the same adds in a possibly different atomic order
    np.testing.assert_allclose(out[layout][3], out["x"][3], rtol=1e-5, atol=1e-6 * np.abs(out["x"][3]).max())
