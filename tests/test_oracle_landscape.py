"""Pins for the oracle's loss landscape (Sec. 3.2: -ZNCC between DRRs at displaced
poses and the DRR at the true pose is minimal, -1, at the true pose and grows
away from it in a neighbourhood)."""
import numpy as np

import oracle
from paper_2208_12737_gb300 import inputs


def _tiny():
    cfg = inputs.TINY
    vol = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    ov = oracle.Volume(vol, cfg["spacing"])
    return ov, cfg["detector"].as_tuple()


def test_minimum_at_the_true_pose_and_affine_invariance():
    ov, det = _tiny()
    truth = inputs.random_poses(1, seed=41)
    fixed = oracle.render(ov, det, truth)[0]
    offs = inputs.landscape_offsets(6, seed=42, rot_range_deg=(20, 20, 10), trans_range_mm=(10, 10, 10))
    poses = np.concatenate([truth, truth + offs]).astype(np.float32)
    L = oracle.loss_landscape(ov, det, fixed, poses, eps=0.0)
    assert abs(L[0] + 1.0) < 1e-12           # identical images: ZNCC = 1
    assert np.all(L[1:] > L[0])              # every displaced DRR correlates less
    assert np.all(L >= -1.0 - 1e-12) and np.all(L <= 1.0 + 1e-12)
    # the fixed image enters only through its normalised form
    L2 = oracle.loss_landscape(ov, det, 3.0 * fixed + 0.5, poses, eps=0.0)
    np.testing.assert_allclose(L2, L, atol=1e-12)


def test_locally_increasing_along_each_parameter():
    ov, det = _tiny()
    truth = inputs.random_poses(1, seed=43)
    fixed = oracle.render(ov, det, truth)[0]
    steps = np.array([np.deg2rad(2.0)] * 3 + [2.0] * 3)
    for j in range(6):
        poses = np.repeat(truth, 5, axis=0).astype(np.float64)
        poses[:, j] += np.array([-2, -1, 0, 1, 2]) * steps[j]
        L = oracle.loss_landscape(ov, det, fixed, poses.astype(np.float32), eps=0.0)
        # convex-looking neighbourhood: the minimum in the middle, rising to both sides
        assert L[2] < L[1] < L[0], (j, L)
        assert L[2] < L[3] < L[4], (j, L)


def test_offsets_follow_the_study_ranges():
    o = inputs.landscape_offsets(20000, seed=44)
    half = np.concatenate([np.deg2rad([45.0, 45.0, 22.5]), [15.0, 15.0, 15.0]])
    assert np.all(np.abs(o) <= half + 1e-6)
    np.testing.assert_allclose(np.abs(o).max(axis=0), half, rtol=2e-3)
    np.testing.assert_allclose(o.mean(axis=0), 0.0, atol=0.02 * half.max())
