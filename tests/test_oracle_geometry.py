"""Pins for the oracle's derivatives of E with respect to the detector parameters
(source-to-detector distance 2 rho and the pixel spacing, which the paper notes the
generator also differentiates, Sec. 3.2): central finite differences of the forward
(Eq. 2) in FP64, and cases with a closed form."""
import numpy as np

import oracle
from paper_2208_12737_gb300 import inputs


def _fd_geometry(vol, det, poses, g, rel=1e-6):
    sdr, H, W, dh, dw = det
    out = np.zeros((len(poses), 3))
    for k, (name, val) in enumerate((("sdr", sdr), ("dh", dh), ("dw", dw))):
        h = rel * val
        dp = {"sdr": (h, 0, 0), "dh": (0, h, 0), "dw": (0, 0, h)}[name]
        plus = (sdr + dp[0], H, W, dh + dp[1], dw + dp[2])
        minus = (sdr - dp[0], H, W, dh - dp[1], dw - dp[2])
        Ep = oracle.render(vol, plus, poses)
        Em = oracle.render(vol, minus, poses)
        out[:, k] = ((Ep - Em) * g).reshape(len(poses), -1).sum(axis=1) / (2 * h)
    return out


def test_geometry_gradient_matches_central_fd():
    rng = np.random.default_rng(51)
    data = rng.uniform(0.0, 0.05, (9, 11, 10)).astype(np.float32)
    vol = oracle.Volume(data, (1.3, 0.9, 1.7))
    det = (80.0, 7, 9, 1.1, 0.9)
    poses = inputs.random_poses(3, seed=52, max_angle_deg=40, max_trans_mm=3)
    g = rng.uniform(-1, 1, (3, 7, 9))
    an = oracle.geometry_grad(vol, det, poses, g)
    fd = _fd_geometry(vol, det, poses, g)
    np.testing.assert_allclose(an, fd, rtol=1e-6, atol=1e-8 * np.abs(fd).max())


def test_central_ray_of_a_centred_uniform_box_ignores_sdr():
    # s and p both outside the box, on the central axis: the chord does not change
    # when they move along the ray, and the spacing does not move the central pixel.
    vol = oracle.Volume(np.full((6, 6, 6), 0.25, np.float32), (1.0, 1.0, 1.0))
    det = (50.0, 3, 3, 1.0, 1.0)
    E, G = oracle.render(vol, det, np.zeros((1, 6), np.float32), geometry=True)
    np.testing.assert_allclose(E[0, 1, 1], 0.25 * 6.0, rtol=1e-14)
    np.testing.assert_allclose(G[0, 1, 1], 0.0, atol=1e-14)


def test_pixel_spacing_derivative_is_zero_on_the_centre_row_and_column():
    # dp/d dh = R (0, 0, h - (H-1)/2) vanishes on the centre row; same for dw and the
    # centre column, whatever the pose and volume.
    rng = np.random.default_rng(53)
    data = rng.uniform(0.0, 0.05, (8, 8, 8)).astype(np.float32)
    vol = oracle.Volume(data, (1.0, 1.0, 1.0))
    det = (60.0, 5, 7, 1.2, 0.8)
    poses = inputs.random_poses(2, seed=54, max_angle_deg=30, max_trans_mm=2)
    _, G = oracle.render(vol, det, poses, geometry=True)
    np.testing.assert_array_equal(G[:, 2, :, 1], 0.0)   # h = (H-1)/2: no dh term
    np.testing.assert_array_equal(G[:, :, 3, 2], 0.0)   # w = (W-1)/2: no dw term
