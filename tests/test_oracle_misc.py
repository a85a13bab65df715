"""Pins for the oracle's pose geometry (Sec. 2.4), HU mapping and 16-bit rounding."""
import numpy as np
import pytest

import oracle


def test_pose_examples(golden):
    pe = golden["pose_examples"]
    for c in pe["cases"]:
        s, p = oracle.ray_endpoints(c["pose"], pe["sdr"], pe["H"], pe["W"], pe["dh"], pe["dw"], c["h"], c["w"])
        np.testing.assert_allclose(s, c["s"], atol=1e-12)
        np.testing.assert_allclose(p, c["p"], atol=1e-12)


def test_rotation_is_proper_and_derivative_matches():
    rng = np.random.default_rng(31)
    for _ in range(20):
        eta = rng.uniform(-np.pi, np.pi, 3)
        R, dR = oracle.pose_matrix(eta)
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        for j in range(3):
            e1, e2 = eta.copy(), eta.copy()
            e1[j] += 1e-6
            e2[j] -= 1e-6
            fd = (oracle.pose_matrix(e1)[0] - oracle.pose_matrix(e2)[0]) / 2e-6
            np.testing.assert_allclose(dR[j], fd, atol=1e-9)


def test_spherical_source_reading():
    # Sec. 2.4: source at spherical (rho, theta, phi); with R = Rz Ry Rx the source direction
    # equals (cos t sin f, sin t sin f, cos f) for theta = rz, phi = ry + pi/2, and rx only rolls.
    rng = np.random.default_rng(32)
    sdr = 510.0
    for _ in range(10):
        rz, ry, rx = rng.uniform(-1.5, 1.5, 3)
        s, p = oracle.ray_endpoints([rz, ry, rx, 0, 0, 0], sdr, 3, 3, 1.0, 1.0, 1, 1)
        th, ph = rz, ry + np.pi / 2
        np.testing.assert_allclose(s, 0.5 * sdr * np.array([np.cos(th) * np.sin(ph), np.sin(th) * np.sin(ph), np.cos(ph)]),
                                   atol=1e-10)
        np.testing.assert_allclose(p, -s, atol=1e-10)  # detector centre at the antipode


def test_detector_geometry():
    rng = np.random.default_rng(33)
    sdr, H, W, dh, dw = 300.0, 7, 9, 1.7, 1.3
    for _ in range(5):
        pose = np.concatenate([rng.uniform(-1, 1, 3), rng.uniform(-20, 20, 3)])
        s, pc = oracle.ray_endpoints(pose, sdr, H, W, dh, dw, 3, 4)  # centre pixel
        assert abs(np.linalg.norm(pc - s) - sdr) < 1e-10
        _, p1 = oracle.ray_endpoints(pose, sdr, H, W, dh, dw, 3, 5)
        _, p2 = oracle.ray_endpoints(pose, sdr, H, W, dh, dw, 4, 4)
        assert abs(np.linalg.norm(p1 - pc) - dw) < 1e-10
        assert abs(np.linalg.norm(p2 - pc) - dh) < 1e-10
        axis = (pc - s) / sdr
        assert abs(np.dot(p1 - pc, axis)) < 1e-10 and abs(np.dot(p2 - pc, axis)) < 1e-10  # plane normal to ray
        # rx rolls the detector about the central ray: source unchanged
        pose2 = pose.copy()
        pose2[2] += 0.7
        s2, pc2 = oracle.ray_endpoints(pose2, sdr, H, W, dh, dw, 3, 4)
        np.testing.assert_allclose(s2, s, atol=1e-10)
        np.testing.assert_allclose(pc2, pc, atol=1e-10)


def test_hu_to_mu():
    hu = np.array([-1024, -1000, -500, 0, 1000, 2000], np.int16)
    mu = oracle.hu_to_mu(hu, 0.02)
    np.testing.assert_allclose(mu, [0.0, 0.0, 0.01, 0.02, 0.04, 0.06], atol=1e-15)


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(34)
    x = np.concatenate([rng.uniform(0, 0.1, 5000), rng.normal(0, 100, 5000),
                        np.array([0.0, 1.0, 1.00390625, 1.01171875, 3.0e-39, 65504.0])]).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), ref)


def test_round_f16_matches_numpy():
    rng = np.random.default_rng(35)
    x = np.concatenate([rng.uniform(0, 1e-4, 4000), rng.uniform(0, 70000, 4000), rng.normal(0, 3, 4000),
                        np.array([0.0, 2.0 ** -25, 3 * 2.0 ** -26, 65519.0, 65520.0, 1.0 + 2.0 ** -11,
                                  1.0 + 3 * 2.0 ** -11])]).astype(np.float32)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float32)
    np.testing.assert_array_equal(oracle.round_f16(x), ref)


def test_f16_scale_rule():
    for m in (1e-6, 0.02, 0.06, 1.0, 3.5, 1000.0):
        sc = oracle.f16_scale(m)
        assert 2.0 ** 13 <= m * sc < 2.0 ** 14
        assert np.log2(sc) == int(np.log2(sc))
    assert oracle.f16_scale(0.0) == 1.0


def test_zncc_closed_forms():
    rng = np.random.default_rng(36)
    I = rng.uniform(0, 5, (3, 17, 13))
    assert np.allclose(oracle.zncc_loss(I, I, eps=0.0), -1.0, atol=1e-14)
    assert np.allclose(oracle.zncc_loss(I, 2.5 * I + 7.0, eps=0.0), -1.0, atol=1e-14)  # affine invariance
    assert np.allclose(oracle.zncc_loss(I, -I, eps=0.0), 1.0, atol=1e-14)
    J = rng.uniform(0, 5, (3, 17, 13))
    L = oracle.zncc_loss(I, J, eps=0.0)
    assert np.all(np.abs(L) < 1.0)
    # symmetric in its arguments
    assert np.allclose(L, oracle.zncc_loss(J, I, eps=0.0), atol=1e-14)


def test_zncc_gradient():
    rng = np.random.default_rng(37)
    I = rng.uniform(0, 5, (2, 9, 11))
    F = rng.uniform(0, 5, (2, 9, 11))
    g = oracle.zncc_loss_grad(I, F, eps=1e-8)
    # invariances (exact for eps = 0): adding a constant or scaling the moving image
    # leaves the loss unchanged
    g0 = oracle.zncc_loss_grad(I, F, eps=0.0)
    assert np.allclose(g0.reshape(2, -1).sum(axis=1), 0.0, atol=1e-12)
    assert np.allclose((g0 * I).reshape(2, -1).sum(axis=1), 0.0, atol=1e-12)
    # central finite differences
    h = 1e-6
    for (b, i, j) in [(0, 0, 0), (1, 4, 7), (0, 8, 10)]:
        Ip, Im = I.copy(), I.copy()
        Ip[b, i, j] += h
        Im[b, i, j] -= h
        fd = (oracle.zncc_loss(Ip, F)[b] - oracle.zncc_loss(Im, F)[b]) / (2 * h)
        assert abs(fd - g[b, i, j]) < 1e-7
