"""Pins for the oracle's analytic gradient (Sec. 2.4: derivative of Eq. 2-4 with
the voxel lookup held fixed) and for its back-projector (the transpose of V -> E)."""
import numpy as np

import oracle

RNG = np.random.default_rng(21)


def _rand_vol(rng, n, sp, zero_frac=0.2):
    data = rng.uniform(0.1, 1.0, (n[2], n[1], n[0])).astype(np.float32)
    data[rng.uniform(size=data.shape) < zero_frac] = 0.0
    return oracle.Volume(data, sp)


def _ray(rng, ext, inside=False):
    def pt(inside_pt):
        if inside_pt:
            return rng.uniform(-0.45, 0.45, 3) * ext
        v = rng.normal(size=3)
        return v / np.linalg.norm(v) * np.linalg.norm(ext) * rng.uniform(0.7, 1.5)
    return pt(inside and rng.uniform() < 0.5), pt(False)


def _fd(f, x, h):
    g = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g[a] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_gradient_vs_central_fd():
    rng = np.random.default_rng(22)
    n = np.array([7, 6, 5])
    sp = np.array([0.9, 1.1, 1.7])
    V = _rand_vol(rng, n, sp)
    checked = 0
    for _ in range(100):
        s, p = _ray(rng, n * sp, inside=True)
        E, gs, gp = oracle.siddon_ray(V, s, p, grad=True)
        if E == 0.0:
            continue
        h = 1e-6
        fs = _fd(lambda x: oracle.siddon_ray(V, x, p), s, h)
        fp = _fd(lambda x: oracle.siddon_ray(V, s, x), p, h)
        scale = max(np.abs(gs).max(), np.abs(gp).max(), 1e-3)
        assert np.abs(fs - gs).max() < 1e-5 * scale, (s, p, fs, gs)
        assert np.abs(fp - gp).max() < 1e-5 * scale, (s, p, fp, gp)
        checked += 1
    assert checked > 20


def test_uniform_box_gradient_vs_brute_force_fd():
    # E = c * chord; differentiate the per-voxel brute force (independent code) numerically
    rng = np.random.default_rng(23)
    n = np.array([3, 4, 2])
    sp = np.array([1.5, 1.0, 2.0])
    V = oracle.Volume(np.full((n[2], n[1], n[0]), 0.8, np.float32), sp)
    for _ in range(20):
        s, p = _ray(rng, n * sp, inside=True)
        E, gs, gp = oracle.siddon_ray(V, s, p, grad=True)
        if E == 0.0:
            continue
        fs = _fd(lambda x: oracle.brute_ray(V, x, p), s, 1e-6)
        fp = _fd(lambda x: oracle.brute_ray(V, s, x), p, 1e-6)
        np.testing.assert_allclose(gs, fs, atol=1e-6)
        np.testing.assert_allclose(gp, fp, atol=1e-6)


def test_directional_invariants():
    # extending a segment whose end lies outside the volume changes nothing: d.dE/dp = 0;
    # with the end inside, d.dE/dp = |d| V(p) and d.dE/ds = -|d| V(s).
    rng = np.random.default_rng(24)
    n = np.array([6, 6, 6])
    sp = np.array([1.0, 1.0, 1.0])
    V = _rand_vol(rng, n, sp, zero_frac=0.0)
    b = -0.5 * n * sp

    def value_at(x):
        idx = np.floor((x - b) / sp).astype(int)
        if np.any(idx < 0) or np.any(idx >= n):
            return 0.0
        return float(V.data[idx[2], idx[1], idx[0]])

    for _ in range(30):
        s = rng.normal(size=3)
        s = s / np.linalg.norm(s) * 20
        p = rng.uniform(-2.9, 2.9, 3)  # inside
        E, gs, gp = oracle.siddon_ray(V, s, p, grad=True)
        d = p - s
        L = np.linalg.norm(d)
        assert abs(np.dot(d, gs)) < 1e-9 * L
        assert abs(np.dot(d, gp) - L * value_at(p)) < 1e-9 * L
        E2, gs2, gp2 = oracle.siddon_ray(V, p, s, grad=True)  # source inside now
        assert abs(np.dot(s - p, gs2) + L * value_at(p)) < 1e-9 * L


def test_pose_jacobian_chain_rule():
    # dE/d eta from the oracle's render vs central differences of E(s(eta), p(eta)) in FP64
    rng = np.random.default_rng(25)
    n = np.array([12, 10, 8])
    sp = np.array([1.0, 1.2, 1.5])
    V = _rand_vol(rng, n, sp)
    det = (60.0, 5, 6, 1.3, 1.1)
    poses = np.array([[0.1, -0.2, 0.3, 0.5, -0.7, 0.2], [-0.4, 0.25, -0.1, -1.0, 0.3, 0.6]], np.float32)
    E, J = oracle.render(V, det, poses, jacobian=True)
    sdr, H, W, dh, dw = det
    for b in range(poses.shape[0]):
        for (h, w) in [(0, 0), (2, 3), (4, 5), (1, 2)]:
            base = poses[b].astype(np.float64)
            s0, p0 = oracle.ray_endpoints(base, sdr, H, W, dh, dw, h, w)
            assert abs(oracle.siddon_ray(V, s0, p0) - E[b, h, w]) < 1e-12
            for k in range(6):
                hstep = 1e-7 if k < 3 else 1e-6
                def f(x):
                    e = base.copy()
                    e[k] = x
                    s, p = oracle.ray_endpoints(e, sdr, H, W, dh, dw, h, w)
                    return oracle.siddon_ray(V, s, p)
                fd = (f(base[k] + hstep) - f(base[k] - hstep)) / (2 * hstep)
                assert abs(fd - J[b, h, w, k]) < 2e-5 * max(1.0, np.abs(J[b, h, w]).max()), (b, h, w, k, fd, J[b, h, w, k])


def test_pose_grad_is_weighted_jacobian_sum():
    rng = np.random.default_rng(26)
    V = _rand_vol(rng, np.array([8, 8, 8]), np.array([1.0, 1.0, 1.0]))
    det = (40.0, 4, 5, 1.5, 1.5)
    poses = np.array([[0.2, 0.1, -0.3, 0.4, 0.0, -0.5]], np.float32)
    g = rng.uniform(-1, 1, (1, 4, 5))
    _, J = oracle.render(V, det, poses, jacobian=True)
    np.testing.assert_allclose(oracle.pose_grad(V, det, poses, g), np.einsum("bhw,bhwk->bk", g, J), rtol=1e-12,
                               atol=1e-12)


def test_backprojection_is_adjoint():
    # <g, A V> = <A^T g, V> for the linear map A: V -> E
    rng = np.random.default_rng(27)
    n = (9, 8, 7)
    sp = (1.0, 0.8, 1.3)
    data = rng.uniform(0, 1, n[::-1]).astype(np.float32)
    V = oracle.Volume(data, sp)
    det = (50.0, 6, 7, 1.4, 1.2)
    poses = np.array([[0.3, -0.2, 0.1, 0.5, 0.2, -0.3], [1.2, 0.4, -0.6, -0.4, 0.1, 0.7]], np.float32)
    g = rng.uniform(-1, 1, (2, 6, 7))
    E = oracle.render(V, det, poses)
    BT = oracle.backproject(n[::-1], sp, det, poses, g)
    lhs = np.sum(g * E)
    rhs = np.sum(BT * data.astype(np.float64))
    assert abs(lhs - rhs) < 1e-10 * max(1.0, abs(lhs))


def test_voxel_adjoint_by_definition_matches_the_siddon_backprojection():
    # The slab-clip definition of A^T g at every voxel against the Siddon
    # back-projection (sorted crossings, midpoint voxels): two independent
    # routes to the same transpose.  Identity-like poses put rays exactly on
    # voxel planes (d_a = 0, the half-open rule), a shifted pose sends some rays
    # past the volume, and SDR 6 puts the source and detector inside the box.
    rng = np.random.default_rng(28)
    n = (7, 6, 5)
    sp = (1.1, 0.9, 1.3)
    shape = n[::-1]
    cases = [
        ((50.0, 6, 7, 1.4, 1.2), np.array([[0.3, -0.2, 0.1, 0.5, 0.2, -0.3], [1.2, 0.4, -0.6, -0.4, 0.1, 0.7]])),
        ((40.0, 5, 7, 1.0, 1.0), np.array([[0.0, 0.0, 0.0, 0.0, 0.0, 0.0], [np.pi / 2, 0.0, 0.0, 0.0, 0.0, 0.0]])),
        ((30.0, 6, 4, 1.5, 1.5), np.array([[0.1, 0.2, 0.0, 0.0, 0.0, 3.2]])),
        ((6.0, 4, 5, 0.8, 0.7), np.array([[0.4, -0.3, 0.2, 0.3, -0.2, 0.1]])),
    ]
    vox = np.arange(int(np.prod(n)))
    for det, poses in cases:
        poses = poses.astype(np.float32)
        g = rng.uniform(-1, 1, (poses.shape[0], det[1], det[2]))
        BT = oracle.backproject(shape, sp, det, poses, g).reshape(-1)
        A, A_abs = oracle.voxel_adjoint(shape, sp, det, poses, g, vox)
        assert np.abs(A_abs).max() > 0
        np.testing.assert_allclose(A, BT, rtol=0, atol=1e-12 * A_abs.max())
        assert np.all(np.abs(A) <= A_abs * (1 + 1e-12))
