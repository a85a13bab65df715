"""Pins for the oracle's line integral (Eq. 1-4): hand-worked examples, closed
forms, an exact per-voxel brute force, midpoint sampling and invariants."""
import numpy as np
import pytest

import oracle


def _vol(golden):
    return oracle.Volume(np.array(golden["volume_zyx"], np.float32), golden["spacing"])


def test_worked_examples(golden):
    V = _vol(golden)
    for ex in golden["examples"]:
        E = oracle.siddon_ray(V, ex["s"], ex["p"])
        if "E" in ex:
            assert abs(E - ex["E"]) <= 1e-12 * max(1.0, abs(ex["E"])), ex["name"]
        else:
            L = np.linalg.norm(ex["d"])
            assert abs(E - L * ex["F"]) <= 1e-12 * L * ex["F"], ex["name"]


def test_worked_backprojection(golden):
    # the transpose of V -> E for a single worked ray, derived by hand from the same segments
    V = np.array(golden["volume_zyx"], dtype=np.float64)
    done = 0
    for ex in golden["examples"]:
        if "backprojection_g1" not in ex:
            continue
        bt = oracle.backproject_ray(V.shape, golden["spacing"], ex["s"], ex["p"], 1.0)
        want = np.array(ex["backprojection_g1"])
        np.testing.assert_allclose(bt, want, rtol=0, atol=1e-12 * np.abs(want).max(), err_msg=ex["name"])
        # adjoint of the worked forward value: <A^T 1, V> = E
        E = oracle.siddon_ray(_vol(golden), ex["s"], ex["p"])
        assert abs(np.sum(bt * V) - E) <= 1e-12 * abs(E), ex["name"]
        done += 1
    assert done == 2


def test_worked_gradient(golden):
    V = _vol(golden)
    ex = [e for e in golden["examples"] if e["name"] == "generic"][0]
    d = np.array(ex["d"])
    L = np.linalg.norm(d)
    F = ex["F"]
    gs_hand = -d * F / L + L * np.array(ex["dF_ds"])
    gp_hand = d * F / L + L * np.array(ex["dF_dp"])
    _, gs, gp = oracle.siddon_ray(V, ex["s"], ex["p"], grad=True)
    np.testing.assert_allclose(gs, gs_hand, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(gp, gp_hand, rtol=1e-12, atol=1e-12)


def test_uniform_cube_axis_and_diagonal():
    # closed forms: chord through a cube of edge a is a along an axis, a*sqrt(3) along the main diagonal
    n, dlt, c = 8, 1.25, 0.37
    a = n * dlt
    V = oracle.Volume(np.full((n, n, n), c, np.float32), (dlt, dlt, dlt))
    E = oracle.siddon_ray(V, [-100.0, 0.1, -0.2], [100.0, 0.1, -0.2])
    assert abs(E - np.float32(c) * a) < 1e-12
    E = oracle.siddon_ray(V, [-50.0, -50.0, -50.0], [50.0, 50.0, 50.0])
    assert abs(E - np.float32(c) * a * np.sqrt(3)) < 1e-11
    E = oracle.siddon_ray(V, [-50.0, -50.0, 0.3], [50.0, 50.0, 0.3])
    assert abs(E - np.float32(c) * a * np.sqrt(2)) < 1e-11


def test_axis_aligned_column_sums():
    rng = np.random.default_rng(11)
    nz, ny, nx = 5, 6, 7
    sp = (0.8, 1.1, 2.0)
    data = rng.uniform(0, 1, (nz, ny, nx)).astype(np.float32)
    V = oracle.Volume(data, sp)
    b = -0.5 * np.array([nx * sp[0], ny * sp[1], nz * sp[2]])
    for (i, j, k) in [(0, 0, 0), (3, 2, 4), (6, 5, 1)]:
        xc, yc, zc = b + (np.array([i, j, k]) + 0.5) * np.array(sp)
        E = oracle.siddon_ray(V, [-100, yc, zc], [100, yc, zc])
        assert abs(E - sp[0] * data[k, j, :].astype(np.float64).sum()) < 1e-12
        E = oracle.siddon_ray(V, [xc, 100, zc], [xc, -100, zc])
        assert abs(E - sp[1] * data[k, :, i].astype(np.float64).sum()) < 1e-12
        E = oracle.siddon_ray(V, [xc, yc, -100], [xc, yc, 100])
        assert abs(E - sp[2] * data[:, j, i].astype(np.float64).sum()) < 1e-12


def _random_ray(rng, ext, inside_prob=0.2):
    """Endpoints on a sphere around the box, sometimes inside the box."""
    def pt():
        if rng.uniform() < inside_prob:
            return rng.uniform(-0.5, 0.5, 3) * ext
        v = rng.normal(size=3)
        return v / np.linalg.norm(v) * np.linalg.norm(ext) * rng.uniform(0.6, 2.0)
    return pt(), pt()


def test_brute_force_random_small_volumes():
    rng = np.random.default_rng(12)
    for trial in range(12):
        n = rng.integers(1, 11, size=3)
        sp = rng.uniform(0.3, 2.5, size=3)
        data = rng.uniform(0, 1, (n[2], n[1], n[0])).astype(np.float32)
        data[rng.uniform(size=data.shape) < 0.3] = 0.0
        V = oracle.Volume(data, sp)
        ext = n * sp
        for _ in range(25):
            s, p = _random_ray(rng, ext)
            E = oracle.siddon_ray(V, s, p)
            Eb = oracle.brute_ray(V, s, p)
            assert abs(E - Eb) <= 1e-12 * max(1.0, abs(Eb)), (trial, s, p, E, Eb)


def test_single_voxel_volume():
    V = oracle.Volume(np.full((1, 1, 1), 2.0, np.float32), (3.0, 4.0, 5.0))
    # through the centre along x: chord 3 mm
    assert abs(oracle.siddon_ray(V, [-10, 0, 0], [10, 0, 0]) - 6.0) < 1e-12
    rng = np.random.default_rng(3)
    for _ in range(50):
        s, p = _random_ray(rng, np.array([3.0, 4.0, 5.0]))
        assert abs(oracle.siddon_ray(V, s, p) - oracle.brute_ray(V, s, p)) < 1e-12


def test_sampling_converges():
    rng = np.random.default_rng(13)
    data = rng.uniform(0, 1, (6, 7, 8)).astype(np.float32)
    V = oracle.Volume(data, (1.0, 0.9, 1.7))
    s, p = np.array([-20.0, -3.1, 2.2]), np.array([15.0, 4.4, -3.7])
    E = oracle.siddon_ray(V, s, p)
    L = np.linalg.norm(p - s)
    n_disc = 8 + 7 + 6 + 2 + 2  # plane crossings plus entry and exit
    for N in (1000, 10000, 100000, 1000000):
        err = abs(oracle.sample_ray(V, s, p, N) - E)
        # a midpoint cell without a discontinuity is exact; one with a jump errs by at most
        # |jump| * L / N, so the error is bounded by L * (#discontinuities) * max V / N
        assert err <= L * n_disc * float(data.max()) / N


def test_sum_of_lengths_is_clipped_chord():
    rng = np.random.default_rng(14)
    n = np.array([9, 7, 5])
    sp = np.array([0.7, 1.3, 2.5])
    ones = oracle.Volume(np.ones((n[2], n[1], n[0]), np.float32), sp)
    for _ in range(40):
        s, p = _random_ray(rng, n * sp, inside_prob=0.3)
        total = oracle.siddon_total_length(ones, s, p)
        # chord of the segment with the box from the per-voxel brute force (independent algorithm)
        assert abs(total - oracle.brute_ray(ones, s, p)) < 1e-12 * max(1, total)


def test_symmetry_and_linearity():
    rng = np.random.default_rng(15)
    n = (6, 5, 4)
    V1 = rng.uniform(0, 1, n[::-1]).astype(np.float32)
    V2 = rng.uniform(0, 1, n[::-1]).astype(np.float32)
    sp = (1.0, 1.2, 0.8)
    a, b = 0.75, 1.5
    comb = (a * V1.astype(np.float64) + b * V2.astype(np.float64)).astype(np.float32)
    for _ in range(20):
        s, p = _random_ray(rng, np.array(n) * sp)
        e1 = oracle.siddon_ray(oracle.Volume(V1, sp), s, p)
        assert abs(e1 - oracle.siddon_ray(oracle.Volume(V1, sp), p, s)) < 1e-12 * max(1, e1)
        e2 = oracle.siddon_ray(oracle.Volume(V2, sp), s, p)
        ec = oracle.siddon_ray(oracle.Volume(comb, sp), s, p)
        assert abs(ec - (a * e1 + b * e2)) < 1e-6 * max(1, ec)  # comb rounded to float32


def test_sphere_convergence():
    # voxelised ball of radius r: E -> c * 2 sqrt(r^2 - dist^2) as voxels shrink
    r, c = 10.0, 1.0
    s, p = np.array([-40.0, 3.0, 2.0]), np.array([40.0, 3.3, 1.9])
    d = p - s
    u = d / np.linalg.norm(d)
    dist2 = np.sum(s * s) - np.dot(s, u) ** 2
    exact = c * 2 * np.sqrt(r * r - dist2)
    errs = []
    for n in (16, 32, 64):
        dl = 2.2 * r / n
        xs = (np.arange(n) + 0.5) * dl - 0.5 * n * dl
        Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
        ball = ((X ** 2 + Y ** 2 + Z ** 2) <= r * r).astype(np.float32) * c
        errs.append(abs(oracle.siddon_ray(oracle.Volume(ball, (dl, dl, dl)), s, p) - exact))
    assert errs[-1] < 0.1 * exact * 0.2
    assert errs[2] < errs[0]


def test_parallel_ray_inside_and_outside():
    data = np.arange(1, 9, dtype=np.float32).reshape(2, 2, 2)
    V = oracle.Volume(data, (1, 1, 1))
    # d_y = d_z = 0, s_y in [-1, 1) -> counted; outside -> 0
    assert oracle.siddon_ray(V, [-5, 0.5, 0.5], [5, 0.5, 0.5]) == pytest.approx(7 + 8, abs=1e-12)
    assert oracle.siddon_ray(V, [-5, 1.5, 0.5], [5, 1.5, 0.5]) == 0.0
    assert oracle.siddon_ray(V, [-5, 0.5, -1.0], [5, 0.5, -1.0]) == pytest.approx(3 + 4, abs=1e-12)


def test_segment_inside_the_box():
    # both endpoints inside: only the part between them counts (clamp to [0, 1])
    data = np.full((4, 4, 4), 0.5, np.float32)
    V = oracle.Volume(data, (1, 1, 1))
    assert oracle.siddon_ray(V, [-1.2, 0.1, 0.1], [0.8, 0.1, 0.1]) == pytest.approx(1.0, abs=1e-12)


def test_segment_count_is_voxels_crossed():
    # with no coincident crossings, segments == voxels the segment passes through with positive length
    rng = np.random.default_rng(16)
    n = np.array([5, 4, 6])
    sp = np.array([1.1, 0.9, 1.3])
    b = -0.5 * n * sp
    det = (30.0, 3, 4, 0.7, 0.9)
    poses = np.array([[0.3, -0.2, 0.1, 0.4, -0.3, 0.2], [1.1, 0.5, -0.7, -0.2, 0.6, -0.1]], np.float32)
    counts = oracle.count_segments(n[::-1], sp, det, poses)
    for bi in range(2):
        for h in range(3):
            for w in range(4):
                s, p = oracle.ray_endpoints(poses[bi].astype(np.float64), *det, h, w)
                d = p - s
                crossed = 0
                for k in range(n[2]):
                    for j in range(n[1]):
                        for i in range(n[0]):
                            lo = b + np.array([i, j, k]) * sp
                            hi = lo + sp
                            t0, t1 = (lo - s) / d, (hi - s) / d
                            tl = max(0.0, np.max(np.minimum(t0, t1)))
                            th = min(1.0, np.min(np.maximum(t0, t1)))
                            crossed += th - tl > 1e-12
                assert counts[bi, h, w] == crossed
