"""The split walk: a fused forward + pose-Jacobian launch too small to fill the
GPU walks each ray on 8 or 4 lanes (whole chunks per lane, the exact walk state
rebuilt at each lane's first chunk boundary, the chunk sums added in chunk
order).  Its DRR and per-ray Jacobian must be the same bits as the one-lane
walk's, which the same rays take inside a launch large enough to fill the GPU;
and they stay within the tolerances of the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import odet, ovol, FP32_TOL, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _cases():
    q = np.pi / 4
    c = np.arctan(1.0 / np.sqrt(2.0))
    yield ("small_ct", lambda: (oracle.hu_to_mu(inputs.ct_phantom_hu((40, 96, 80), (1.4, 1.2, 3.1), seed=51),
                                                inputs.MU_WATER).astype(np.float32), (1.4, 1.2, 3.1)),
           inputs.Detector(420.0, 45, 61, 2.4, 2.1), inputs.random_poses(2, seed=52))
    # near-coincident crossings: chunks taken by the exact re-walk, ties at chunk boundaries
    yield ("coincident", lambda: (inputs.ellipsoid_phantom((32, 32, 32), (1.0, 1.0, 1.0), seed=61), (1.0, 1.0, 1.0)),
           inputs.Detector(200.0, 24, 24, 1.0, 1.0),
           np.array([[q + 1e-5, 0, 0, 0.13, 0.07, 0.02], [q + 1e-5, c + 2e-5, 0, 0.1, 0.05, -0.07]], np.float32))
    # source and detector inside the volume: clamped entry and exit
    rng = np.random.default_rng(47)
    yield ("inside", lambda: (rng.uniform(0.0, 0.05, (30, 34, 38)).astype(np.float32), (1.0, 1.0, 1.0)),
           inputs.Detector(20.0, 16, 16, 0.9, 0.9),
           np.concatenate([inputs.random_poses(1, seed=48, max_angle_deg=90, max_trans_mm=5),
                           np.zeros((1, 6), np.float32)]))
    # exact quarter turns: rays parallel to voxel planes
    rng2 = np.random.default_rng(49)
    yield ("axis", lambda: (rng2.uniform(0.0, 0.05, (20, 22, 24)).astype(np.float32), (1.1, 0.9, 1.3)),
           inputs.Detector(200.0, 9, 11, 1.0, 1.0),
           np.array([[0, 0, 0, 0.1, 0.2, 0.3], [np.pi / 2, 0, 0, 0, 0, 0]], np.float32))


    # one voxel: every ray has a single segment (no crossing at all)
    yield ("one_voxel", lambda: (np.full((1, 1, 1), 0.02, np.float32), (40.0, 40.0, 40.0)),
           inputs.Detector(200.0, 12, 10, 1.0, 1.0), inputs.random_poses(2, seed=53, max_angle_deg=20))


@pytest.mark.parametrize("case,storage", [(c[0], "f32") for c in _cases()] + [("small_ct", "bf16"),
                                                                             ("coincident", "f16")])
def test_split_walk_gives_the_one_lane_bits(drr, case, storage):
    name, make, det, poses_np = next(c for c in _cases() if c[0] == case)
    vol_np, sp = make()
    vol = drr.Volume(vol_np, sp, storage=storage)
    B = poses_np.shape[0]
    res = {}
    for reps in (1, 3, 256):  # 8 lanes, 4 (or 8) lanes, and one lane per ray
        P = torch.from_numpy(np.concatenate([poses_np] * reps)).cuda()
        drr.profile_reset()
        drr.profile_enable(True)
        E, J = drr.render(vol, det, P, jacobian=True)
        drr.profile_enable(False)
        res[reps] = (E[:B].cpu().numpy(), J[:B].cpu().numpy(), drr.profile_read("siddon_fwd_jac_split")[1])
        drr.profile_reset()
    assert res[1][2] == 1 and res[256][2] == 0  # the small launch was split, the large one not
    for reps in (1, 3):
        np.testing.assert_array_equal(res[reps][0], res[256][0])
        np.testing.assert_array_equal(res[reps][1], res[256][1])
    if storage == "f32":
        E_ref = oracle.render(ovol(vol_np, sp), odet(det), poses_np)
        assert rel_err(res[1][0], E_ref).max() < FP32_TOL
