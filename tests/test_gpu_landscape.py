"""GPU tests of the loss-landscape sweep (Sec. 3.2): -ZNCC of DRRs at displaced
poses against one fixed image, through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import FP32_TOL, f32, odet, ovol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def _zncc_tol(fixed):
    # Every pixel of a DRR is within FP32_TOL * max E of the oracle's; a
    # perturbation dI moves the normalised image by at most 2 |dI| / std(I), so
    # -ZNCC moves by at most 2 * FP32_TOL * max / std (doubled for margin).
    f = np.asarray(fixed, np.float64)
    return 4.0 * FP32_TOL * f.max() / f.std()


def test_landscape_vs_oracle_tiny(drr):
    cfg = inputs.TINY
    vol_np = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    vol = drr.Volume(vol_np, cfg["spacing"])
    truth = inputs.random_poses(1, seed=120)
    poses = np.concatenate([truth, truth + inputs.landscape_offsets(40, seed=121)]).astype(np.float32)
    ov, od = ovol(vol_np, cfg["spacing"]), odet(det)
    fixed = oracle.render(ov, od, truth)[0].astype(np.float32)
    ref = oracle.loss_landscape(ov, od, fixed, poses)
    P = torch.from_numpy(poses).cuda()
    Fd = torch.from_numpy(fixed).cuda()
    got = drr.loss_landscape(vol, det, Fd, P).cpu().numpy()
    assert np.abs(got - ref).max() < _zncc_tol(fixed)
    assert got[0] < -1.0 + 1e-5  # the true pose reproduces the fixed image
    # chunking changes nothing: each pose is rendered and scored on its own
    got3 = drr.loss_landscape(vol, det, Fd, P, chunk=3).cpu().numpy()
    np.testing.assert_array_equal(got, got3)
    # and equals render + zncc called separately
    E = drr.render(vol, det, P)
    sep = drr.zncc(E, Fd.expand_as(E).contiguous(), grad=False).cpu().numpy()
    np.testing.assert_array_equal(got, sep)


def test_landscape_ct_full_size_sampled(drr):
    cfg = inputs.LANDSCAPE
    hu = inputs.ct_volume_hu()
    det = cfg["detector"]
    vol = drr.Volume(hu, cfg["spacing"], hu=True)
    truth = inputs.random_poses(1, seed=cfg["truth_seed"])
    offs = inputs.landscape_offsets(cfg["n"], seed=cfg["offset_seed"])
    poses = (truth + offs).astype(np.float32)
    P = torch.from_numpy(poses).cuda()
    fixed = drr.render(vol, det, torch.from_numpy(truth).cuda())[0]
    got = drr.loss_landscape(vol, det, fixed, P).cpu().numpy()
    assert got.shape == (cfg["n"],) and np.all(np.isfinite(got))
    assert np.all(got >= -1.0 - 1e-5) and np.all(got <= 1.0 + 1e-5)
    # sampled poses against the oracle (full DRRs, so only a few)
    mu = oracle.hu_to_mu(hu, inputs.MU_WATER).astype(np.float32)
    ov, od = ovol(mu, cfg["spacing"]), odet(det)
    fixed_ref = oracle.render(ov, od, truth)[0]
    idx = np.array([0, 1, 1000, cfg["n"] - 1])
    ref = oracle.loss_landscape(ov, od, fixed.cpu().numpy(), poses[idx])
    assert np.abs(got[idx] - ref).max() < _zncc_tol(fixed_ref)


def test_landscape_argument_errors(drr):
    cfg = inputs.TINY
    vol = drr.Volume(np.ones((8, 8, 8), np.float32), (1.0, 1.0, 1.0))
    det = inputs.Detector(100.0, 8, 8, 1.0, 1.0)
    P = torch.zeros((2, 6), device="cuda")
    F = torch.ones((8, 8), device="cuda")
    with pytest.raises(drr.DrrError):
        drr.loss_landscape(vol, det, F, P, eps=-1.0)
    with pytest.raises(drr.DrrError):
        drr.loss_landscape(vol, det, F, P, chunk=-2)
    with pytest.raises(Exception):
        drr.loss_landscape(vol, det, torch.ones((7, 8), device="cuda"), P)
