"""The bench's context baseline for the paper's own vectorised formulation (Sec. 2.3,
plain tensor ops in FP32) computes the same integral as the FP64 oracle, to FP32
accuracy; checked on the CPU on the 64^3 configuration."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs

torch = pytest.importorskip("torch")


def test_vectorised_tensor_siddon_matches_oracle():
    import bench
    cfg = inputs.TINY
    vol = inputs.ellipsoid_phantom(cfg["shape_zyx"], cfg["spacing"], seed=cfg["phantom_seed"])
    det = cfg["detector"]
    poses = inputs.random_poses(2, seed=5)
    E = bench.vgs_torch_forward(torch.from_numpy(vol), cfg["spacing"], det, torch.from_numpy(poses)).numpy()
    ref = oracle.render(oracle.Volume(vol, cfg["spacing"]), det.as_tuple(), poses)
    r = np.abs(E - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    assert r.max() < 1e-3 and np.median(r) < 1e-5, (r.max(), np.median(r))
    assert np.all(E[ref == 0] == 0)
