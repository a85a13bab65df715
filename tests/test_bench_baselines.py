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


def test_fifo_replay_of_the_plain_serving_baseline():
    import bench
    # three requests at once, one unit each: they leave at 1, 2, 3
    np.testing.assert_allclose(bench.fifo_latencies([0.0, 0.0, 0.0], [1.0, 1.0, 1.0]), [1.0, 2.0, 3.0])
    # arrivals spaced wider than the service: no waiting
    np.testing.assert_allclose(bench.fifo_latencies([0.0, 5.0, 9.0], [1.0, 2.0, 0.5]), [1.0, 2.0, 0.5])
    # a queue that builds and drains
    np.testing.assert_allclose(bench.fifo_latencies([0.0, 0.5, 1.0, 10.0], [2.0, 2.0, 2.0, 1.0]),
                               [2.0, 3.5, 5.0, 1.0])
