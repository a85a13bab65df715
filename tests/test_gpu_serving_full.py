"""The serving workload at its full sizes: 8 resident volumes {128^3, 256^3,
512x512x133, 512x512x300} x {FP32, BF16}, one pose per request, square
detectors of 128..512 pixels, half of the requests with a pose gradient, all
queued at once so that the server packs them into capped ticks.  Every 10th
request is checked against the FP64 oracle on sampled pixels (16-bit volumes
against the oracle on the de-quantised volume, which the kernel must meet to the
FP32 bound), its gradient equal to the direct calls' bit for bit; a few
requests served again alone give the same bits as in the mix."""
import numpy as np
import pytest

import oracle
from paper_2208_12737_gb300 import inputs
from tests._parity import FP32_TOL, GRAD_TOL, grad_err, odet, ovol, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_REQ = 60
SAMPLES = 64  # pixels per checked request


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


@pytest.fixture(scope="module")
def volumes(drr):
    """(name, device volume, FP32 attenuation the oracle sees for that storage, spacing)."""
    specs = [
        ("128^3", inputs.ellipsoid_phantom((128, 128, 128), (2.0, 2.0, 2.0), seed=81, semi_range=(10, 60),
                                           density_range=(0.0, 0.01)), False, (2.0, 2.0, 2.0)),
        ("256^3", inputs.ellipsoid_phantom((256, 256, 256), (1.0, 1.0, 1.0), seed=82, semi_range=(10, 60),
                                           density_range=(0.0, 0.01)), False, (1.0, 1.0, 1.0)),
        ("512x512x133", inputs.ct_phantom_hu((133, 512, 512), (0.703, 0.703, 2.5), seed=2), True,
         (0.703, 0.703, 2.5)),
        ("512x512x300", inputs.ct_phantom_hu((300, 512, 512), (0.703, 0.703, 1.1), seed=83), True,
         (0.703, 0.703, 1.1)),
    ]
    out = []
    for name, data, hu, sp in specs:
        mu = oracle.hu_to_mu(data, inputs.MU_WATER).astype(np.float32) if hu else data
        for storage in ("f32", "bf16"):
            vol = drr.Volume(data, sp, hu=hu, storage=storage)
            seen = mu if storage == "f32" else oracle.round_bf16(mu)
            out.append((f"{name}/{storage}", vol, seen, sp))
    return out


def _requests(n_vols, seed=8):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(N_REQ):
        v = int(rng.integers(n_vols))
        n = int(rng.integers(128, 513))
        det = inputs.Detector(510.0, n, n, 280.0 / n, 280.0 / n)
        pose = inputs.random_poses(1, seed=900 + i)
        g = inputs.upstream_grad((1, n, n), seed=n) if rng.uniform() < 0.5 else None
        reqs.append((v, det, pose, g))
    return reqs


def test_full_size_stream(drr, volumes):
    reqs = _requests(len(volumes))
    srv = drr.Server(device_budget=2 << 30, max_inflight=64, max_tick_work=1 << 30)
    tickets = [srv.submit(volumes[v][1], det, pose, g) for (v, det, pose, g) in reqs]
    results = [t.wait(120000) for t in tickets]
    st = srv.stats()
    assert st["completed"] == N_REQ and st["failed"] == 0
    assert st["ticks"] > 1  # the cap split the stream into several ticks
    srv.close()

    rng = np.random.default_rng(9)
    for i in range(0, N_REQ, 10):
        v, det, pose, g = reqs[i]
        name, vol, seen, sp = volumes[v]
        E, G = results[i]
        n = det.height
        pix = rng.choice(n * n, SAMPLES, replace=False)
        E_ref = oracle.render(ovol(seen, sp), odet(det), pose, pixels=pix)
        err = rel_err(E.reshape(1, -1)[:, pix], E_ref)
        assert err.max() < FP32_TOL, (name, n, float(err.max()))
        if g is None:
            continue
        # the server's gradient is the direct call's (same walk, same partial sums and order)
        poses_d = torch.from_numpy(pose).cuda()
        G_d = drr.render_backward(vol, det, poses_d, torch.from_numpy(g).cuda()).cpu().numpy()
        np.testing.assert_array_equal(G, G_d)

    # the smallest gradient request's whole-image pose gradient against the oracle
    i = min((i for i in range(N_REQ) if reqs[i][3] is not None), key=lambda i: reqs[i][1].height)
    v, det, pose, g = reqs[i]
    name, vol, seen, sp = volumes[v]
    G_ref = oracle.pose_grad(ovol(seen, sp), odet(det), pose, g.astype(np.float64))
    assert grad_err(results[i][1], G_ref).max() < GRAD_TOL, (name, det.height)

    # alone and in the mix: the same bits
    for i in (3, 27, 51):
        v, det, pose, g = reqs[i]
        srv = drr.Server(device_budget=2 << 30)
        E1, G1 = srv.submit(volumes[v][1], det, pose, g).wait(120000)
        srv.close()
        np.testing.assert_array_equal(E1, results[i][0])
        if g is not None:
            np.testing.assert_array_equal(G1, results[i][1])
