"""The C ABI's render and pose-gradient calls can be captured in a CUDA graph (their
scratch comes from the stream-ordered allocator) and replayed with new poses and
upstream gradients written into the captured input buffers; replays give the same
bits as direct calls."""
import numpy as np
import pytest

from paper_2208_12737_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def test_capture_and_replay_matches_direct_calls(drr):
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    hu = inputs.ct_phantom_hu(shape, sp, seed=71)
    vol = drr.Volume(hu, sp, hu=True)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    B = 3
    poses = torch.from_numpy(inputs.random_poses(B, seed=72)).cuda()
    g = torch.from_numpy(inputs.upstream_grad((B, det.height, det.width), seed=73)).cuda()
    E = torch.empty((B, det.height, det.width), device="cuda")
    J = torch.empty((B, 6, det.height, det.width), device="cuda")
    G = torch.empty((B, 6), device="cuda")

    def step():
        drr.render(vol, det, poses, jacobian=True, out=E, jac=J)
        G.copy_(drr.render_backward(vol, det, poses, g, jac=J))

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(2):  # warm-up outside the capture
            step()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for seed in (74, 75):
        new_p = torch.from_numpy(inputs.random_poses(B, seed=seed)).cuda()
        new_g = torch.from_numpy(inputs.upstream_grad((B, det.height, det.width), seed=seed)).cuda()
        poses.copy_(new_p)
        g.copy_(new_g)
        graph.replay()
        torch.cuda.synchronize()
        E_d, J_d = drr.render(vol, det, new_p, jacobian=True)
        G_d = drr.render_backward(vol, det, new_p, new_g, jac=J_d)
        np.testing.assert_array_equal(E.cpu().numpy(), E_d.cpu().numpy())
        np.testing.assert_array_equal(G.cpu().numpy(), G_d.cpu().numpy())
