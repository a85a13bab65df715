"""Stream order across the library's launches.  Pose setup, the walks and the
stored-Jacobian reduction are launched with programmatic dependent launch: each
may be scheduled while the kernel before it is still running, and must wait for
it before touching memory.  Here torch kernels and library calls alternate on
one stream with no host synchronisation between them: every call must see the
inputs the kernel just before it wrote, and must not overwrite a buffer that
kernel is still reading."""
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


def test_inputs_written_just_before_a_call_are_seen(drr):
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    vol = drr.Volume(inputs.ct_phantom_hu(shape, sp, seed=91), sp, hu=True)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    B, n = 4, 12
    sets = [torch.from_numpy(inputs.random_poses(B, seed=100 + i)).cuda() for i in range(n)]
    grads = [torch.from_numpy(inputs.upstream_grad((B, 45, 61), seed=200 + i)).cuda() for i in range(n)]
    # references, each computed alone with the device idle before the call
    ref_E, ref_G = [], []
    for P, g in zip(sets, grads):
        torch.cuda.synchronize()
        E, J = drr.render(vol, det, P, jacobian=True)
        G = drr.render_backward(vol, det, P, g, jac=J)
        torch.cuda.synchronize()
        ref_E.append(E.clone())
        ref_G.append(G.clone())
    # one pose buffer and one gradient buffer rewritten by a torch kernel right
    # before each call; the library's outputs go to buffers that the next torch
    # kernel reads right after
    P = torch.empty_like(sets[0])
    g = torch.empty_like(grads[0])
    E = torch.empty((B, 45, 61), device="cuda")
    J = torch.empty((B, 6, 45, 61), device="cuda")
    outs_E, outs_G = [], []
    torch.cuda.synchronize()
    for i in range(n):
        P.copy_(sets[i])
        drr.render(vol, det, P, jacobian=True, out=E, jac=J)
        outs_E.append(E.clone())  # read right after the walk, before E is overwritten
        g.copy_(grads[i])
        outs_G.append(drr.render_backward(vol, det, P, g, jac=J))
        P.fill_(float("nan"))  # the next iteration's copy must land before its setup runs
    torch.cuda.synchronize()
    for i in range(n):
        assert torch.equal(outs_E[i], ref_E[i]), i
        assert torch.equal(outs_G[i], ref_G[i]), i


def test_rewalk_gradient_and_backprojection_in_one_stream(drr):
    shape, sp = (24, 30, 28), (1.1, 1.3, 0.9)
    rng = np.random.default_rng(92)
    vol = drr.Volume(rng.uniform(0.0, 0.05, shape).astype(np.float32), sp)
    det = inputs.Detector(300.0, 33, 29, 1.6, 1.7)
    P = torch.from_numpy(inputs.random_poses(3, seed=93)).cuda()
    g = torch.from_numpy(inputs.upstream_grad((3, 33, 29), seed=94)).cuda()
    torch.cuda.synchronize()
    G_ref = drr.render_backward(vol, det, P, g)
    gv_ref = torch.zeros(shape, device="cuda")
    drr.render_backward(vol, det, P, g, pose_grad=False, grad_volume=gv_ref)
    torch.cuda.synchronize()
    # the same calls with the inputs produced by the kernels just before them
    P2 = torch.zeros_like(P)
    g2 = torch.zeros_like(g)
    gv = torch.zeros(shape, device="cuda")
    P2.add_(P)
    g2.add_(g)
    G = drr.render_backward(vol, det, P2, g2)
    g2.mul_(2.0)
    drr.render_backward(vol, det, P2, g2, pose_grad=False, grad_volume=gv)
    torch.cuda.synchronize()
    assert torch.equal(G, G_ref)
    # the back-projection accumulates with atomics: equal up to the order of the adds
    scale = float(gv_ref.abs().max())
    assert float((gv - 2.0 * gv_ref).abs().max()) <= 1e-5 * scale


def test_calls_from_several_threads_on_their_own_streams(drr):
    # four host threads, each with its own stream, render and differentiate at once
    # (the library's per-device launch caches and stream-ordered scratch are shared):
    # every result equals the same call made alone
    import threading
    shape, sp = (40, 96, 80), (1.4, 1.2, 3.1)
    vol = drr.Volume(inputs.ct_phantom_hu(shape, sp, seed=92), sp, hu=True)
    det = inputs.Detector(420.0, 45, 61, 2.4, 2.1)
    work = [(torch.from_numpy(inputs.random_poses(1 + i % 3, seed=300 + i)).cuda(),
             torch.from_numpy(inputs.upstream_grad((1 + i % 3, 45, 61), seed=400 + i)).cuda()) for i in range(4)]
    ref = []
    for P, g in work:
        E, J = drr.render(vol, det, P, jacobian=True)
        ref.append((E.cpu().numpy(), drr.render_backward(vol, det, P, g, jac=J).cpu().numpy(),
                    drr.render_backward(vol, det, P, g).cpu().numpy()))
    torch.cuda.synchronize()
    got = [None] * 4
    errors = []

    def run(i):
        try:
            P, g = work[i]
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                out = []
                for _ in range(5):
                    E, J = drr.render(vol, det, P, jacobian=True, stream=s)
                    G = drr.render_backward(vol, det, P, g, jac=J, stream=s)
                    Gw = drr.render_backward(vol, det, P, g, stream=s)
                    out.append((E, G, Gw))
                s.synchronize()
                got[i] = [(E.cpu().numpy(), G.cpu().numpy(), Gw.cpu().numpy()) for E, G, Gw in out]
        except Exception as e:  # reported below
            errors.append(e)

    threads = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=120)
    assert not errors, errors
    for i in range(4):
        for E, G, Gw in got[i]:
            np.testing.assert_array_equal(E, ref[i][0])
            np.testing.assert_array_equal(G, ref[i][1])
            np.testing.assert_array_equal(Gw, ref[i][2])
    drr.stream_check()
