"""Buffers in page-locked host memory: drr_render and drr_render_backward read
poses and upstream gradients from, and write E, the Jacobian and dL/d eta to,
pinned host memory in place, with the same bits as with device buffers; a
pageable host buffer, or host memory for the atomically accumulated volume
gradient, is rejected before any launch."""
import ctypes

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


@pytest.fixture(scope="module")
def case(drr):
    hu = inputs.ct_phantom_hu((40, 96, 80), (1.4, 1.2, 3.1), seed=61)
    vol = drr.Volume(hu, (1.4, 1.2, 3.1), hu=True)
    det = inputs.Detector(420.0, 45, 53, 1.9, 1.7)
    poses = inputs.random_poses(5, seed=62)
    g = inputs.upstream_grad((5, 45, 53), seed=63)
    return vol, det, poses, g


def test_pinned_host_buffers_give_the_device_bits(drr, case):
    vol, det, poses_np, g_np = case
    poses_d = torch.from_numpy(poses_np).cuda()
    E_d, J_d = drr.render(vol, det, poses_d, jacobian=True)
    G_d = drr.render_backward(vol, det, poses_d, torch.from_numpy(g_np).cuda(), jac=J_d)
    F_d = drr.render(vol, det, poses_d)
    G_w = drr.render_backward(vol, det, poses_d, torch.from_numpy(g_np).cuda())

    poses_h = torch.from_numpy(poses_np).pin_memory()
    g_h = torch.from_numpy(g_np).pin_memory()
    E_h = torch.empty((5, 45, 53)).pin_memory()
    J_h = torch.empty((5, 6, 45, 53)).pin_memory()
    G_h = torch.empty((5, 6)).pin_memory()
    F_h = torch.empty((5, 45, 53)).pin_memory()
    Gw_h = torch.empty((5, 6)).pin_memory()
    drr.render(vol, det, poses_h, jacobian=True, out=E_h, jac=J_h)
    drr.render_backward(vol, det, poses_h, g_h, jac=J_h, grad_pose_out=G_h)
    drr.render(vol, det, poses_h, out=F_h)
    drr.render_backward(vol, det, poses_h, g_h, grad_pose_out=Gw_h)
    torch.cuda.synchronize()
    for host, dev in ((E_h, E_d), (J_h, J_d), (G_h, G_d), (F_h, F_d), (Gw_h, G_w)):
        np.testing.assert_array_equal(host.numpy(), dev.cpu().numpy())


def test_pageable_and_misplaced_buffers_are_rejected(drr, case):
    vol, det, poses_np, g_np = case
    lib = drr.load()
    d = drr.detector(det)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    poses_d = torch.from_numpy(poses_np).cuda()
    out_d = torch.empty((5, 45, 53), device="cuda")
    pageable = np.zeros((5, 45, 53), np.float32)
    pageable_poses = np.ascontiguousarray(poses_np, np.float32)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    # pageable output / poses: DRR_ERR_INVALID, nothing launched
    st = lib.drr_render(vol.handle, ctypes.byref(d), ptr(poses_d), 5, ctypes.c_void_p(pageable.ctypes.data), None,
                        stream)
    assert st == 1 and "pageable" in lib.drr_last_error().decode()
    st = lib.drr_render(vol.handle, ctypes.byref(d), ctypes.c_void_p(pageable_poses.ctypes.data), 5, ptr(out_d),
                        None, stream)
    assert st == 1
    # the volume gradient is accumulated with atomics: device memory only
    gv_h = torch.zeros(vol.shape_zyx).pin_memory()
    st = lib.drr_render_backward(vol.handle, ctypes.byref(d), ptr(poses_d), 5, ptr(torch.from_numpy(g_np).cuda()),
                                 None, None, ptr(gv_h), stream)
    assert st == 1 and "device memory" in lib.drr_last_error().decode()
    assert np.all(pageable == 0) and float(gv_h.abs().sum()) == 0.0
    # the other entry points check their buffers the same way
    st = lib.drr_zncc(ctypes.c_void_p(pageable.ctypes.data), ptr(out_d), 5, 45 * 53, ctypes.c_float(1e-8),
                      ptr(torch.empty(5, device="cuda")), None, stream)
    assert st == 1
    jac_d = torch.zeros((5, 6, 45, 53), device="cuda")
    st = lib.drr_pose_grad_noalloc(ctypes.byref(d), 5, ctypes.c_void_p(pageable.ctypes.data), ptr(jac_d),
                                   ptr(torch.empty((5, 6), device="cuda")), stream)
    assert st == 1
    # the Python binding refuses a CPU tensor that is not pinned
    with pytest.raises(TypeError):
        drr.render(vol, det, torch.from_numpy(poses_np))
    drr.stream_check()


def test_autograd_with_pinned_host_poses(drr, case):
    # drr.drr on pinned host poses: E on the device, dL/d poses back on the host, equal to
    # the device-pose gradient
    vol, det, poses_np, g_np = case
    p_dev = torch.from_numpy(poses_np).cuda().requires_grad_(True)
    p_host = torch.from_numpy(poses_np).pin_memory().requires_grad_(True)
    g = torch.from_numpy(g_np).cuda()
    (drr.drr(vol, det, p_dev) * g).sum().backward()
    (drr.drr(vol, det, p_host) * g).sum().backward()
    assert p_host.grad.device.type == "cpu"
    np.testing.assert_array_equal(p_host.grad.numpy(), p_dev.grad.cpu().numpy())
