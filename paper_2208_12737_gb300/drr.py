"""ctypes binding of libdrr (include/drr.h) and a torch.autograd.Function.

Argument marshalling only: torch supplies device memory and the current
CUDA stream; every step of the DRR computation runs in libdrr's kernels.
The library must have been built (``paper_2208_12737_gb300.build.build()``);
if it is missing, loading raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdrr.so")

DRR_F32, DRR_BF16, DRR_F16, DRR_I16_HU = 0, 1, 2, 3
LAYOUT = {"default": 0, "x": 1, "y": 2, "z": 3}  # drr_layout: the fastest axis of the padded storage
_STATUS = {0: "DRR_OK", 1: "DRR_ERR_INVALID", 2: "DRR_ERR_OOM", 3: "DRR_ERR_CUDA", 4: "DRR_ERR_TIMEOUT",
           5: "DRR_ERR_BUSY", 6: "DRR_ERR_NOT_FOUND", 7: "DRR_ERR_DEVICE", 8: "DRR_ERR_CANCELLED"}
STORAGE = {"f32": DRR_F32, "bf16": DRR_BF16, "f16": DRR_F16}

# Every symbol include/drr.h declares (checked by the CPU tests).
EXPORTS = (
    "drr_volume_create", "drr_volume_destroy", "drr_volume_info", "drr_render", "drr_render_backward",
    "drr_ray_setup", "drr_count_segments", "drr_profile_enable", "drr_profile_read", "drr_profile_reset",
    "drr_launch_count", "drr_stream_check", "drr_last_error", "drr_version",
    "drr_server_create", "drr_server_submit", "drr_server_wait", "drr_server_cancel", "drr_server_get_stats",
    "drr_server_pause", "drr_server_destroy", "drr_arena_create", "drr_arena_alloc", "drr_arena_free", "drr_arena_in_use",
    "drr_arena_largest_free", "drr_arena_destroy", "drr_pose_grad_noalloc", "drr_zncc", "drr_adam_step",
    "drr_loss_landscape", "drr_geometry_grad", "drr_probe_l2_read", "drr_render_plain_fp32",
    "drr_server_poll", "drr_server_inject_device_status", "drr_serve_tick_layout", "drr_bounds_checked",
)


class DrrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class drr_detector(ctypes.Structure):
    _fields_ = [("sdr_mm", ctypes.c_float), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("delta_h_mm", ctypes.c_float), ("delta_w_mm", ctypes.c_float)]


class drr_volume_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("hu_mu_water", ctypes.c_float), ("layout", ctypes.c_int32)]


class drr_server_config(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_size_t), ("host_budget_bytes", ctypes.c_size_t),
                ("max_inflight", ctypes.c_int32), ("max_tick_poses", ctypes.c_int32),
                ("use_cuda_graph", ctypes.c_int32), ("device", ctypes.c_int32),
                ("max_tick_work", ctypes.c_int64), ("plain_fp32_baseline", ctypes.c_int32),
                ("tick_depth", ctypes.c_int32), ("spin_poll_us", ctypes.c_int32)]


class drr_request(ctypes.Structure):
    _fields_ = [("volume", ctypes.c_void_p), ("detector", drr_detector), ("B", ctypes.c_int32),
                ("poses", ctypes.c_void_p), ("grad_drr", ctypes.c_void_p), ("drr_out", ctypes.c_void_p),
                ("grad_pose_out", ctypes.c_void_p), ("fixed", ctypes.c_void_p), ("loss_out", ctypes.c_void_p),
                ("zncc_eps", ctypes.c_float)]


class drr_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double),
                ("tick", ctypes.c_int64)]


class drr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("ticks", ctypes.c_int64), ("pending", ctypes.c_int32),
                ("inflight", ctypes.c_int32), ("device_in_use", ctypes.c_size_t),
                ("device_budget", ctypes.c_size_t), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("gpu_busy_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32


def load(path: str = None):
    """Load libdrr.so and declare its signatures.  Raises if it is missing.
    DRR_LIBRARY in the environment names another build of the same ABI (the
    tests load the bounds-checked one this way)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if path is None:
            path = os.environ.get("DRR_LIBRARY") or LIB_PATH
        if not os.path.exists(path):
            raise FileNotFoundError(f"libdrr not built: {path} is missing (run paper_2208_12737_gb300.build.build())")
        lib = ctypes.CDLL(path)
        lib.drr_last_error.restype = ctypes.c_char_p
        lib.drr_last_error.argtypes = []
        lib.drr_version.restype = ctypes.c_char_p
        lib.drr_version.argtypes = []
        lib.drr_volume_create.argtypes = [_vp, _i32, _i32, _i32, _i32, _i32, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, ctypes.POINTER(drr_volume_options), _vp,
                                          ctypes.POINTER(_vp)]
        lib.drr_volume_destroy.argtypes = [_vp]
        lib.drr_volume_info.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(_i32), ctypes.POINTER(ctypes.c_float),
                                        ctypes.POINTER(ctypes.c_size_t)]
        lib.drr_render.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp, _vp]
        lib.drr_render_backward.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp, _vp, _vp, _vp]
        lib.drr_ray_setup.argtypes = [ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp]
        lib.drr_stream_check.argtypes = [_vp]
        lib.drr_count_segments.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp]
        lib.drr_profile_enable.argtypes = [_i32]
        lib.drr_profile_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64)]
        lib.drr_profile_reset.argtypes = []
        lib.drr_launch_count.argtypes = []
        lib.drr_server_create.argtypes = [ctypes.POINTER(drr_server_config), ctypes.POINTER(_vp)]
        lib.drr_server_submit.argtypes = [_vp, ctypes.POINTER(drr_request), ctypes.POINTER(ctypes.c_uint64)]
        lib.drr_server_wait.argtypes = [_vp, ctypes.c_uint64, _i32, ctypes.POINTER(drr_result)]
        lib.drr_server_cancel.argtypes = [_vp, ctypes.c_uint64]
        lib.drr_server_get_stats.argtypes = [_vp, ctypes.POINTER(drr_server_stats)]
        lib.drr_server_destroy.argtypes = [_vp]
        lib.drr_server_pause.argtypes = [_vp, _i32]
        lib.drr_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(_i32)]
        lib.drr_server_inject_device_status.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint32]
        lib.drr_serve_tick_layout.argtypes = [_i32, _vp, _vp, _vp, _vp, _vp]
        lib.drr_arena_create.argtypes = [ctypes.c_size_t, ctypes.c_size_t, ctypes.POINTER(_vp)]
        lib.drr_arena_alloc.argtypes = [_vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
        lib.drr_arena_free.argtypes = [_vp, ctypes.c_size_t]
        lib.drr_arena_in_use.argtypes = [_vp]
        lib.drr_arena_largest_free.argtypes = [_vp]
        lib.drr_arena_destroy.argtypes = [_vp]
        lib.drr_pose_grad_noalloc.argtypes = [ctypes.POINTER(drr_detector), _i32, _vp, _vp, _vp, _vp]
        lib.drr_zncc.argtypes = [_vp, _vp, _i32, _i32, ctypes.c_float, _vp, _vp, _vp]
        lib.drr_render_plain_fp32.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp]
        lib.drr_probe_l2_read.argtypes = [_vp, ctypes.c_size_t, _i32, _vp, _vp]
        lib.drr_geometry_grad.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _i32, _vp, _vp, _vp]
        lib.drr_loss_landscape.argtypes = [_vp, ctypes.POINTER(drr_detector), _vp, _vp, _i32, ctypes.c_float, _vp,
                                           _i32, _vp]
        lib.drr_adam_step.argtypes = [_vp, _vp, _vp, _vp, _i32, _i32, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp]
        for name in EXPORTS:
            if name not in ("drr_last_error", "drr_version"):
                getattr(lib, name).restype = ctypes.c_int
        lib.drr_launch_count.restype = ctypes.c_int64
        lib.drr_bounds_checked.argtypes = []
        lib.drr_bounds_checked.restype = ctypes.c_int32
        lib.drr_arena_in_use.restype = ctypes.c_size_t
        lib.drr_arena_largest_free.restype = ctypes.c_size_t
        _lib = lib
        return lib


def check(status: int):
    if status != 0:
        msg = _lib.drr_last_error().decode() if _lib is not None else ""
        raise DrrError(status, msg)


def detector(det) -> drr_detector:
    """From an inputs.Detector, a (sdr, H, W, dh, dw) tuple or a drr_detector."""
    if isinstance(det, drr_detector):
        return det
    if hasattr(det, "as_tuple"):
        det = det.as_tuple()
    sdr, H, W, dh, dw = det
    return drr_detector(float(sdr), int(H), int(W), float(dh), float(dw))


def _stream_ptr(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_ptr(t, dtype=None, shape=None, name="tensor", host_ok=False):
    """Address of a contiguous tensor the kernels may access: a CUDA tensor, or with
    host_ok a pinned CPU tensor (read or written in place across the host link)."""
    import torch
    if not isinstance(t, torch.Tensor) or not (t.is_cuda or (host_ok and t.is_pinned())):
        raise TypeError(f"{name} must be a CUDA torch.Tensor" + (" or a pinned CPU tensor" if host_ok else ""))
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


class Volume:
    """A device-resident CT volume (drr_volume_create / drr_volume_destroy).

    data: (nz, ny, nx) float32 attenuation (/mm) or int16 HU (``hu=True``), as a numpy
    array (uploaded from host) or a CUDA tensor.  spacing = (dx, dy, dz) mm.
    """

    def __init__(self, data, spacing, storage: str = "f32", hu: bool = False, mu_water: float = 0.02,
                 layout="default", stream=None):
        import torch
        lib = load()
        self._lib = lib
        self.handle = ctypes.c_void_p()
        src_dtype = DRR_I16_HU if hu else DRR_F32
        want = np.int16 if hu else np.float32
        if isinstance(data, torch.Tensor):
            tdt = torch.int16 if hu else torch.float32
            t = data.to(tdt).contiguous()
            if not t.is_cuda:
                t = t.cuda()
            ptr = ctypes.c_void_p(t.data_ptr())
            on_dev = 1
            shape = tuple(t.shape)
            self._keep = t
        else:
            arr = np.ascontiguousarray(data, dtype=want)
            ptr = arr.ctypes.data_as(ctypes.c_void_p)
            on_dev = 0
            shape = arr.shape
            self._keep = arr
        if len(shape) != 3:
            raise ValueError("volume must be (nz, ny, nx)")
        nz, ny, nx = shape
        lay = LAYOUT[layout] if isinstance(layout, str) else int(layout)
        opt = drr_volume_options(STORAGE[storage], float(mu_water) if hu else 0.0, lay)
        torch.cuda.init()
        check(lib.drr_volume_create(ptr, on_dev, src_dtype, nx, ny, nz, float(spacing[0]), float(spacing[1]),
                                    float(spacing[2]), ctypes.byref(opt), _stream_ptr(stream),
                                    ctypes.byref(self.handle)))
        self._keep = None
        self.shape_zyx = (nz, ny, nx)
        self.spacing = tuple(float(s) for s in spacing)
        self.storage = storage

    def info(self):
        dims = (_i32 * 3)()
        sp = (ctypes.c_float * 3)()
        st = _i32()
        sc = ctypes.c_float()
        nb = ctypes.c_size_t()
        check(self._lib.drr_volume_info(self.handle, dims, sp, ctypes.byref(st), ctypes.byref(sc), ctypes.byref(nb)))
        return dict(dims=tuple(dims), spacing=tuple(sp), storage=st.value, scale=sc.value, bytes=nb.value)

    def close(self):
        if self.handle is not None and self.handle.value:
            check(self._lib.drr_volume_destroy(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            if self.handle is not None and self.handle.value:
                self._lib.drr_volume_destroy(self.handle)
        except Exception:
            pass


def render(volume: Volume, det, poses, jacobian: bool = False, out=None, jac=None, stream=None):
    """E (B, H, W) float32; with jacobian=True also dE/d eta (B, 6, H, W).  poses, out and
    jac may be CUDA tensors or pinned CPU tensors (the kernels read and write those in
    place: keep a pinned tensor alive, and read it, only after the stream's work is done,
    e.g. after torch.cuda.synchronize()); outputs not given are allocated on the poses'
    device (the current CUDA device for pinned poses)."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses", host_ok=True)
    dev = poses.device if poses.is_cuda else torch.device("cuda", torch.cuda.current_device())
    if out is None:
        out = torch.empty((B, d.height, d.width), device=dev, dtype=torch.float32)
    op = _dev_ptr(out, torch.float32, (B, d.height, d.width), "out", host_ok=True)
    jp = None
    if jacobian:
        if jac is None:
            jac = torch.empty((B, 6, d.height, d.width), device=dev, dtype=torch.float32)
        jp = _dev_ptr(jac, torch.float32, (B, 6, d.height, d.width), "jac", host_ok=True)
    check(lib.drr_render(volume.handle, ctypes.byref(d), pp, B, op, jp, _stream_ptr(stream)))
    return (out, jac) if jacobian else out


def render_backward(volume: Volume, det, poses, grad_drr, jac=None, pose_grad: bool = True, grad_volume=None,
                    stream=None, grad_pose_out=None):
    """Returns dL/d eta (B, 6) (or None) and accumulates dL/dV into grad_volume if given.
    poses, grad_drr, jac and grad_pose_out (where dL/d eta is written, else a new tensor
    on the poses' device) may be pinned CPU tensors; grad_volume must be on the device."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses", host_ok=True)
    gp = _dev_ptr(grad_drr, torch.float32, (B, d.height, d.width), "grad_drr", host_ok=True)
    jp = _dev_ptr(jac, torch.float32, (B, 6, d.height, d.width), "jac", host_ok=True) if jac is not None else None
    gpose = None
    if pose_grad:
        dev = poses.device if poses.is_cuda else torch.device("cuda", torch.cuda.current_device())
        gpose = grad_pose_out if grad_pose_out is not None else torch.empty((B, 6), device=dev, dtype=torch.float32)
    gpp = _dev_ptr(gpose, torch.float32, (B, 6), "grad_pose", host_ok=True) if pose_grad else None
    gvp = _dev_ptr(grad_volume, torch.float32, volume.shape_zyx, "grad_volume") if grad_volume is not None else None
    check(lib.drr_render_backward(volume.handle, ctypes.byref(d), pp, B, gp, jp, gpp, gvp, _stream_ptr(stream)))
    return gpose


def ray_setup(det, poses, stream=None):
    """Source and pixel centres (B, H, W, 6) = (sx, sy, sz, px, py, pz) from the ray-setup kernel."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses")
    rays = torch.empty((B, d.height, d.width, 6), device=poses.device, dtype=torch.float32)
    check(lib.drr_ray_setup(ctypes.byref(d), pp, B, ctypes.c_void_p(rays.data_ptr()), _stream_ptr(stream)))
    return rays


def count_segments(volume: Volume, det, poses, stream=None):
    """Per-ray Siddon segment counts (B, H, W) int32."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses")
    out = torch.empty((B, d.height, d.width), device=poses.device, dtype=torch.int32)
    check(lib.drr_count_segments(volume.handle, ctypes.byref(d), pp, B, ctypes.c_void_p(out.data_ptr()),
                                 _stream_ptr(stream)))
    return out


def profile_enable(on: bool = True):
    check(load().drr_profile_enable(1 if on else 0))


def profile_reset():
    check(load().drr_profile_reset())


def profile_read(kernel: str):
    """(total device ms, launches) of one kernel since the last reset."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    check(load().drr_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def launch_count() -> int:
    return int(load().drr_launch_count())


def zncc(moving, fixed, eps: float = 1e-8, grad: bool = True, stream=None):
    """Negative ZNCC per image pair (B,) and, with grad=True, d loss / d moving (same shape)."""
    import torch
    lib = load()
    B = moving.shape[0]
    npix = moving[0].numel()
    mp = _dev_ptr(moving, torch.float32, name="moving")
    fp = _dev_ptr(fixed, torch.float32, tuple(moving.shape), "fixed")
    loss = torch.empty((B,), device=moving.device, dtype=torch.float32)
    g = torch.empty_like(moving) if grad else None
    check(lib.drr_zncc(mp, fp, B, npix, float(eps), ctypes.c_void_p(loss.data_ptr()),
                       ctypes.c_void_p(g.data_ptr()) if grad else None, _stream_ptr(stream)))
    return (loss, g) if grad else loss


def geometry_grad(volume: Volume, det, poses, grad_drr, stream=None):
    """dL/d(sdr, delta_h, delta_w) per pose (B, 3): the gradient with respect to the detector
    parameters for an upstream gradient grad_drr (B, H, W)."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses")
    gp = _dev_ptr(grad_drr, torch.float32, (B, d.height, d.width), "grad_drr")
    out = torch.empty((B, 3), device=poses.device, dtype=torch.float32)
    check(lib.drr_geometry_grad(volume.handle, ctypes.byref(d), pp, B, gp, ctypes.c_void_p(out.data_ptr()),
                                _stream_ptr(stream)))
    return out


def render_plain_fp32(volume: Volume, det, poses, out=None, stream=None):
    """The comparison baseline: the plain FP32 forward walk, (B, H, W)."""
    import torch
    lib = load()
    d = detector(det)
    B = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (B, 6), "poses")
    if out is None:
        out = torch.empty((B, d.height, d.width), device=poses.device, dtype=torch.float32)
    op = _dev_ptr(out, torch.float32, (B, d.height, d.width), "out")
    check(lib.drr_render_plain_fp32(volume.handle, ctypes.byref(d), pp, B, op, _stream_ptr(stream)))
    return out


def probe_l2_read(buf, reps: int, sink, stream=None):
    """Stream a device buffer (uint8/float tensor, 16-byte aligned) reps times from L2."""
    lib = load()
    check(lib.drr_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(), int(reps),
                                ctypes.c_void_p(sink.data_ptr()), _stream_ptr(stream)))


def loss_landscape(volume: Volume, det, fixed, poses, eps: float = 1e-8, chunk: int = 0, out=None, stream=None):
    """-ZNCC(DRR(pose_i), fixed) for each of N poses (N,), the landscape study of Sec. 3.2.
    fixed: (H, W) float32 on the device; poses: (N, 6) float32 on the device."""
    import torch
    lib = load()
    d = detector(det)
    N = poses.shape[0]
    pp = _dev_ptr(poses, torch.float32, (N, 6), "poses")
    fp = _dev_ptr(fixed, torch.float32, (d.height, d.width), "fixed")
    if out is None:
        out = torch.empty((N,), device=poses.device, dtype=torch.float32)
    op = _dev_ptr(out, torch.float32, (N,), "out")
    check(lib.drr_loss_landscape(volume.handle, ctypes.byref(d), fp, pp, N, float(eps), op, int(chunk),
                                 _stream_ptr(stream)))
    return out


def adam_step(params, grads, m, v, step: int, lr_rot: float, lr_trans: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, stream=None):
    """In-place Adam update of (B, 6) pose parameters (separate rotation / translation rates)."""
    import torch
    lib = load()
    B = params.shape[0]
    ptrs = [_dev_ptr(t, torch.float32, (B, 6), n) for t, n in ((params, "params"), (grads, "grads"), (m, "m"),
                                                                (v, "v"))]
    check(lib.drr_adam_step(*ptrs, B, int(step), float(lr_rot), float(lr_trans), float(beta1), float(beta2),
                            float(eps), _stream_ptr(stream)))


def register(volume: Volume, det, fixed, init_poses, steps: int = 200, lr_rot: float = 1e-2, lr_trans: float = 1.0,
             tol: float = -0.999, eps: float = 1e-8):
    """Gradient registration (Sec. 3.2): minimise -ZNCC(DRR(pose), fixed) over the 6 pose parameters
    of B independent problems with Adam.  Every step runs on the GPU: fused forward + Jacobian,
    ZNCC loss and gradient, the pose-gradient reduction and the Adam update.

    Returns (final poses (B, 6), loss history (steps, B), first step at which each problem reached
    loss < tol or -1), all on the host."""
    import torch
    d = detector(det)
    poses = init_poses.clone().contiguous().float()
    B = poses.shape[0]
    m = torch.zeros_like(poses)
    v = torch.zeros_like(poses)
    E = torch.empty((B, d.height, d.width), device=poses.device)
    J = torch.empty((B, 6, d.height, d.width), device=poses.device)
    hist = torch.empty((steps, B), device=poses.device)
    for t in range(steps):
        render(volume, d, poses, jacobian=True, out=E, jac=J)
        loss, g = zncc(E, fixed, eps)
        hist[t].copy_(loss)
        G = render_backward(volume, d, poses, g, jac=J)
        adam_step(poses, G, m, v, t + 1, lr_rot, lr_trans)
    h = hist.cpu().numpy()
    ok = h < tol
    first = np.where(ok.any(axis=0), ok.argmax(axis=0), -1)
    return poses.cpu().numpy(), h, first


def stream_check(stream=None):
    lib = load()
    check(lib.drr_stream_check(_stream_ptr(stream)))


class Arena:
    """The serving loop's host-side offset allocator (no CUDA calls)."""

    def __init__(self, capacity: int, align: int = 256):
        self._lib = load()
        self.h = ctypes.c_void_p()
        check(self._lib.drr_arena_create(capacity, align, ctypes.byref(self.h)))

    def alloc(self, nbytes: int) -> int:
        off = ctypes.c_size_t()
        check(self._lib.drr_arena_alloc(self.h, nbytes, ctypes.byref(off)))
        return off.value

    def free(self, offset: int):
        check(self._lib.drr_arena_free(self.h, offset))

    def in_use(self) -> int:
        return int(self._lib.drr_arena_in_use(self.h))

    def largest_free(self) -> int:
        return int(self._lib.drr_arena_largest_free(self.h))

    def close(self):
        if self.h.value:
            self._lib.drr_arena_destroy(self.h)
            self.h = ctypes.c_void_p()

    __del__ = close


class Ticket:
    """A submitted request.  Its host buffers (and its volume) are held by the server
    object until wait() returns the request's result, so dropping a ticket that was
    never waited for cannot free memory the request loop still writes into."""

    def __init__(self, server, tid, out, grad_pose, keep, loss=None):
        self.server = server
        self.id = tid
        self.out = out
        self.grad_pose = grad_pose
        self.loss = loss
        self._keep = keep
        self.result = None

    def wait(self, timeout_ms: int = -1):
        res = drr_result()
        st = self.server._lib.drr_server_wait(self.server.h, self.id, int(timeout_ms), ctypes.byref(res))
        if st == 4:  # DRR_ERR_TIMEOUT: ticket still valid
            raise DrrError(st, self.server._lib.drr_last_error().decode())
        self.result = res
        self._keep = None
        self.server._live.pop(self.id, None)  # the request is finished and released
        if st != 0:
            raise DrrError(st, self.server._lib.drr_last_error().decode())
        if self.loss is not None:
            return self.out, self.grad_pose, self.loss
        return self.out, self.grad_pose

    def cancel(self):
        check(self.server._lib.drr_server_cancel(self.server.h, self.id))

    def poll(self) -> str:
        """'queued', 'running' or 'done', without waiting (the ticket is kept)."""
        st = _i32()
        check(self.server._lib.drr_server_poll(self.server.h, self.id, ctypes.byref(st)))
        return ("queued", "running", "done")[st.value]

    def inject_device_status(self, bits: int):
        """Test hook: make this queued request's device status word start with `bits`
        set, so the server reports DRR_ERR_DEVICE for it after its tick."""
        check(self.server._lib.drr_server_inject_device_status(self.server.h, self.id, int(bits)))


class Server:
    """Continuous-batching request loop (drr_server_*): host buffers in, host buffers out."""

    def __init__(self, device_budget: int = 512 << 20, host_budget: int = 0, max_inflight: int = 64,
                 max_tick_poses: int = 4096, use_cuda_graph: bool = True, device: int = -1,
                 max_tick_work: int = 0, plain_fp32_baseline: bool = False, tick_depth: int = 0,
                 spin_poll_us: int = 0):
        self._lib = load()
        cfg = drr_server_config(device_budget, host_budget, max_inflight, max_tick_poses,
                                1 if use_cuda_graph else 0, device, int(max_tick_work),
                                1 if plain_fp32_baseline else 0, int(tick_depth), int(spin_poll_us))
        self.h = ctypes.c_void_p()
        self._live = {}  # ticket id -> the buffers and volume of a request not yet waited for
        check(self._lib.drr_server_create(ctypes.byref(cfg), ctypes.byref(self.h)))

    def submit(self, volume: Volume, det, poses, grad=None, fixed=None, eps: float = 1e-8, out=None) -> Ticket:
        """Queue a render (grad=None, fixed=None), a render with the pose gradient of the
        upstream gradient `grad`, or a registration step against the fixed images `fixed`
        (loss -ZNCC and its pose gradient; wait() then returns (E, dL/d eta, loss)).
        `out`: a C-contiguous float32 (B, H, W) array to receive E (reused buffers spare the
        server's copy the page faults of fresh memory), else a new one."""
        d = detector(det)
        poses = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 6)
        B = poses.shape[0]
        if out is None:
            out = np.empty((B, d.height, d.width), np.float32)
        elif (not isinstance(out, np.ndarray) or out.dtype != np.float32 or out.shape != (B, d.height, d.width)
              or not out.flags.c_contiguous or not out.flags.writeable):
            raise ValueError(f"out must be a writeable C-contiguous float32 array of shape {(B, d.height, d.width)}")
        keep = [poses, out]
        req = drr_request(volume.handle, d, B, poses.ctypes.data, None, out.ctypes.data, None)
        gpose = None
        if grad is not None:
            grad = np.ascontiguousarray(grad, dtype=np.float32).reshape(B, d.height, d.width)
            gpose = np.empty((B, 6), np.float32)
            keep += [grad, gpose]
            req.grad_drr = grad.ctypes.data
            req.grad_pose_out = gpose.ctypes.data
        loss = None
        if fixed is not None:
            fixed = np.ascontiguousarray(fixed, dtype=np.float32).reshape(B, d.height, d.width)
            gpose = np.empty((B, 6), np.float32)
            loss = np.empty(B, np.float32)
            keep += [fixed, gpose, loss]
            req.fixed = fixed.ctypes.data
            req.grad_pose_out = gpose.ctypes.data
            req.loss_out = loss.ctypes.data
            req.zncc_eps = float(eps)
        tid = ctypes.c_uint64()
        check(self._lib.drr_server_submit(self.h, ctypes.byref(req), ctypes.byref(tid)))
        self._live[tid.value] = keep + [volume]
        return Ticket(self, tid.value, out, gpose, keep, loss)

    def pause(self, paused: bool = True):
        """Stop (or resume) admitting queued requests; running ticks finish."""
        check(self._lib.drr_server_pause(self.h, 1 if paused else 0))

    def stats(self) -> dict:
        st = drr_server_stats()
        check(self._lib.drr_server_get_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in drr_server_stats._fields_}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def close(self):
        if self.h is not None and self.h.value:
            check(self._lib.drr_server_destroy(self.h))  # every request has finished or been cancelled
            self.h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _autograd():
    import torch

    class DRRFunction(torch.autograd.Function):
        """poses (B, 6) -> DRR (B, H, W); backward gives dL/d poses via the fused Jacobian."""

        @staticmethod
        def forward(ctx, poses, volume, det):
            E, J = render(volume, det, poses.contiguous(), jacobian=True)
            ctx.volume = volume
            ctx.det = det
            ctx.save_for_backward(poses, J)
            return E

        @staticmethod
        def backward(ctx, grad):
            poses, J = ctx.saved_tensors
            g = render_backward(ctx.volume, ctx.det, poses.contiguous(), grad.contiguous().float(), jac=J)
            return g.to(poses.device), None, None  # pinned host poses get a host gradient

    class DRRVolumeFunction(torch.autograd.Function):
        """(mu (nz, ny, nx), poses (B, 6)) -> DRR (B, H, W).  E is linear in the volume
        (Eq. 2), so dL/d mu is the back-projection of dL/dE (the transpose of the forward
        map); dL/d poses comes from the fused Jacobian.  Each is computed only if needed."""

        @staticmethod
        def forward(ctx, mu, poses, spacing, det):
            vol = Volume(mu.detach(), spacing)  # device-to-device copy into the padded layout
            poses = poses.contiguous()
            if ctx.needs_input_grad[1]:
                E, J = render(vol, det, poses, jacobian=True)
            else:
                E, J = render(vol, det, poses), None
            ctx.volume = vol
            ctx.det = det
            ctx.save_for_backward(poses, J)
            return E

        @staticmethod
        def backward(ctx, grad):
            poses, J = ctx.saved_tensors
            g = grad.contiguous().float()
            g_mu = g_pose = None
            if ctx.needs_input_grad[1]:
                g_pose = render_backward(ctx.volume, ctx.det, poses, g, jac=J).to(poses.device)
            if ctx.needs_input_grad[0]:
                g_mu = torch.zeros(ctx.volume.shape_zyx, device=g.device, dtype=torch.float32)
                render_backward(ctx.volume, ctx.det, poses, g, pose_grad=False, grad_volume=g_mu)
            return g_mu, g_pose, None, None

    return DRRFunction, DRRVolumeFunction


_fn = None
_vfn = None


def drr(volume: Volume, det, poses):
    """Differentiable DRR: E = drr(volume, det, poses) with gradients to poses."""
    global _fn, _vfn
    if _fn is None:
        _fn, _vfn = _autograd()
    return _fn.apply(poses, volume, det)


def drr_volume(mu, spacing, det, poses):
    """Differentiable DRR of a volume held as a tensor: E = drr_volume(mu, spacing, det, poses)
    with mu a (nz, ny, nx) FP32 CUDA tensor of attenuation (/mm); gradients flow to mu (by
    the back-projection) and to poses, whichever requires them.  The volume is copied into
    the library's padded layout on every call."""
    global _fn, _vfn
    if _fn is None:
        _fn, _vfn = _autograd()
    return _vfn.apply(mu, poses, tuple(float(x) for x in spacing), det)


class DRR:
    """Callable renderer bound to a volume and detector: ``DRR(vol, det)(poses)``."""

    def __init__(self, volume: Volume, det):
        self.volume = volume
        self.det = det

    def __call__(self, poses):
        return drr(self.volume, self.det, poses)
