"""FP64 CPU oracle for Siddon DRR rendering (arXiv 2208.12737, Eq. 1-4, Sec. 2.3-2.4).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously-correct
reference the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  It shares no code with the CUDA library and the
library never calls it.

The arithmetic lives in ``siddon_oracle.c`` (double precision, OpenMP over
rays); this module is argument marshalling through ctypes plus the pose
helpers.  ``build()`` compiles the C file with gcc.

Pinned by the CPU tests in ``tests/test_oracle_*.py`` against closed forms,
an exact per-voxel brute force, midpoint sampling, hand-worked examples in
``tests/golden/`` and central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i16p = ctypes.POINTER(ctypes.c_int16)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the .so path."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC]
    try:
        subprocess.run(base + ["-fopenmp", "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.oracle_pose_matrix.argtypes = [_dp, _dp, _dp]
        lib.oracle_pose_matrix.restype = None
        lib.oracle_ray_endpoints.argtypes = [_dp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                             ctypes.c_int32, _dp, _dp]
        lib.oracle_ray_endpoints.restype = None
        for name in ("oracle_siddon_ray",):
            fn = getattr(lib, name)
            fn.argtypes = [_ip, _dp, _fp, _dp, _dp, _dp, _dp]
            fn.restype = ctypes.c_double
        for name in ("oracle_brute_ray", "oracle_siddon_total_length"):
            fn = getattr(lib, name)
            fn.argtypes = [_ip, _dp, _fp, _dp, _dp]
            fn.restype = ctypes.c_double
        lib.oracle_sample_ray.argtypes = [_ip, _dp, _fp, _dp, _dp, ctypes.c_int64]
        lib.oracle_sample_ray.restype = ctypes.c_double
        lib.oracle_render.argtypes = [_ip, _dp, _fp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_double, ctypes.c_double, _fp, ctypes.c_int32, _i64p,
                                      ctypes.c_int64, _dp, _dp, _dp, ctypes.c_int32]
        lib.oracle_render.restype = ctypes.c_int
        lib.oracle_pose_grad.argtypes = [_ip, _dp, _fp, ctypes.c_double, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_double, _fp,
                                         ctypes.c_int32, _dp, _dp, ctypes.c_int32]
        lib.oracle_pose_grad.restype = ctypes.c_int
        lib.oracle_backproject.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_double, ctypes.c_double, _fp, ctypes.c_int32,
                                           _dp, _dp]
        lib.oracle_backproject.restype = ctypes.c_int
        lib.oracle_backproject_ray.argtypes = [_ip, _dp, _dp, _dp, ctypes.c_double, _dp]
        lib.oracle_backproject_ray.restype = ctypes.c_int
        lib.oracle_voxel_adjoint.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.c_double, ctypes.c_double, _fp, ctypes.c_int32, _dp,
                                             _i64p, ctypes.c_int64, _dp, _dp]
        lib.oracle_voxel_adjoint.restype = ctypes.c_int
        lib.oracle_count_segments.argtypes = [_ip, _dp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_double, _fp, ctypes.c_int32, _i64p,
                                              ctypes.c_int64, _ip]
        lib.oracle_count_segments.restype = ctypes.c_int
        lib.oracle_hu_to_mu.argtypes = [_i16p, ctypes.c_int64, ctypes.c_double, _dp]
        lib.oracle_hu_to_mu.restype = None
        for name in ("oracle_round_bf16", "oracle_round_f16"):
            fn = getattr(lib, name)
            fn.argtypes = [_fp, ctypes.c_int64, _fp]
            fn.restype = None
        _lib = lib
        return lib


def _c(arr, dtype):
    return np.ascontiguousarray(arr, dtype=dtype)


def _ptr(arr, ctype):
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


class Volume:
    """A CT volume as the oracle sees it: float32 (nz, ny, nx), x fastest, spacing (dx, dy, dz) mm."""

    def __init__(self, data, spacing):
        data = _c(data, np.float32)
        if data.ndim != 3:
            raise ValueError("volume must be (nz, ny, nx)")
        self.data = data
        self.n = np.array([data.shape[2], data.shape[1], data.shape[0]], dtype=np.int32)
        self.delta = np.array(spacing, dtype=np.float64).reshape(3)

    def _args(self):
        return _ptr(self.n, ctypes.c_int32), _ptr(self.delta, ctypes.c_double), _ptr(self.data, ctypes.c_float)


def pose_matrix(eta):
    """R = Rz(eta0) Ry(eta1) Rx(eta2) and dR/d eta_j (Sec. 2.4 reading)."""
    lib = _load()
    e = _c(eta, np.float64)[:3].copy()
    R = np.zeros(9)
    dR = np.zeros(27)
    lib.oracle_pose_matrix(_ptr(e, ctypes.c_double), _ptr(R, ctypes.c_double), _ptr(dR, ctypes.c_double))
    return R.reshape(3, 3), dR.reshape(3, 3, 3)


def ray_endpoints(pose, sdr, H, W, dh, dw, h, w):
    """World-space source s and pixel centre p for one pose (Sec. 2.4)."""
    lib = _load()
    e = _c(pose, np.float64).reshape(6)
    s = np.zeros(3)
    p = np.zeros(3)
    lib.oracle_ray_endpoints(_ptr(e, ctypes.c_double), float(sdr), int(H), int(W), float(dh), float(dw),
                             int(h), int(w), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double))
    return s, p


def siddon_ray(vol: Volume, s, p, grad: bool = False):
    """E = |p-s| sum (a_{m+1}-a_m) V[mid] (Eq. 2); with grad=True also dE/ds, dE/dp."""
    lib = _load()
    s = _c(s, np.float64)
    p = _c(p, np.float64)
    if grad:
        gs = np.zeros(3)
        gp = np.zeros(3)
        E = lib.oracle_siddon_ray(*vol._args(), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double),
                                  _ptr(gs, ctypes.c_double), _ptr(gp, ctypes.c_double))
        return E, gs, gp
    return lib.oracle_siddon_ray(*vol._args(), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double), None, None)


def siddon_total_length(vol: Volume, s, p):
    """|p-s| times the sum of all Siddon segment lengths (the clipped chord)."""
    lib = _load()
    s = _c(s, np.float64)
    p = _c(p, np.float64)
    return lib.oracle_siddon_total_length(*vol._args(), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double))


def brute_ray(vol: Volume, s, p):
    """Exact per-voxel brute force of Eq. (1) for a piecewise-constant volume."""
    lib = _load()
    s = _c(s, np.float64)
    p = _c(p, np.float64)
    return lib.oracle_brute_ray(*vol._args(), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double))


def sample_ray(vol: Volume, s, p, nsamples: int):
    """Midpoint-rule sampling of Eq. (1) with nsamples points."""
    lib = _load()
    s = _c(s, np.float64)
    p = _c(p, np.float64)
    return lib.oracle_sample_ray(*vol._args(), _ptr(s, ctypes.c_double), _ptr(p, ctypes.c_double),
                                 int(nsamples))


def render(vol: Volume, det, poses, pixels=None, jacobian: bool = False, threads: int = 0,
           geometry: bool = False):
    """DRR for every pose: (B, H, W) float64, or (B, len(pixels)) for a flat pixel list.

    det = (sdr, H, W, dh, dw).  With jacobian=True also returns dE/d(rz,ry,rx,tx,ty,tz)
    per ray: (B, H, W, 6) or (B, npix, 6); with geometry=True (after it) dE/d(sdr, dh, dw)
    per ray: (B, H, W, 3) or (B, npix, 3).
    """
    lib = _load()
    sdr, H, W, dh, dw = det
    poses = _c(poses, np.float32).reshape(-1, 6)
    B = poses.shape[0]
    if pixels is None:
        npix = H * W
        pix_ptr = None
    else:
        pixels = _c(pixels, np.int64).reshape(-1)
        npix = pixels.size
        pix_ptr = _ptr(pixels, ctypes.c_int64)
    out = np.zeros((B, npix))
    jac = np.zeros((B, npix, 6)) if jacobian else None
    geo = np.zeros((B, npix, 3)) if geometry else None
    lib.oracle_render(*vol._args(), float(sdr), int(H), int(W), float(dh), float(dw),
                      _ptr(poses, ctypes.c_float), int(B), pix_ptr, int(npix), _ptr(out, ctypes.c_double),
                      _ptr(jac, ctypes.c_double) if jacobian else None,
                      _ptr(geo, ctypes.c_double) if geometry else None, int(threads))
    if pixels is None:
        out = out.reshape(B, H, W)
        if jacobian:
            jac = jac.reshape(B, H, W, 6)
        if geometry:
            geo = geo.reshape(B, H, W, 3)
    res = (out,) + ((jac,) if jacobian else ()) + ((geo,) if geometry else ())
    return res if len(res) > 1 else out


def geometry_grad(vol: Volume, det, poses, grad_out, threads: int = 0):
    """dL/d(sdr, dh, dw) per pose: sum over pixels of grad_out * dE/d(sdr, dh, dw), (B, 3)."""
    _, geo = render(vol, det, poses, geometry=True, threads=threads)
    g = np.asarray(grad_out, np.float64).reshape(geo.shape[:-1])
    return np.einsum("bhw,bhwk->bk", g, geo)


def pose_grad(vol: Volume, det, poses, grad_out, threads: int = 0):
    """sum_{h,w} grad_out[b,h,w] * dE[b,h,w]/d eta  -> (B, 6) float64."""
    lib = _load()
    sdr, H, W, dh, dw = det
    poses = _c(poses, np.float32).reshape(-1, 6)
    B = poses.shape[0]
    g = _c(grad_out, np.float64).reshape(B, H, W)
    out = np.zeros((B, 6))
    rc = lib.oracle_pose_grad(*vol._args(), float(sdr), int(H), int(W), float(dh), float(dw),
                              _ptr(poses, ctypes.c_float), int(B), _ptr(g, ctypes.c_double),
                              _ptr(out, ctypes.c_double), int(threads))
    if rc != 0:
        raise MemoryError("oracle_pose_grad: allocation failed")
    return out


def backproject(shape_zyx, spacing, det, poses, grad_out):
    """Transpose of V -> E: (nz, ny, nx) float64 volume gradient."""
    lib = _load()
    sdr, H, W, dh, dw = det
    nz, ny, nx = shape_zyx
    n = np.array([nx, ny, nz], dtype=np.int32)
    delta = np.array(spacing, dtype=np.float64)
    poses = _c(poses, np.float32).reshape(-1, 6)
    B = poses.shape[0]
    g = _c(grad_out, np.float64).reshape(B, H, W)
    out = np.zeros((nz, ny, nx))
    lib.oracle_backproject(_ptr(n, ctypes.c_int32), _ptr(delta, ctypes.c_double), float(sdr), int(H), int(W),
                           float(dh), float(dw), _ptr(poses, ctypes.c_float), int(B), _ptr(g, ctypes.c_double),
                           _ptr(out, ctypes.c_double))
    return out


def backproject_ray(shape_zyx, spacing, s, p, g: float = 1.0):
    """Transpose of V -> E for the single ray s -> p: (nz, ny, nx) float64, g |p - s| times
    each Siddon segment's length (in alpha) in its voxel (Eq. 2 read as linear in V)."""
    lib = _load()
    nz, ny, nx = shape_zyx
    n = np.array([nx, ny, nz], dtype=np.int32)
    delta = np.array(spacing, dtype=np.float64)
    s = _c(s, np.float64)
    p = _c(p, np.float64)
    out = np.zeros((nz, ny, nx))
    lib.oracle_backproject_ray(_ptr(n, ctypes.c_int32), _ptr(delta, ctypes.c_double), _ptr(s, ctypes.c_double),
                               _ptr(p, ctypes.c_double), float(g), _ptr(out, ctypes.c_double))
    return out


def voxel_adjoint(shape_zyx, spacing, det, poses, grad_out, voxels):
    """The transpose of V -> E at the voxels with linear indices `voxels`
    (i + nx (j + ny k)), by its definition: the sum over every ray of
    g |p - s| times the ray's clipped chord (in alpha) through the voxel's box,
    slab method per voxel as in the brute force of Eq. (1).  Returns the values
    and the same sums with |g| (their rounding-error scale)."""
    lib = _load()
    sdr, H, W, dh, dw = det
    nz, ny, nx = shape_zyx
    n = np.array([nx, ny, nz], dtype=np.int32)
    delta = np.array(spacing, dtype=np.float64)
    poses = _c(poses, np.float32).reshape(-1, 6)
    B = poses.shape[0]
    g = _c(grad_out, np.float64).reshape(B, H, W)
    vox = _c(voxels, np.int64).reshape(-1)
    out = np.zeros(vox.size)
    out_abs = np.zeros(vox.size)
    if lib.oracle_voxel_adjoint(_ptr(n, ctypes.c_int32), _ptr(delta, ctypes.c_double), float(sdr), int(H), int(W),
                                float(dh), float(dw), _ptr(poses, ctypes.c_float), int(B), _ptr(g, ctypes.c_double),
                                _ptr(vox, ctypes.c_int64), int(vox.size), _ptr(out, ctypes.c_double),
                                _ptr(out_abs, ctypes.c_double)) != 0:
        raise MemoryError("oracle_voxel_adjoint: allocation failed")
    return out, out_abs


def count_segments(shape_zyx, spacing, det, poses, pixels=None):
    """Segments per ray (consecutive pairs of the sorted crossing list, Eq. 4): (B, H, W) or (B, npix) int32."""
    lib = _load()
    sdr, H, W, dh, dw = det
    nz, ny, nx = shape_zyx
    n = np.array([nx, ny, nz], dtype=np.int32)
    delta = np.array(spacing, dtype=np.float64)
    poses = _c(poses, np.float32).reshape(-1, 6)
    B = poses.shape[0]
    if pixels is None:
        npix, pix_ptr = H * W, None
    else:
        pixels = _c(pixels, np.int64).reshape(-1)
        npix, pix_ptr = pixels.size, _ptr(pixels, ctypes.c_int64)
    out = np.zeros((B, npix), np.int32)
    lib.oracle_count_segments(_ptr(n, ctypes.c_int32), _ptr(delta, ctypes.c_double), float(sdr), int(H), int(W),
                              float(dh), float(dw), _ptr(poses, ctypes.c_float), int(B), pix_ptr, int(npix),
                              _ptr(out, ctypes.c_int32))
    return out.reshape(B, H, W) if pixels is None else out


def hu_to_mu(hu, mu_water: float):
    """mu = max(0, mu_water (1 + HU/1000)), float64."""
    lib = _load()
    hu = _c(hu, np.int16)
    out = np.zeros(hu.shape)
    lib.oracle_hu_to_mu(_ptr(hu, ctypes.c_int16), int(hu.size), float(mu_water), _ptr(out, ctypes.c_double))
    return out


def round_bf16(x):
    """Round-to-nearest-even to bfloat16, returned as float32."""
    lib = _load()
    x = _c(x, np.float32)
    out = np.empty_like(x)
    lib.oracle_round_bf16(_ptr(x, ctypes.c_float), int(x.size), _ptr(out, ctypes.c_float))
    return out


def round_f16(x):
    """Round-to-nearest-even to IEEE half (with subnormals), returned as float32."""
    lib = _load()
    x = _c(x, np.float32)
    out = np.empty_like(x)
    lib.oracle_round_f16(_ptr(x, ctypes.c_float), int(x.size), _ptr(out, ctypes.c_float))
    return out


def f16_scale(max_value: float) -> float:
    """Power-of-two scale applied before half-precision storage: brings the
    largest value into [2^13, 2^14) so small attenuations stay normal halves.
    A volume whose maximum is 0 gets scale 1."""
    if not (max_value > 0.0):
        return 1.0
    _, e = np.frexp(np.float64(max_value))  # max = m 2^e, m in [0.5, 1)
    return float(2.0 ** (14 - int(e)))


# ---------------------------------------------------------------------------
# Registration loss (Sec. 3.2): negative zero-normalised cross-correlation.
# Population statistics; I^ = (I - mean I) / (std I + eps), F^ likewise.
# ---------------------------------------------------------------------------

def zncc_loss(moving, fixed, eps: float = 1e-8):
    """-mean(I^ F^) per image; moving, fixed: (B, ...) -> (B,) float64."""
    I = np.asarray(moving, np.float64).reshape(len(moving), -1)
    F = np.asarray(fixed, np.float64).reshape(len(fixed), -1)
    Ic = I - I.mean(axis=1, keepdims=True)
    Fc = F - F.mean(axis=1, keepdims=True)
    Ih = Ic / (np.sqrt((Ic ** 2).mean(axis=1, keepdims=True)) + eps)
    Fh = Fc / (np.sqrt((Fc ** 2).mean(axis=1, keepdims=True)) + eps)
    return -(Ih * Fh).mean(axis=1)


def loss_landscape(vol: Volume, det, fixed, poses, eps: float = 1e-8, threads: int = 0):
    """-ZNCC between the DRR at each pose and one fixed image (the loss-landscape study,
    Sec. 3.2): render every pose (Eq. 2), then zncc_loss against the same fixed image."""
    poses = np.asarray(poses, np.float32).reshape(-1, 6)
    E = render(vol, det, poses, threads=threads)
    F = np.broadcast_to(np.asarray(fixed, np.float64), E.shape)
    return zncc_loss(E, F, eps)


def zncc_loss_grad(moving, fixed, eps: float = 1e-8):
    """d zncc_loss / d moving, by differentiating the definition term by term
    (mean, centring, population std, normalisation, mean of the product)."""
    shape = np.shape(moving)
    I = np.asarray(moving, np.float64).reshape(shape[0], -1)
    F = np.asarray(fixed, np.float64).reshape(shape[0], -1)
    N = I.shape[1]
    Ic = I - I.mean(axis=1, keepdims=True)
    s = np.sqrt((Ic ** 2).mean(axis=1, keepdims=True))
    Fc = F - F.mean(axis=1, keepdims=True)
    Fh = Fc / (np.sqrt((Fc ** 2).mean(axis=1, keepdims=True)) + eps)
    # loss = -(1/N) sum_i Fh_i Ic_i / (s + eps)
    # d Ic_i / d I_j = delta_ij - 1/N ;  d s / d I_j = Ic_j / (N s)
    dL_dIc = -Fh / (N * (s + eps))                                  # through the numerator
    dL_ds = ((Fh * Ic).sum(axis=1, keepdims=True)) / (N * (s + eps) ** 2)
    g = dL_dIc - dL_dIc.mean(axis=1, keepdims=True)                 # chain through the centring
    g = g + dL_ds * np.where(s > 0, Ic / (N * np.where(s > 0, s, 1.0)), 0.0)
    return g.reshape(shape)
