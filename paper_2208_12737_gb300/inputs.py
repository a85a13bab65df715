"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module only synthesises inputs (phantom volumes, poses, upstream
gradients); it contains none of the DRR arithmetic.  The paper's chest CT
(Sec. 3, 360 x 360 x 332.5 mm) is not available, so seeded ellipsoid phantoms
of the same shape and spacing stand in for it.

All generators use ``numpy.random.default_rng(seed)`` (PCG64) and return
numpy arrays; volumes are (nz, ny, nx), x fastest.
"""
from __future__ import annotations

import dataclasses

import numpy as np

DEG = np.pi / 180.0


@dataclasses.dataclass(frozen=True)
class Detector:
    """Source-to-detector distance (mm), detector rows/cols and pixel spacing (mm)."""

    sdr: float
    height: int
    width: int
    delta_h: float
    delta_w: float

    def as_tuple(self):
        return (self.sdr, self.height, self.width, self.delta_h, self.delta_w)


def _rotation(rng) -> np.ndarray:
    """A random orientation for an ellipsoid (input synthesis only)."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _paint_ellipsoid(vol, spacing, centre_mm, semi_mm, rot, value, mode="add"):
    """Add (or set) `value` inside an ellipsoid, voxel centres tested, bbox-restricted.

    `rot` has the ellipsoid axes as columns (world = rot @ local)."""
    nz, ny, nx = vol.shape
    dx, dy, dz = spacing
    ext = np.array([nx * dx, ny * dy, nz * dz])
    b = -0.5 * ext
    r = float(np.max(semi_mm))
    lo = np.floor((np.asarray(centre_mm) - r - b) / np.array([dx, dy, dz])).astype(int)
    hi = np.ceil((np.asarray(centre_mm) + r - b) / np.array([dx, dy, dz])).astype(int)
    lo = np.clip(lo, 0, [nx, ny, nz])
    hi = np.clip(hi, 0, [nx, ny, nz])
    if np.any(hi <= lo):
        return
    xs = (b[0] + (np.arange(lo[0], hi[0]) + 0.5) * dx - centre_mm[0]).astype(np.float32)
    ys = (b[1] + (np.arange(lo[1], hi[1]) + 0.5) * dy - centre_mm[1]).astype(np.float32)
    zs = (b[2] + (np.arange(lo[2], hi[2]) + 0.5) * dz - centre_mm[2]).astype(np.float32)
    q = np.zeros((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), np.float32)
    for k in range(3):  # local coordinate k = sum_a world_a * rot[a, k]
        u = (zs[:, None, None] * np.float32(rot[2, k]) + ys[None, :, None] * np.float32(rot[1, k])
             + xs[None, None, :] * np.float32(rot[0, k]))
        q += (u / np.float32(semi_mm[k])) ** 2
    inside = q <= 1.0
    sub = vol[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]
    if mode == "add":
        sub[inside] += value
    else:
        sub[inside] = value


def ellipsoid_phantom(shape_zyx=(64, 64, 64), spacing=(1.0, 1.0, 1.0), n_ellipsoids=6, seed=0,
                      semi_range=(4.0, 24.0), density_range=(0.0, 0.005)) -> np.ndarray:
    """Sum of random ellipsoids (float32 attenuation, /mm): centres uniform in the
    inner 60% of the box, semi-axes U(semi_range) mm, random orientation,
    density U(density_range) each."""
    rng = np.random.default_rng(seed)
    vol = np.zeros(shape_zyx, dtype=np.float64)
    nz, ny, nx = shape_zyx
    ext = np.array([nx * spacing[0], ny * spacing[1], nz * spacing[2]])
    for _ in range(n_ellipsoids):
        c = rng.uniform(-0.3, 0.3, size=3) * ext
        semi = rng.uniform(*semi_range, size=3)
        rot = _rotation(rng)
        val = rng.uniform(*density_range)
        _paint_ellipsoid(vol, spacing, c, semi, rot, val)
    return vol.astype(np.float32)


def ct_phantom_hu(shape_zyx=(133, 512, 512), spacing=(0.703, 0.703, 2.5), seed=2) -> np.ndarray:
    """Chest-CT-shaped int16 HU phantom: air (-1000), an elliptic body (~40 HU)
    with two lungs (~-800), a spine and rib-like bone ellipsoids (700-2000 HU),
    seeded Gaussian noise (sigma 10 HU) inside the body, clipped to [-1000, 2000]."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape_zyx
    dx, dy, dz = spacing
    ext = np.array([nx * dx, ny * dy, nz * dz])
    hu = np.full(shape_zyx, -1000.0, dtype=np.float32)
    eye = np.eye(3)
    zlen = 0.45 * ext[2]
    body = np.array([0.42 * ext[0], 0.32 * ext[1], zlen * 1.5])
    _paint_ellipsoid(hu, spacing, np.zeros(3), body, eye, 40.0, mode="set")
    body_mask = hu > -999.0
    for side in (-1.0, 1.0):
        c = np.array([side * 0.17 * ext[0], 0.02 * ext[1], 0.05 * ext[2]])
        semi = np.array([0.13 * ext[0], 0.2 * ext[1], 0.42 * ext[2]]) * rng.uniform(0.9, 1.1, 3)
        _paint_ellipsoid(hu, spacing, c, semi, eye, -800.0, mode="set")
    # spine: a column of vertebra-like ellipsoids behind the centre
    nvert = 8
    for v in range(nvert):
        zc = (-0.45 + 0.9 * (v + 0.5) / nvert) * ext[2]
        c = np.array([0.0, -0.22 * ext[1], zc])
        semi = np.array([18.0, 16.0, 0.45 * ext[2] / nvert]) * rng.uniform(0.9, 1.1, 3)
        _paint_ellipsoid(hu, spacing, c, semi, eye, float(rng.uniform(700, 1400)), mode="set")
    # ribs: thin elongated ellipsoids around the lungs
    for r in range(12):
        ang = rng.uniform(0, 2 * np.pi)
        rad = np.array([0.38 * ext[0], 0.28 * ext[1]])
        c = np.array([rad[0] * np.cos(ang), rad[1] * np.sin(ang), rng.uniform(-0.4, 0.4) * ext[2]])
        semi = np.array([rng.uniform(25, 45), 4.0, 4.0])
        rot = np.array([[np.cos(ang + np.pi / 2), -np.sin(ang + np.pi / 2), 0],
                        [np.sin(ang + np.pi / 2), np.cos(ang + np.pi / 2), 0], [0, 0, 1]]).T
        _paint_ellipsoid(hu, spacing, c, semi, rot, float(rng.uniform(1000, 2000)), mode="set")
    noise = rng.standard_normal(size=shape_zyx, dtype=np.float32) * np.float32(10.0)
    hu = np.where(body_mask, hu + noise, hu)
    return np.clip(np.rint(hu), -1000, 2000).astype(np.int16)


def bone_tissue_phantom(shape_zyx=(512, 512, 512), spacing=(0.5, 0.5, 0.5), seed=6) -> np.ndarray:
    """Air (0), soft-tissue ellipsoids (0.02 /mm) and bone ellipsoids
    (0.04-0.06 /mm), float32."""
    rng = np.random.default_rng(seed)
    vol = np.zeros(shape_zyx, dtype=np.float32)
    nz, ny, nx = shape_zyx
    ext = np.array([nx * spacing[0], ny * spacing[1], nz * spacing[2]])
    _paint_ellipsoid(vol, spacing, np.zeros(3), 0.4 * ext * rng.uniform(0.9, 1.0, 3), _rotation(rng), 0.02, "set")
    for _ in range(6):
        c = rng.uniform(-0.2, 0.2, 3) * ext
        semi = rng.uniform(0.05, 0.15, 3) * ext
        _paint_ellipsoid(vol, spacing, c, semi, _rotation(rng), 0.02, "set")
    for _ in range(8):
        c = rng.uniform(-0.25, 0.25, 3) * ext
        semi = rng.uniform(0.02, 0.08, 3) * ext
        _paint_ellipsoid(vol, spacing, c, semi, _rotation(rng), float(rng.uniform(0.04, 0.06)), "set")
    return vol


def random_poses(batch: int, seed: int, max_angle_deg: float = 30.0, max_trans_mm: float = 10.0) -> np.ndarray:
    """(batch, 6) float32 poses: three Euler angles U(-max, max) deg (in radians)
    and three translations U(-max, max) mm."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(-max_angle_deg, max_angle_deg, size=(batch, 3)) * DEG
    tr = rng.uniform(-max_trans_mm, max_trans_mm, size=(batch, 3))
    return np.concatenate([ang, tr], axis=1).astype(np.float32)


def pose_offsets(batch: int, seed: int, max_angle_deg: float = 15.0, max_trans_mm: float = 20.0) -> np.ndarray:
    """(batch, 6) float32 initial offsets from a ground-truth pose."""
    return random_poses(batch, seed, max_angle_deg, max_trans_mm)


def landscape_offsets(n: int, seed: int, rot_range_deg=(90.0, 90.0, 45.0),
                      trans_range_mm=(30.0, 30.0, 30.0)) -> np.ndarray:
    """(n, 6) float32 pose displacements for a loss-landscape sweep: each parameter
    uniform on an interval of the given width centred on zero.  The defaults are the
    widths of the paper's landscape study (Sec. 3.2): 90 deg for the two source
    angles (rz, ry here), 45 deg for the roll (rx), 30 mm per translation."""
    rng = np.random.default_rng(seed)
    half = np.concatenate([np.deg2rad(np.asarray(rot_range_deg, np.float64)),
                           np.asarray(trans_range_mm, np.float64)]) / 2.0
    return rng.uniform(-half, half, size=(n, 6)).astype(np.float32)


def upstream_grad(shape, seed: int) -> np.ndarray:
    """Seeded upstream gradient dL/dDRR ~ U(-1, 1), float32."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=shape).astype(np.float32)


# --- the workloads ---------------------------------------------------------

MU_WATER = 0.02  # /mm, attenuation of water used for the HU -> mu mapping

TINY = dict(  # 64^3 FP32 volume, one pose, forward only
    name="tiny_64cube_64x64",
    shape_zyx=(64, 64, 64), spacing=(1.0, 1.0, 1.0),
    detector=Detector(300.0, 64, 64, 2.0, 2.0), batch=1, phantom_seed=0, pose_seed=1,
)

CT = dict(  # 512x512x133 chest-CT-shaped volume, 200x200 detector, 16 poses
    name="ct_512x512x133_200x200_b16",
    shape_zyx=(133, 512, 512), spacing=(0.703, 0.703, 2.5),
    detector=Detector(510.0, 200, 200, 1.4, 1.4), batch=16, phantom_seed=2, pose_seed=3,
)

REGISTRATION = dict(  # same CT, 256x256 detector, 64 concurrent registrations
    name="registration_512x512x133_256x256_b64",
    shape_zyx=(133, 512, 512), spacing=(0.703, 0.703, 2.5),
    detector=Detector(510.0, 256, 256, 1.4, 1.4), batch=64, truth_seed=4, offset_seed=5, steps=200,
)

LANDSCAPE = dict(  # same CT, 200x200 detector: -ZNCC at 4096 displacements around one pose
    name="landscape_512x512x133_200x200_n4096",
    shape_zyx=(133, 512, 512), spacing=(0.703, 0.703, 2.5),
    detector=Detector(510.0, 200, 200, 1.4, 1.4), n=4096, truth_seed=9, offset_seed=10,
)

PRECISION = dict(  # 512^3 at 0.5 mm, 1024x1024 detector, 8 poses
    name="precision_512cube_1024x1024_b8",
    shape_zyx=(512, 512, 512), spacing=(0.5, 0.5, 0.5),
    detector=Detector(510.0, 1024, 1024, 0.4, 0.4), batch=8, phantom_seed=6, pose_seed=7,
)


def ct_volume_hu(seed: int | None = None) -> np.ndarray:
    return ct_phantom_hu(CT["shape_zyx"], CT["spacing"], CT["phantom_seed"] if seed is None else seed)
