"""Shared helpers for the GPU parity tests (no DRR arithmetic here)."""
import numpy as np

FP32_TOL = 2e-5      # max per-pixel relative error, FP32 volume, vs the FP64 oracle
HALF_TOL = 5e-3      # same for 16-bit volumes vs the oracle on the FP32 volume
GRAD_TOL = 1e-4      # pose gradient, per pose and parameter group, relative to that group's max


def rel_err(E, E_ref, floor_frac=1e-3):
    """|E - E*| / max(|E*|, floor_frac * max|E*|), per pixel."""
    E = np.asarray(E, np.float64)
    E_ref = np.asarray(E_ref, np.float64)
    floor = floor_frac * max(np.abs(E_ref).max(), 1e-30)
    return np.abs(E - E_ref) / np.maximum(np.abs(E_ref), floor)


def grad_err(G, G_ref):
    """Per pose and group (rotations, translations): max|dG| / max|G*|."""
    G = np.asarray(G, np.float64)
    G_ref = np.asarray(G_ref, np.float64)
    out = []
    for grp in (slice(0, 3), slice(3, 6)):
        den = np.maximum(np.abs(G_ref[:, grp]).max(axis=1), 1e-30)
        out.append(np.abs(G[:, grp] - G_ref[:, grp]).max(axis=1) / den)
    return np.stack(out, axis=1)  # (B, 2)


def f32(x):
    """The float32 value the C ABI receives for a geometry parameter."""
    return float(np.float32(x))


def odet(det):
    """Detector tuple for the oracle with the float32 values the ABI sees."""
    sdr, H, W, dh, dw = det.as_tuple() if hasattr(det, "as_tuple") else det
    return (f32(sdr), int(H), int(W), f32(dh), f32(dw))


def ovol(data, spacing):
    """Oracle volume with the float32 spacing the ABI sees."""
    import oracle
    return oracle.Volume(data, tuple(f32(s) for s in spacing))


def osp(spacing):
    return tuple(f32(s) for s in spacing)
