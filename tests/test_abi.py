"""CPU checks of the C ABI: the library loads and exports every function
include/drr.h declares.  No compute call is made (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(drr_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2208_12737_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("drr_volume_create", "drr_volume_destroy", "drr_render", "drr_render_backward",
                     "drr_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2208_12737_gb300 import drr
    assert set(drr.EXPORTS) == _declared()


def test_version_and_error_string(lib):
    lib.drr_version.restype = ctypes.c_char_p
    lib.drr_last_error.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.drr_version()
    assert lib.drr_last_error() is not None


def test_argument_errors_without_gpu(lib):
    # argument validation happens before any CUDA call
    lib.drr_render.restype = ctypes.c_int
    assert lib.drr_render(None, None, None, 1, None, None, None) == 1  # DRR_ERR_INVALID
    lib.drr_volume_create.restype = ctypes.c_int
    out = ctypes.c_void_p()
    assert lib.drr_volume_create(None, 0, 0, 1, 1, 1, ctypes.c_float(1), ctypes.c_float(1), ctypes.c_float(1),
                                 None, None, ctypes.byref(out)) == 1


def _create(lib, data, nx, ny, nz, dx=1.0, dy=1.0, dz=1.0, src_dtype=0):
    out = ctypes.c_void_p()
    lib.drr_volume_create.restype = ctypes.c_int
    lib.drr_last_error.restype = ctypes.c_char_p
    st = lib.drr_volume_create(data, 0, src_dtype, nx, ny, nz, ctypes.c_float(dx), ctypes.c_float(dy),
                               ctypes.c_float(dz), None, None, ctypes.byref(out))
    return st, lib.drr_last_error().decode(), out.value


def test_volume_limits_are_checked_before_any_device_work(lib):
    # argument validation happens on the host before any CUDA call, so it runs here
    buf = ctypes.create_string_buffer(64)
    st, msg, h = _create(lib, buf, 1291, 1291, 1291)  # (n+2)^3 = 2.16e9 padded voxels >= 2^31
    assert st == 1 and "too large" in msg and h is None
    st, msg, _ = _create(lib, buf, 2147483646, 2, 2)  # no int32 overflow in the size check
    assert st == 1 and "too large" in msg
    st, msg, _ = _create(lib, buf, 0, 4, 4)
    assert st == 1 and "positive" in msg
    st, msg, _ = _create(lib, buf, 4, 4, 4, dx=0.0)
    assert st == 1 and "spacing" in msg
    st, msg, _ = _create(lib, buf, 4, 4, 4, dz=float("inf"))
    assert st == 1 and "spacing" in msg
    st, msg, _ = _create(lib, None, 4, 4, 4)
    assert st == 1 and "NULL" in msg
    st, msg, _ = _create(lib, buf, 4, 4, 4, src_dtype=1)  # BF16 is a storage type, not an input type
    assert st == 1 and "src_dtype" in msg


def test_only_the_padded_linear_layouts_and_known_storage_are_accepted(lib):
    class Options(ctypes.Structure):  # drr_volume_options of include/drr.h
        _fields_ = [("storage", ctypes.c_int32), ("hu_mu_water", ctypes.c_float), ("layout", ctypes.c_int32)]
    buf = ctypes.create_string_buffer(4 * 64)
    out = ctypes.c_void_p()
    lib.drr_volume_create.restype = ctypes.c_int
    lib.drr_last_error.restype = ctypes.c_char_p
    for opt, word in ((Options(0, 0.0, 4), b"layout"), (Options(0, 0.0, -1), b"layout"),
                      (Options(3, 0.0, 0), b"storage"), (Options(0, -1.0, 0), b"mu_water")):
        st = lib.drr_volume_create(buf, 0, 0, 4, 4, 4, ctypes.c_float(1.0), ctypes.c_float(1.0), ctypes.c_float(1.0),
                                   ctypes.byref(opt), None, ctypes.byref(out))
        assert st == 1 and word in lib.drr_last_error() and out.value is None


def test_calls_on_a_null_volume_fail_cleanly(lib):
    lib.drr_render.restype = ctypes.c_int
    lib.drr_last_error.restype = ctypes.c_char_p
    st = lib.drr_render(None, None, None, 1, None, None, None)
    assert st == 1 and b"NULL" in lib.drr_last_error()


def test_server_configs_are_checked_before_any_device_work(lib):
    from paper_2208_12737_gb300 import drr
    lib = drr.load()
    out = ctypes.c_void_p()
    for field, value in (("tick_depth", 5), ("tick_depth", 1), ("max_tick_work", -1), ("max_inflight", 5000),
                         ("max_tick_poses", (1 << 20) + 1), ("spin_poll_us", -1), ("spin_poll_us", 2_000_000)):
        cfg = drr.drr_server_config()
        setattr(cfg, field, value)
        assert lib.drr_server_create(ctypes.byref(cfg), ctypes.byref(out)) == 1, field
        assert out.value is None
