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
