"""GPU test of the L2 read-bandwidth probe used as the gather roofline's denominator."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def test_probe_reads_and_leaves_the_sink(drr):
    buf = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    sink = torch.full((1,), 7.0, device="cuda")
    drr.probe_l2_read(buf, 3, sink)
    torch.cuda.synchronize()
    assert sink.item() == 7.0  # a zero buffer never triggers the sink write
    assert drr.launch_count() > 0


def test_probe_argument_errors(drr):
    lib = drr.load()
    buf = torch.zeros(1 << 12, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, device="cuda")
    st = lib.drr_probe_l2_read(ctypes.c_void_p(buf.data_ptr() + 4), 1024, 1, ctypes.c_void_p(sink.data_ptr()), None)
    assert st == 1  # DRR_ERR_INVALID: not 16-byte aligned
    st = lib.drr_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), 8, 1, ctypes.c_void_p(sink.data_ptr()), None)
    assert st == 1  # fewer than 16 bytes
    st = lib.drr_probe_l2_read(ctypes.c_void_p(buf.data_ptr()), 1024, 0, ctypes.c_void_p(sink.data_ptr()), None)
    assert st == 1  # no repetitions
