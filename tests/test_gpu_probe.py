"""des3_pipe_probe, the in-run measurement of the roofline denominators: it
launches, reports its instruction count and SM count, and gives a clock and
per-SM rates in the physically possible range (a warp instruction per SM
sub-partition per clock at most, i.e. 128 lanes per SM per clock)."""
import pytest

from paper_1305_4376_gb300 import des3

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


@pytest.mark.parametrize("kind", ["lop3", "imad", "lop3+imad", "lds"])
def test_probe_rates_are_plausible(kind):
    sink = torch.zeros(4, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    des3.des3_pipe_probe(kind, 50, sink)  # warm-up
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    ins, sms = des3.des3_pipe_probe(kind, 400, sink)
    b.record(stream)
    torch.cuda.synchronize()
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    assert ins == sms * 8 * 256 * 8 * 16 * 400
    cyc, ns = int(sink[1].item()), int(sink[2].item())
    assert cyc > 0 and ns > 0
    mhz = cyc / ns * 1e3
    assert 300 < mhz < 3000
    per_sm_clk = ins / (a.elapsed_time(b) * 1e-3) / sms / (mhz * 1e6)
    assert 4 < per_sm_clk <= 140, per_sm_clk


def test_probe_rejects_bad_arguments():
    lib = des3.lib()
    import ctypes
    sink = torch.zeros(4, dtype=torch.int64, device="cuda")
    ins, sms = ctypes.c_uint64(), ctypes.c_uint32()
    args = (ctypes.byref(ins), ctypes.byref(sms), None)
    assert lib.des3_pipe_probe(4, 10, sink.data_ptr(), *args) == des3.DES3_EINVAL
    assert lib.des3_pipe_probe(0, 0, sink.data_ptr(), *args) == des3.DES3_EINVAL
    assert lib.des3_pipe_probe(0, 10, None, *args) == des3.DES3_EINVAL
    assert lib.des3_pipe_probe(0, 10, sink.data_ptr() + 4, *args) == des3.DES3_EINVAL
