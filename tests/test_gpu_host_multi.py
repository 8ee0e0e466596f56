"""des3_ecb_host_multi: a host buffer split into contiguous block ranges, each
range streamed through its own device.  This run has one GPU, so device 0 is
named several times (each range with its own workspace); every output byte is
compared with the oracle, with pinned and pageable memory, in place, with
more ranges than the buffer has tiles, and with a ragged tail."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("nranges,nbytes", [(3, 3 * (1 << 20) + 8 * 1234), (4, 8 * 2048 + 8 * 5), (2, 64 << 20)])
def test_ranges_on_one_device_match_the_oracle(pinned, nranges, nbytes):
    key = inputs.key_triple(5100 + nranges)
    data = inputs.data_bytes(5101, nbytes)
    ks = des3.des3_key_schedule(key)
    h_in = torch.from_numpy(data.copy())
    h_out = torch.zeros(nbytes, dtype=torch.uint8)
    if pinned:
        h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
    first = des3.des3_range_split(nbytes // 8, nranges)
    works = [torch.empty(6 << 20, dtype=torch.uint8, device="cuda") for _ in range(nranges)]
    d_work = [w if first[i + 1] > first[i] else None for i, w in enumerate(works)]
    des3.des3_ecb_host_multi(ks, h_in.data_ptr(), h_out.data_ptr(), nbytes, False, [0] * nranges, d_work,
                             [w.numel() for w in works])
    assert np.array_equal(h_out.numpy(), oracle.tdes_ecb(key, data))
    # decryption in place
    des3.des3_ecb_host_multi(ks, h_out.data_ptr(), h_out.data_ptr(), nbytes, True, [0] * nranges, d_work,
                             [w.numel() for w in works])
    assert np.array_equal(h_out.numpy(), data)


def test_multi_argument_errors():
    lib = des3.lib()
    ks = des3.des3_key_schedule(inputs.key_triple(1))
    n = 8 * 4096
    h = torch.zeros(n, dtype=torch.uint8).pin_memory()
    w = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    p = h.data_ptr()
    devs2 = (ctypes.c_int * 2)(0, 0)
    same = (ctypes.c_void_p * 2)(w.data_ptr(), w.data_ptr())
    sizes2 = (ctypes.c_size_t * 2)(4 << 20, 4 << 20)
    # one workspace for two non-empty ranges would race
    assert lib.des3_ecb_host_multi(ctypes.byref(ks), p, p, n, 0, 2, devs2, same, sizes2) == des3.DES3_EINVAL
    bad_dev = (ctypes.c_int * 1)(torch.cuda.device_count())
    one = (ctypes.c_void_p * 1)(w.data_ptr())
    size1 = (ctypes.c_size_t * 1)(4 << 20)
    assert lib.des3_ecb_host_multi(ctypes.byref(ks), p, p, n, 0, 1, bad_dev, one, size1) == des3.DES3_ENODEV
    small = (ctypes.c_size_t * 1)(1 << 20)
    dev0 = (ctypes.c_int * 1)(0)
    assert lib.des3_ecb_host_multi(ctypes.byref(ks), p, p, n, 0, 1, dev0, one, small) == des3.DES3_EINVAL
    cur = torch.cuda.current_device()
    assert lib.des3_ecb_host_multi(ctypes.byref(ks), p, p, n, 0, 1, dev0, one, size1) == des3.DES3_OK
    assert torch.cuda.current_device() == cur
