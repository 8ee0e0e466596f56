"""des3_ecb_host (host buffers through a device workspace, copies overlapped
with the kernels) against the oracle, and concurrent calls from several host
threads on distinct streams."""
import ctypes
import threading

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
@pytest.mark.parametrize("work_mib", [2, 7, 192])
def test_host_pipeline_matches_oracle(pinned, work_mib):
    nbytes = 3 * (1 << 20) + 8 * 1234  # several chunks plus a ragged tail
    key = inputs.key_triple(3000 + work_mib)
    data = inputs.data_bytes(3001, nbytes)
    ks = des3.des3_key_schedule(key)
    h_in = torch.from_numpy(data.copy())
    h_out = torch.zeros(nbytes, dtype=torch.uint8)
    if pinned:
        h_in, h_out = h_in.pin_memory(), h_out.pin_memory()
    work = torch.empty(work_mib << 20, dtype=torch.uint8, device="cuda")
    des3.des3_ecb_host(ks, h_in.data_ptr(), h_out.data_ptr(), nbytes, False, work.data_ptr(), work.numel())
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), oracle.tdes_ecb(key, data))
    # decrypt in place (h_in == h_out)
    des3.des3_ecb_host(ks, h_out.data_ptr(), h_out.data_ptr(), nbytes, True, work.data_ptr(), work.numel())
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), data)


def test_host_pipeline_argument_errors():
    lib = des3.lib()
    ks = des3.des3_key_schedule(inputs.key_triple(1))
    h = torch.zeros(4096, dtype=torch.uint8).pin_memory()
    work = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    p, w = h.data_ptr(), work.data_ptr()
    assert lib.des3_ecb_host(ctypes.byref(ks), p, p, 4096, 0, w, 1 << 20, s) == des3.DES3_EINVAL  # workspace too small
    assert lib.des3_ecb_host(ctypes.byref(ks), p, p, 4096, 0, w + 8, 4 << 20, s) == des3.DES3_EINVAL  # unaligned
    assert lib.des3_ecb_host(ctypes.byref(ks), p, p, 4092, 0, w, 4 << 20, s) == des3.DES3_EINVAL  # ragged size
    assert lib.des3_ecb_host(ctypes.byref(ks), p, p + 8, 4000, 0, w, 4 << 20, s) == des3.DES3_EINVAL  # overlap
    assert lib.des3_ecb_host(ctypes.byref(ks), p, p, 0, 0, w, 4 << 20, s) == des3.DES3_OK


def test_concurrent_calls_on_distinct_streams():
    """Several host threads, each with its own stream, key and buffers."""
    n = 6
    nbytes = 4 << 20
    keys = inputs.key_triples(3100, n)
    datas = [inputs.data_bytes(3200 + i, nbytes) for i in range(n)]
    srcs = [torch.from_numpy(d).cuda() for d in datas]
    outs = [torch.empty_like(s) for s in srcs]
    torch.cuda.synchronize()  # the worker streams do not wait on the default stream
    errors = []

    def work(i):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            ks = des3.des3_key_schedule(keys[i])
            for _ in range(5):
                des3.des3_ecb_crypt_ex(ks, srcs[i], outs[i], nbytes, i % 2 == 1, "auto", stream=st)
            st.synchronize()
        except Exception as e:  # noqa: BLE001
            errors.append(e)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(n)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors
    for i in range(n):
        assert np.array_equal(outs[i].cpu().numpy(), oracle.tdes_ecb(keys[i], datas[i], i % 2 == 1))
