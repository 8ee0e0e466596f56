"""des3_ecb_batch_noalloc: the batched call for callers that cannot allocate
device memory (for example a process whose device memory all belongs to its
own pool allocator).  It keeps its job and key tables in a fixed array
inside the library instead of allocating them, so its results must equal
des3_ecb_batch's byte for byte (the cipher's tolerance is zero), call after
call, even though every call reuses the same array.

This file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes

import pytest

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


def _case(seed, njobs, nkeys):
    """Seeded jobs over one device arena: mixed sizes (ragged, tile-sized,
    multi-tile), mixed directions, some in place."""
    w = inputs.splitmix64(seed, 0, 3 * njobs)
    sizes = [8 * int(1 + w[i] % 20000) for i in range(njobs)]
    sizes[0] = 8 * 1024
    offs, pos = [], 0
    for n in sizes:
        offs.append(pos)
        pos += (n + 255) // 256 * 256
    src = inputs.splitmix64_torch(seed + 1, 0, pos // 8 + 32, "cuda").view(torch.uint8)
    keys = des3.make_keys([des3.des3_key_schedule(k) for k in inputs.key_triples(seed + 2, nkeys)])
    spec = [(o, n, int(w[njobs + i] % nkeys), bool(w[2 * njobs + i] & 1), i % 4 == 3)
            for i, (o, n) in enumerate(zip(offs, sizes))]
    return src, keys, spec


def _jobs(src, out, spec):
    return des3.make_jobs([(src[o:o + n] if inplace else src[o:o + n], (src if inplace else out)[o:o + n],
                            n, k, dec) for (o, n, k, dec, inplace) in spec])


def _run_both(src, keys, spec):
    """The same batch through des3_ecb_batch and des3_ecb_batch_noalloc."""
    lib = des3.lib()
    s = torch.cuda.current_stream().cuda_stream
    a_src, b_src = src.clone(), src.clone()
    a_out, b_out = torch.zeros_like(src), torch.zeros_like(src)
    ja, jb = _jobs(a_src, a_out, spec), _jobs(b_src, b_out, spec)
    assert lib.des3_ecb_batch(keys, len(keys), ja, len(ja), s) == des3.DES3_OK
    assert lib.des3_ecb_batch_noalloc(keys, len(keys), jb, len(jb), s) == des3.DES3_OK
    torch.cuda.synchronize()
    return (a_src, a_out), (b_src, b_out)


def test_noalloc_matches_allocating_batch_on_two_calls_in_a_row():
    for seed, njobs, nkeys in ((9001, 37, 5), (9101, 300, 64)):
        src, keys, spec = _case(seed, njobs, nkeys)
        (a_src, a_out), (b_src, b_out) = _run_both(src, keys, spec)
        assert torch.equal(a_out, b_out)
        assert torch.equal(a_src, b_src)  # in-place jobs
        assert not torch.equal(a_out, torch.zeros_like(a_out))


def test_noalloc_rejects_more_than_its_maximum():
    lib = des3.lib()
    keys = des3.make_keys([des3.des3_key_schedule(inputs.key_triple(1))])
    fake = 1 << 40  # never touched: the size check comes first
    too_many = des3.make_jobs([(fake, fake, 8, 0, False)] * 1025)
    assert lib.des3_ecb_batch_noalloc(keys, 1, too_many, 1025, None) == des3.DES3_EINVAL
    many_keys = des3.make_keys([des3.des3_key_schedule(inputs.key_triple(1))] * 1025)
    one = des3.make_jobs([(fake, fake, 8, 0, False)])
    assert lib.des3_ecb_batch_noalloc(many_keys, 1025, one, 1, None) == des3.DES3_EINVAL
    assert ctypes.sizeof(des3.des3_job_t) == 32


def _cudart():
    """The CUDA runtime as a shared library (the one torch loaded, found by its
    soname, or the toolkit's), for reading the device's memory state."""
    for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("no shared CUDA runtime to read the memory state with")


def _memory_state(rt, pool):
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    used_high, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 0x8, ctypes.byref(used_high)) == 0  # UsedMemHigh
    assert rt.cudaMemPoolGetAttribute(pool, 0x5, ctypes.byref(reserved)) == 0  # ReservedMemCurrent
    return free.value, used_high.value, reserved.value


def test_noalloc_allocates_nothing():
    """The call's defining promise: around it, the device's free memory and
    the default memory pool (which cudaMallocAsync draws from) do not move.
    The allocating batch call, measured the same way, does move the pool's
    high-water mark, which shows the measurement can see an allocation."""
    rt = _cudart()
    lib = des3.lib()
    src, keys, spec = _case(9201, 40, 6)
    out = torch.zeros_like(src)
    jobs = _jobs(src, out, spec)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.des3_ecb_batch_noalloc(keys, len(keys), jobs, len(jobs), s) == des3.DES3_OK  # first call: set-up
    torch.cuda.synchronize()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    zero = ctypes.c_uint64(0)
    assert rt.cudaMemPoolSetAttribute(pool, 0x8, ctypes.byref(zero)) == 0  # reset UsedMemHigh
    before = _memory_state(rt, pool)
    for _ in range(3):
        assert lib.des3_ecb_batch_noalloc(keys, len(keys), jobs, len(jobs), s) == des3.DES3_OK
    torch.cuda.synchronize()
    after = _memory_state(rt, pool)
    assert after == before, (before, after)
    # control: the allocating call raises the pool's high-water mark
    assert lib.des3_ecb_batch(keys, len(keys), jobs, len(jobs), s) == des3.DES3_OK
    torch.cuda.synchronize()
    assert _memory_state(rt, pool)[1] > before[1]


def test_noalloc_refuses_a_capturing_stream():
    """A stream under graph capture is refused before anything is enqueued;
    the capture then ends cleanly and the next call runs normally."""
    lib = des3.lib()
    src, keys, spec = _case(9301, 12, 3)
    out = torch.zeros_like(src)
    jobs = _jobs(src, out, spec)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            rc = lib.des3_ecb_batch_noalloc(keys, len(keys), jobs, len(jobs), side.cuda_stream)
    assert rc == des3.DES3_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(out, torch.zeros_like(out))
    (a_src, a_out), (b_src, b_out) = _run_both(src, keys, spec)
    assert torch.equal(a_out, b_out) and torch.equal(a_src, b_src)
