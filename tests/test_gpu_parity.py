"""Parity of the CUDA kernels with the CPU oracle, through the C ABI.

Every comparison is bit-exact: a cipher's output is a unique bit string, so
the tolerance is zero (the paper's 3DES-EDE, Sec. II.A, in ECB mode)."""
import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

KERNELS = ["bitslice", "sptable"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


def _dev(a: np.ndarray, offset: int = 0):
    """A device copy of the bytes of `a`, starting `offset` bytes into its allocation."""
    buf = torch.zeros(a.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + a.size]
    view.copy_(torch.from_numpy(a))
    return buf, view


def _host(t) -> np.ndarray:
    return t.cpu().numpy()


def _run(ks, src, dst, decrypt, kernel):
    des3.des3_ecb_crypt_ex(ks, src, dst, src.numel(), decrypt, kernel)
    torch.cuda.synchronize()


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("decrypt", [False, True])
def test_config1_1mib_full_parity(kernel, decrypt):
    """1 MiB = 131072 blocks, one 3-key triple: every byte equals the oracle's."""
    key = inputs.key_triple(inputs.key_seed(1))
    data = inputs.data_bytes(inputs.data_seed(1), 1 << 20)
    ks = des3.des3_key_schedule(key)
    _, src = _dev(data)
    dst = torch.empty_like(src)
    _run(ks, src, dst, decrypt, kernel)
    ref = oracle.tdes_ecb(key, data, decrypt)
    assert np.array_equal(_host(dst), ref)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("keying", ["3key", "2key", "1key"])
@pytest.mark.parametrize("nblocks", [1, 2, 3, 31, 32, 33, 63, 64, 65, 1023, 1024, 1025, 2047, 4099, 65536 + 77])
def test_edge_sizes(kernel, keying, nblocks):
    key = inputs.key_triple(500 + nblocks, keying)
    data = inputs.data_bytes(600 + nblocks, 8 * nblocks)
    ks = des3.des3_key_schedule(key)
    for decrypt in (False, True):
        _, src = _dev(data)
        dst = torch.empty_like(src)
        _run(ks, src, dst, decrypt, kernel)
        assert np.array_equal(_host(dst), oracle.tdes_ecb(key, data, decrypt)), (decrypt,)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("off_in,off_out", [(8, 8), (0, 8), (8, 0), (24, 40)])
def test_unaligned_buffers(kernel, off_in, off_out):
    """8-byte aligned but not 16-byte aligned buffers, matching and mismatched."""
    nblocks = 3000
    key = inputs.key_triple(700)
    data = inputs.data_bytes(701, 8 * nblocks)
    ks = des3.des3_key_schedule(key)
    _, src = _dev(data, off_in)
    obuf = torch.full((8 * nblocks + off_out + 16,), 0xA5, dtype=torch.uint8, device="cuda")
    dst = obuf[off_out:off_out + 8 * nblocks]
    _run(ks, src, dst, False, kernel)
    assert np.array_equal(_host(dst), oracle.tdes_ecb(key, data))
    # guard bytes around the output are untouched
    o = _host(obuf)
    assert (o[:off_out] == 0xA5).all() and (o[off_out + 8 * nblocks:] == 0xA5).all()


@pytest.mark.parametrize("kernel", KERNELS)
def test_in_place_equals_out_of_place(kernel):
    key = inputs.key_triple(800)
    data = inputs.data_bytes(801, 8 * 50001)
    ks = des3.des3_key_schedule(key)
    _, a = _dev(data)
    b = torch.empty_like(a)
    _run(ks, a, b, False, kernel)
    _run(ks, a, a, False, kernel)
    assert torch.equal(a, b)
    assert np.array_equal(_host(a), oracle.tdes_ecb(key, data))


def test_kernels_agree_and_round_trip_16mib():
    key = inputs.key_triple(inputs.key_seed(3), "2key")
    data = inputs.data_bytes(inputs.data_seed(3), 16 << 20)
    ks = des3.des3_key_schedule(key)
    _, src = _dev(data)
    bs = torch.empty_like(src)
    sp = torch.empty_like(src)
    _run(ks, src, bs, False, "bitslice")
    _run(ks, src, sp, False, "sptable")
    assert torch.equal(bs, sp)
    assert np.array_equal(_host(bs), oracle.tdes_ecb(key, data))
    back = torch.empty_like(src)
    _run(ks, bs, back, True, "auto")
    assert torch.equal(back, src)


def test_errors_through_the_c_abi():
    lib = des3.lib()
    ks = des3.des3_key_schedule(inputs.key_triple(1))
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    import ctypes
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p, p, 12, 0, 0, s) == des3.DES3_EINVAL  # not a multiple of 8
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p + 4, p + 4, 16, 0, 0, s) == des3.DES3_EINVAL  # misaligned
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p, p + 8, 64, 0, 0, s) == des3.DES3_EINVAL  # partial overlap
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p, p, 64, 2, 0, s) == des3.DES3_EINVAL  # bad direction
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p, p, 64, 0, 9, s) == des3.DES3_EINVAL  # bad kernel
    assert lib.des3_ecb_crypt_ex(ctypes.byref(ks), p, p, 0, 0, 0, s) == des3.DES3_OK  # empty is a no-op
    bad = des3.des3_ks_t()
    assert lib.des3_ecb_crypt_ex(ctypes.byref(bad), p, p, 64, 0, 0, s) == des3.DES3_EKEY
    torch.cuda.synchronize()
    assert (buf == 0).all()


@pytest.mark.parametrize("size", [64 << 10, 1 << 20, 16 << 20, 256 << 20])
@pytest.mark.parametrize("keying", ["3key", "2key"])
def test_size_sweep(size, keying):
    """The size/keying sweep workload: both kernels, both directions.  The
    oracle checks every block up to 16 MiB and a seeded sample of 2^16
    blocks beyond; the two independent kernels must agree on every byte."""
    key = inputs.key_triple(inputs.key_seed(3) + size, keying)
    ks = des3.des3_key_schedule(key)
    nblocks = size // 8
    words = inputs.splitmix64_torch(inputs.data_seed(3) + size, 0, nblocks, "cuda")
    src = words.view(torch.uint8)
    for decrypt in (False, True):
        bs = torch.empty_like(src)
        sp = torch.empty_like(src)
        _run(ks, src, bs, decrypt, "bitslice")
        _run(ks, src, sp, decrypt, "sptable")
        assert torch.equal(bs, sp)
        if size <= (16 << 20):
            ref = oracle.tdes_ecb(key, _host(src), decrypt)
            assert np.array_equal(_host(bs), ref)
        else:
            idx = np.unique(inputs.splitmix64(99, 0, 1 << 16) % np.uint64(nblocks)).astype(np.int64)
            plain = inputs.splitmix64_at(inputs.data_seed(3) + size, idx).astype("<u8").view(np.uint8)
            ref = oracle.tdes_ecb(key, plain, decrypt).view("<u8")
            got = bs.view(torch.int64)[torch.from_numpy(idx).cuda()].cpu().numpy().view("<u8")
            assert np.array_equal(got, ref)


def _tunables():
    from paper_1305_4376_gb300 import autotune
    return autotune.SINGLE_CANDIDATES


@pytest.mark.parametrize("shape", _tunables())
def test_every_tunable_launch_shape_is_bit_exact(shape):
    """Whatever the autotuner picks for a size class, the bytes are the same."""
    from paper_1305_4376_gb300 import autotune
    kernel, threads, ctas = shape
    nblocks = 65536 + 77  # size class 19
    key = inputs.key_triple(900)
    data = inputs.data_bytes(901, 8 * nblocks)
    ks = des3.des3_key_schedule(key)
    _, src = _dev(data)
    dst = torch.empty_like(src)
    try:
        autotune.set_entries(des3.DES3_TUNE_SINGLE, [(19, kernel, threads, ctas)])
        _run(ks, src, dst, False, "auto")
    finally:
        autotune.reset()
    assert np.array_equal(_host(dst), oracle.tdes_ecb(key, data))


@pytest.mark.parametrize("threads,ctas", [(384, 3), (256, 3), (128, 2), (64, 1)])
def test_table_kernel_blocks_per_thread_switch_points(threads, ctas):
    """The table kernel runs 1, 2 or 4 blocks per thread depending on how the
    buffer compares with the grid's thread slots (SMs x CTAs x threads).  At
    and around both switch points, with ragged remainders and an unaligned
    start, both directions: every byte equals the bitsliced kernel's, and the
    oracle checks the first, last and seeded blocks."""
    from paper_1305_4376_gb300 import autotune
    slots = torch.cuda.get_device_properties(0).multi_processor_count * ctas * threads
    key = inputs.key_triple(950 + threads)
    ks = des3.des3_key_schedule(key)
    try:
        autotune.set_entries(des3.DES3_TUNE_SINGLE, [(c, des3.DES3_KERNEL_SPTABLE, threads, ctas) for c in range(40)])
        for nblocks in (slots - 1, slots, slots + 3, 4 * slots - 1, 4 * slots, 4 * slots + 5):
            data = inputs.data_bytes(960 + nblocks % 97, 8 * nblocks)
            for offset in (0, 8):
                _, src = _dev(data, offset)
                for decrypt in (False, True):
                    sp = torch.empty_like(src)
                    bs = torch.empty_like(src)
                    des3.des3_ecb_crypt_ex(ks, src, sp, src.numel(), decrypt, "sptable")
                    des3.des3_ecb_crypt_ex(ks, src, bs, src.numel(), decrypt, "bitslice")
                    torch.cuda.synchronize()
                    assert torch.equal(sp, bs), (nblocks, offset, decrypt)
                    seeded = inputs.splitmix64(nblocks, 0, 64) % np.uint64(nblocks)
                    pick = np.unique(np.concatenate([np.array([0, nblocks - 1], dtype=np.uint64), seeded]))
                    pick = pick.astype(np.int64)
                    idx = (pick[:, None] * 8 + np.arange(8)).reshape(-1)
                    want = oracle.tdes_ecb(key, data.reshape(-1, 8)[pick].reshape(-1), decrypt)
                    assert np.array_equal(_host(sp)[idx], want), (nblocks, offset, decrypt)
    finally:
        autotune.reset()
