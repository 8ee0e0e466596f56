"""CTR and CBC decryption (NIST SP 800-38A) on the GPU against the oracle:
bit-exact on ragged sizes, unaligned buffers, counters that carry across 2^32
and wrap at 2^64, and in-place CTR; CBC refuses any overlap."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 32, 33, 1023, 1024, 1025, 4099, 65536 + 77]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


def _dev(a: np.ndarray, offset: int = 0):
    buf = torch.zeros(a.size + offset + 16, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + a.size]
    view.copy_(torch.from_numpy(a))
    return view


@pytest.mark.parametrize("nblocks", SIZES)
@pytest.mark.parametrize("start", [0, 0xFFFFFFFF - 100, (1 << 64) - 700, 0x0123456789ABCDEF])
def test_ctr_matches_oracle(nblocks, start):
    key = inputs.key_triple(2000 + nblocks)
    ctr0 = start.to_bytes(8, "big")
    data = inputs.data_bytes(2100 + nblocks, 8 * nblocks)
    ks = des3.des3_key_schedule(key)
    src = _dev(data)
    dst = torch.empty_like(src)
    des3.des3_ctr_crypt(ks, ctr0, src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.tdes_ctr(key, ctr0, data))
    # in place, and twice gives back the input
    des3.des3_ctr_crypt(ks, ctr0, dst, dst)
    torch.cuda.synchronize()
    assert torch.equal(dst, src)


@pytest.mark.parametrize("nblocks", SIZES)
def test_cbc_decrypt_matches_oracle(nblocks):
    key = inputs.key_triple(2200 + nblocks)
    iv = inputs.data_bytes(2300 + nblocks, 8).tobytes()
    plain = inputs.data_bytes(2400 + nblocks, 8 * nblocks)
    ct = oracle.tdes_cbc(key, iv, plain)  # CBC encryption is the oracle's (sequential)
    ks = des3.des3_key_schedule(key)
    src = _dev(ct)
    dst = torch.empty_like(src)
    des3.des3_cbc_decrypt(ks, iv, src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), plain)
    assert np.array_equal(dst.cpu().numpy(), oracle.tdes_cbc(key, iv, ct, decrypt=True))


@pytest.mark.parametrize("off_in,off_out", [(8, 8), (0, 8), (8, 24)])
def test_modes_unaligned(off_in, off_out):
    nblocks = 5000
    key = inputs.key_triple(2500)
    iv = inputs.data_bytes(2501, 8).tobytes()
    data = inputs.data_bytes(2502, 8 * nblocks)
    ks = des3.des3_key_schedule(key)
    src = _dev(data, off_in)
    obuf = torch.zeros(8 * nblocks + off_out + 16, dtype=torch.uint8, device="cuda")
    dst = obuf[off_out:off_out + 8 * nblocks]
    des3.des3_ctr_crypt(ks, iv, src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.tdes_ctr(key, iv, data))
    des3.des3_cbc_decrypt(ks, iv, src, dst)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), oracle.tdes_cbc(key, iv, data, decrypt=True))


def test_cbc_refuses_overlap_and_ctr_checks_arguments():
    lib = des3.lib()
    ks = des3.des3_key_schedule(inputs.key_triple(1))
    buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    p = buf.data_ptr()
    s = torch.cuda.current_stream().cuda_stream
    iv = bytes(8)
    assert lib.des3_cbc_decrypt(ctypes.byref(ks), iv, p, p, 64, s) == des3.DES3_EINVAL  # in place
    assert lib.des3_cbc_decrypt(ctypes.byref(ks), iv, p, p + 8, 64, s) == des3.DES3_EINVAL  # overlap
    assert lib.des3_ctr_crypt(ctypes.byref(ks), iv, p, p, 12, s) == des3.DES3_EINVAL
    assert lib.des3_ctr_crypt(ctypes.byref(ks), None, p, p, 16, s) == des3.DES3_EINVAL
    assert lib.des3_ctr_crypt(ctypes.byref(ks), iv, p, p, 0, s) == des3.DES3_OK
    torch.cuda.synchronize()
    assert (buf == 0).all()


def test_ctr_256mib_sampled():
    """A large CTR buffer: the oracle checks 2^16 seeded blocks and the ends."""
    nblocks = (256 << 20) // 8
    key = inputs.key_triple(2600)
    ctr0 = ((1 << 64) - 12345).to_bytes(8, "big")  # wraps inside the buffer
    words = inputs.splitmix64_torch(2601, 0, nblocks, "cuda")
    src = words.view(torch.uint8)
    dst = torch.empty_like(src)
    ks = des3.des3_key_schedule(key)
    des3.des3_ctr_crypt(ks, ctr0, src, dst)
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([inputs.splitmix64(2602, 0, 1 << 16) % np.uint64(nblocks),
                                    np.array([0, 12344, 12345, 12346, nblocks - 1], dtype=np.uint64)])).astype(np.int64)
    t0 = int.from_bytes(ctr0, "big")
    got = dst.view(torch.int64)[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint8)
    plain = src.view(torch.int64)[torch.from_numpy(idx).cuda()].cpu().numpy().view(np.uint8)
    ctrs = b"".join(((t0 + int(i)) % (1 << 64)).to_bytes(8, "big") for i in idx)
    ks_stream = oracle.tdes_ecb(key, ctrs)
    assert np.array_equal(got, plain ^ ks_stream)


# ---------------------------------------------------------------- single DES

@pytest.mark.parametrize("kernel", ["bitslice", "sptable"])
@pytest.mark.parametrize("nblocks", [1, 33, 1025, 65536 + 77])
def test_single_des_ecb_matches_oracle(kernel, nblocks):
    """Single DES (16 rounds, the building block of Sec. II.A) on both kernels."""
    key = inputs.key_triple(2700 + nblocks)[:8]
    data = inputs.data_bytes(2701 + nblocks, 8 * nblocks)
    ks = des3.des3_key_schedule_des(key)
    src = _dev(data)
    for decrypt in (False, True):
        dst = torch.empty_like(src)
        des3.des3_ecb_crypt_ex(ks, src, dst, decrypt=decrypt, kernel=kernel)
        torch.cuda.synchronize()
        assert np.array_equal(dst.cpu().numpy(), oracle.des_ecb(key, data, decrypt))


def test_single_des_key_in_batch_ctr_and_host_paths():
    """The 48-round paths run a single-DES key as 3DES with K1 = K2 = K3."""
    key = inputs.key_triple(2800)[:8]
    ks = des3.des3_key_schedule_des(key)
    data = inputs.data_bytes(2801, 8 * 3000)
    src = _dev(data)
    out = torch.zeros_like(src)
    des3.des3_ecb_batch(des3.make_keys([ks]), des3.make_jobs([(src, out, src.numel(), 0, True)]))
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.des_ecb(key, data, True))
    ctr0 = bytes(range(8))
    des3.des3_ctr_crypt(ks, ctr0, src, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), oracle.tdes_ctr(key * 3, ctr0, data))
    h_in = torch.from_numpy(data.copy()).pin_memory()
    h_out = torch.zeros_like(h_in).pin_memory()
    work = torch.empty(2 << 20, dtype=torch.uint8, device="cuda")
    des3.des3_ecb_host(ks, h_in.data_ptr(), h_out.data_ptr(), data.size, False, work.data_ptr(), work.numel())
    torch.cuda.synchronize()
    assert np.array_equal(h_out.numpy(), oracle.des_ecb(key, data))


def _weak_key(c0: int, d0: int) -> bytes:
    """Invert PC-1 for C0||D0 (the oracle's table) and set odd parity."""
    pc1 = oracle.table("PC1")
    cd = (c0 << 28) | d0
    bits = [0] * 64
    for i, pos in enumerate(pc1):
        bits[pos - 1] = (cd >> (55 - i)) & 1
    out = []
    for b in range(8):
        v = 0
        for i in range(8):
            v = (v << 1) | bits[8 * b + i]
        out.append(inputs.odd_parity(v))
    return bytes(out)


def test_weak_keys_are_involutions_on_the_gpu():
    """The degenerate keys of DES: with a weak key, encrypting twice is the
    identity, for single DES (16 rounds) and 3DES with K1 = K2 = K3."""
    ones = (1 << 28) - 1
    data = inputs.data_bytes(2900, 8 * 5000)
    src = _dev(data)
    for c0, d0 in ((0, 0), (0, ones), (ones, 0), (ones, ones)):
        k = _weak_key(c0, d0)
        for ks in (des3.des3_key_schedule_des(k), des3.des3_key_schedule(k * 3)):
            for kernel in ("bitslice", "sptable"):
                once = torch.empty_like(src)
                twice = torch.empty_like(src)
                des3.des3_ecb_crypt_ex(ks, src, once, kernel=kernel)
                des3.des3_ecb_crypt_ex(ks, once, twice, kernel=kernel)
                torch.cuda.synchronize()
                assert not torch.equal(once, src)
                assert torch.equal(twice, src)
                assert np.array_equal(once.cpu().numpy(), oracle.des_ecb(k, data))
