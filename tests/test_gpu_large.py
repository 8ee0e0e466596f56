"""The 4 GiB single-buffer workload in the launch configuration the benchmark
times (in place, default kernel): the two independent kernels agree on every
byte, decryption restores the input, the oracle checks 2^22 seeded blocks one
by one, and the whole encrypted and decrypted outputs match the oracle's
digests of the full workload.  The same holds at 4 GiB for 2-key triples and
for the table kernel's decryption (the size and keying sweep's largest
cells)."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

CONFIG_ID = 2
NBYTES = 4 << 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


def test_4gib_in_place_parity():
    key = inputs.key_triple(inputs.key_seed(CONFIG_ID))
    ks = des3.des3_key_schedule(key)
    nblocks = NBYTES // 8
    words = inputs.splitmix64_torch(inputs.data_seed(CONFIG_ID), 0, nblocks, "cuda")
    buf = words.view(torch.uint8)
    plain = words.clone()
    # the benchmark's call: default kernel, in place
    des3.des3_ecb_encrypt(ks, buf, buf)
    other = plain.clone()
    des3.des3_ecb_crypt_ex(ks, other, other, decrypt=False, kernel="sptable")
    torch.cuda.synchronize()
    assert torch.equal(words, other)
    del other
    idx = np.unique(inputs.splitmix64(4242, 0, 1 << 22) % np.uint64(nblocks)).astype(np.int64)
    idx = np.concatenate([idx, [0, nblocks - 1]])
    t = torch.from_numpy(idx).cuda()
    p = plain[t].cpu().numpy().view(np.uint8)
    c = words[t].cpu().numpy().view(np.uint8)
    assert np.array_equal(c, oracle.tdes_ecb(key, p))
    des3.des3_ecb_decrypt(ks, buf, buf)
    torch.cuda.synchronize()
    assert torch.equal(words, plain)


def _sample_idx(nblocks, seed=4242):
    idx = np.unique(inputs.splitmix64(seed, 0, 1 << 22) % np.uint64(nblocks)).astype(np.int64)
    return np.concatenate([idx, [0, nblocks - 1]])


@pytest.mark.parametrize("keying", ["3key", "2key"])
def test_4gib_both_kernels_both_directions(keying):
    """Encryption and decryption of the 4 GiB workload with each kernel, in
    place: the kernels agree on every byte in both directions, the oracle
    checks 2^22 seeded blocks of each direction, and each kernel's decryption
    of its own ciphertext restores the input."""
    key = inputs.key_triple(inputs.key_seed(CONFIG_ID), keying)
    ks = des3.des3_key_schedule(key)
    nblocks = NBYTES // 8
    plain = inputs.splitmix64_torch(inputs.data_seed(CONFIG_ID), 0, nblocks, "cuda")
    t = torch.from_numpy(_sample_idx(nblocks)).cuda()
    p = plain[t].cpu().numpy().view(np.uint8)
    for decrypt in (False, True):
        bs = plain.clone()
        sp = plain.clone()
        des3.des3_ecb_crypt_ex(ks, bs, bs, decrypt=decrypt, kernel="bitslice")
        des3.des3_ecb_crypt_ex(ks, sp, sp, decrypt=decrypt, kernel="sptable")
        torch.cuda.synchronize()
        assert torch.equal(bs, sp), (keying, decrypt)
        assert np.array_equal(bs[t].cpu().numpy().view(np.uint8), oracle.tdes_ecb(key, p, decrypt)), (keying, decrypt)
        des3.des3_ecb_crypt_ex(ks, bs, bs, decrypt=not decrypt, kernel="bitslice")
        des3.des3_ecb_crypt_ex(ks, sp, sp, decrypt=not decrypt, kernel="sptable")
        torch.cuda.synchronize()
        assert torch.equal(bs, plain) and torch.equal(sp, plain), (keying, decrypt)
        del bs, sp


def _sha256_device(t, piece=256 << 20):
    """SHA-256 of a device byte tensor, copied to the host piece by piece."""
    h = hashlib.sha256()
    for off in range(0, t.numel(), piece):
        h.update(t[off:off + piece].cpu().numpy().tobytes())
    return h.hexdigest()


@pytest.mark.parametrize("keying,decrypt", [("3key", False), ("3key", True), ("2key", False), ("2key", True)])
def test_4gib_whole_output_equals_the_oracle(keying, decrypt):
    """Every byte of the 4 GiB workload, through the benchmark's call (default
    kernel, in place), against the oracle's digest of the same workload
    (tests/golden/oracle_4gib_digests.json and, for the 2-key triple,
    oracle_4gib_2key_digests.json, written by make_full_4gib.py)."""
    name = "oracle_4gib_digests.json" if keying == "3key" else "oracle_4gib_2key_digests.json"
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", name)))
    key = inputs.key_triple(inputs.key_seed(CONFIG_ID), keying)
    assert gold["key"] == key.hex() and gold["nbytes"] == NBYTES
    assert gold["data_seed"] == inputs.data_seed(CONFIG_ID)
    ks = des3.des3_key_schedule(key)
    words = inputs.splitmix64_torch(inputs.data_seed(CONFIG_ID), 0, NBYTES // 8, "cuda")
    buf = words.view(torch.uint8)
    assert _sha256_device(buf) == gold["sha256_in"]
    if decrypt:
        des3.des3_ecb_decrypt(ks, buf, buf)
    else:
        des3.des3_ecb_encrypt(ks, buf, buf)
    torch.cuda.synchronize()
    assert _sha256_device(buf) == gold["sha256_decrypt" if decrypt else "sha256_encrypt"]


def test_beyond_4gib_ragged_64bit_offsets():
    """2^30 + 1 blocks (8 GiB + 8 bytes): block indices and byte offsets past
    2^32 on both kernels; the kernels agree everywhere, the oracle checks the
    blocks around the 4 GiB boundary and the end."""
    nblocks = (1 << 30) + 1
    key = inputs.key_triple(4444)
    ks = des3.des3_key_schedule(key)
    words = inputs.splitmix64_torch(4445, 0, nblocks, "cuda")
    plain_sample_idx = np.array([0, (1 << 29) - 1, 1 << 29, (1 << 29) + 1, (1 << 30) - 1, 1 << 30], dtype=np.int64)
    t = torch.from_numpy(plain_sample_idx).cuda()
    plain = words[t].cpu().numpy().view(np.uint8)
    bs = words.view(torch.uint8)
    sp = torch.empty_like(bs)
    des3.des3_ecb_crypt_ex(ks, bs, sp, decrypt=False, kernel="sptable")
    des3.des3_ecb_crypt_ex(ks, bs, bs, decrypt=False, kernel="bitslice")
    torch.cuda.synchronize()
    assert torch.equal(bs, sp)
    del sp
    got = words[t].cpu().numpy().view(np.uint8)
    assert np.array_equal(got, oracle.tdes_ecb(key, plain))
