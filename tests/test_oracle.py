"""Pins for the CPU oracle: structure of the standard's tables, agreement with
independent crypto libraries, and the algebraic properties DES is known to
have.  None of these re-types the oracle's own formulas."""
import hashlib
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import inputs

GOLDEN_DIR = os.path.join(os.path.dirname(__file__), "golden")


def _rand_bytes(seed, n):
    return inputs.data_bytes(seed, n).tobytes()


# ---------------------------------------------------------------- structure

def test_ip_fp_are_inverse_permutations():
    ip, fp = oracle.table("IP"), oracle.table("FP")
    assert sorted(ip) == list(range(1, 65))
    assert sorted(fp) == list(range(1, 65))
    # FP(IP(x)) = x: output bit i of FP is bit FP[i] of IP's output, which is input bit IP[FP[i]].
    assert [ip[fp[i] - 1] for i in range(64)] == list(range(1, 65))
    assert [fp[ip[i] - 1] for i in range(64)] == list(range(1, 65))


def test_p_is_permutation_and_e_covers_each_bit_once_or_twice():
    assert sorted(oracle.table("P")) == list(range(1, 33))
    e = oracle.table("E")
    counts = np.bincount(e, minlength=33)[1:]
    assert counts.min() == 1 and counts.max() == 2
    assert int((counts == 2).sum()) == 16
    # Each S-box sees a 6-bit window whose middle four bits are its own nibble.
    for j in range(8):
        assert e[6 * j + 1:6 * j + 5] == [4 * j + 1, 4 * j + 2, 4 * j + 3, 4 * j + 4]


def test_key_schedule_tables():
    pc1, pc2, sh = oracle.table("PC1"), oracle.table("PC2"), oracle.table("SHIFT")
    assert len(set(pc1)) == 56
    assert all(p % 8 != 0 for p in pc1)  # the parity bits 8,16,...,64 are never selected
    assert len(set(pc2)) == 48 and all(1 <= p <= 56 for p in pc2)
    # PC-2 draws its first 24 bits from C (1..28) and the rest from D (29..56).
    assert all(p <= 28 for p in pc2[:24]) and all(p > 28 for p in pc2[24:])
    assert sum(sh) == 28 and len(sh) == 16


def test_sbox_rows_are_permutations():
    s = np.array(oracle.table("SBOX")).reshape(8, 4, 16)
    for j in range(8):
        for r in range(4):
            assert sorted(s[j, r]) == list(range(16))


# ---------------------------------------------------- independent libraries

def _crypto_tdes(key, data, decrypt):
    mod = pytest.importorskip("cryptography.hazmat.decrepit.ciphers.algorithms")
    from cryptography.hazmat.primitives.ciphers import Cipher, modes
    c = Cipher(mod.TripleDES(key), modes.ECB())
    ctx = c.decryptor() if decrypt else c.encryptor()
    return ctx.update(data) + ctx.finalize()


@pytest.mark.parametrize("keying", ["3key", "2key", "1key"])
@pytest.mark.parametrize("decrypt", [False, True])
def test_matches_cryptography_library(keying, decrypt):
    for t in range(4):
        key = inputs.key_triple(1000 + t, keying)
        data = _rand_bytes(2000 + t, 8 * (1 + 97 * t))
        got = oracle.tdes_ecb(key, data, decrypt).tobytes()
        assert got == _crypto_tdes(key, data, decrypt)


def test_config1_digest_matches_cryptography_library():
    """The 1 MiB workload: the whole ciphertext agrees with the library."""
    key = inputs.key_triple(inputs.key_seed(1))
    data = inputs.data_bytes(inputs.data_seed(1), 1 << 20).tobytes()
    ours = oracle.tdes_ecb(key, data).tobytes()
    assert ours == _crypto_tdes(key, data, False)


@pytest.mark.skipif(shutil.which("openssl") is None, reason="openssl CLI not installed")
@pytest.mark.parametrize("decrypt", [False, True])
def test_matches_openssl_cli(decrypt):
    key = inputs.key_triple(77)
    data = _rand_bytes(78, 8 * 513)
    cmd = ["openssl", "enc", "-des-ede3", "-nopad", "-K", key.hex()]
    if decrypt:
        cmd.append("-d")
    res = subprocess.run(cmd, input=data, capture_output=True)
    if res.returncode != 0:
        pytest.skip("openssl des-ede3 unavailable: %s" % res.stderr[:200])
    assert oracle.tdes_ecb(key, data, decrypt).tobytes() == res.stdout


# ------------------------------------------------------- algebraic properties

def test_round_trip():
    for t in range(3):
        key = inputs.key_triple(300 + t)
        data = _rand_bytes(400 + t, 8 * 1000)
        ct = oracle.tdes_ecb(key, data)
        assert ct.tobytes() != data
        assert oracle.tdes_ecb(key, ct, decrypt=True).tobytes() == data


def test_single_des_round_trip_and_three_equal_keys_reduce_to_des():
    key = inputs.key_triple(55)[:8]
    data = _rand_bytes(56, 8 * 300)
    ct = oracle.des_ecb(key, data)
    assert oracle.des_ecb(key, ct, decrypt=True).tobytes() == data
    assert oracle.tdes_ecb(key * 3, data).tobytes() == ct.tobytes()
    assert oracle.tdes_ecb(key * 3, ct, decrypt=True).tobytes() == data


def test_two_key_composition_is_e_d_e():
    k = inputs.key_triple(91)
    k1, k2 = k[:8], k[8:16]
    data = _rand_bytes(92, 8 * 64)
    step = oracle.des_ecb(k1, data)
    step = oracle.des_ecb(k2, step, decrypt=True)
    step = oracle.des_ecb(k1, step)
    assert oracle.tdes_ecb(k1 + k2 + k1, data).tobytes() == step.tobytes()


def test_complementation_property():
    """E_{~k}(~x) = ~E_k(x), for DES and for 3DES with all three keys complemented."""
    data = np.frombuffer(_rand_bytes(60, 8 * 256), dtype=np.uint8)
    key = np.frombuffer(inputs.key_triple(61), dtype=np.uint8)
    c = oracle.des_ecb(key[:8], data)
    cc = oracle.des_ecb(~key[:8], ~data)
    assert np.array_equal(cc, ~c)
    t = oracle.tdes_ecb(key, data)
    tc = oracle.tdes_ecb(~key, ~data)
    assert np.array_equal(tc, ~t)


def _key_from_cd(c0: int, d0: int) -> bytes:
    """Invert PC-1: place the 56 bits C0||D0 at their key positions and set
    each byte's low bit for odd parity."""
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


ALT0 = int("01" * 14, 2)
ALT1 = int("10" * 14, 2)
ONES = (1 << 28) - 1


def test_weak_keys_are_involutions():
    data = _rand_bytes(70, 8 * 128)
    for c0 in (0, ONES):
        for d0 in (0, ONES):
            k = _key_from_cd(c0, d0)
            ks = oracle.des_key_schedule(k)
            assert len(set(ks)) == 1  # all sixteen round keys equal
            once = oracle.des_ecb(k, data)
            assert once.tobytes() != data
            assert oracle.des_ecb(k, once).tobytes() == data


def test_semi_weak_pairs():
    """Keys whose C0, D0 are constant or alternating: encrypting with k then
    with its partner (alternating halves flipped in phase) is the identity."""
    data = _rand_bytes(71, 8 * 128)
    pats = [0, ONES, ALT0, ALT1]
    flip = {0: 0, ONES: ONES, ALT0: ALT1, ALT1: ALT0}
    n = 0
    for c0 in pats:
        for d0 in pats:
            if c0 in (0, ONES) and d0 in (0, ONES):
                continue
            k, kp = _key_from_cd(c0, d0), _key_from_cd(flip[c0], flip[d0])
            assert k != kp
            ks, ksp = oracle.des_key_schedule(k), oracle.des_key_schedule(kp)
            assert ksp == ks[::-1]
            assert oracle.des_ecb(kp, oracle.des_ecb(k, data)).tobytes() == data
            n += 1
    assert n == 12


def test_parity_bits_are_ignored():
    key = bytearray(inputs.key_triple(80))
    data = _rand_bytes(81, 8 * 64)
    ref = oracle.tdes_ecb(bytes(key), data).tobytes()
    flipped = bytes(b ^ 1 for b in key)
    assert oracle.tdes_ecb(flipped, data).tobytes() == ref


def test_rejects_ragged_length():
    with pytest.raises(ValueError):
        oracle.tdes_ecb(bytes(24), bytes(12))


def test_empty_input():
    assert oracle.tdes_ecb(bytes(24), b"").size == 0


# ------------------------------------------------------------- golden files

def test_golden_digests_reproduce_and_match_library():
    """tests/golden/oracle_digests.json is written by make_golden.py from the
    oracle alone; it must still reproduce, and the independent library must
    agree with it."""
    with open(os.path.join(GOLDEN_DIR, "oracle_digests.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        key = bytes.fromhex(case["key"])
        data = inputs.data_bytes(case["data_seed"], case["nbytes"]).tobytes()
        assert hashlib.sha256(data).hexdigest() == case["sha256_in"]
        out = oracle.tdes_ecb(key, data, case["decrypt"]).tobytes()
        assert hashlib.sha256(out).hexdigest() == case["sha256_out"]
        if case["nbytes"] <= (1 << 20):
            try:
                ref = _crypto_tdes(key, data, case["decrypt"])
            except pytest.skip.Exception:
                continue
            assert hashlib.sha256(ref).hexdigest() == case["sha256_out"]


# ----------------------------------------------------------- input streams

def test_splitmix64_implementations_agree():
    seed = 0xDE5C0DE1
    ref = [inputs.splitmix64_scalar(seed, i) for i in range(50)]
    assert [int(v) for v in inputs.splitmix64(seed, 0, 50)] == ref
    assert [int(v) for v in inputs.splitmix64_at(seed, np.arange(50))] == ref
    assert [int(v) for v in inputs.splitmix64(seed, 20, 30)] == ref[20:]
    # The sequential definition: state += golden; output = mix(state).
    s = seed
    seq = []
    for _ in range(50):
        s = (s + inputs.GOLDEN) & inputs.MASK64
        z = s
        z = ((z ^ (z >> 30)) * inputs.M1) & inputs.MASK64
        z = ((z ^ (z >> 27)) * inputs.M2) & inputs.MASK64
        seq.append(z ^ (z >> 31))
    assert seq == ref


def test_splitmix64_torch_matches_numpy():
    torch = pytest.importorskip("torch")
    t = inputs.splitmix64_torch(123456789, 5, 1000, "cpu", chunk=300)
    n = inputs.splitmix64(123456789, 5, 1000)
    assert np.array_equal(t.numpy().view(np.uint64), n)


def test_keys_have_odd_parity():
    for keying in ("3key", "2key", "1key"):
        k = inputs.key_triple(5, keying)
        assert len(k) == 24
        assert all(bin(b).count("1") % 2 == 1 for b in k)
    assert inputs.key_triple(5, "2key")[16:] == inputs.key_triple(5, "2key")[:8]


# ------------------------------------------------ CBC and CTR (extension)

def _crypto_tdes_cbc(key, iv, data, decrypt):
    mod = pytest.importorskip("cryptography.hazmat.decrepit.ciphers.algorithms")
    from cryptography.hazmat.primitives.ciphers import Cipher, modes
    c = Cipher(mod.TripleDES(key), modes.CBC(iv))
    ctx = c.decryptor() if decrypt else c.encryptor()
    return ctx.update(data) + ctx.finalize()


@pytest.mark.parametrize("decrypt", [False, True])
def test_cbc_matches_cryptography_library(decrypt):
    for t in range(3):
        key = inputs.key_triple(1100 + t)
        iv = _rand_bytes(1200 + t, 8)
        data = _rand_bytes(1300 + t, 8 * (1 + 301 * t))
        assert oracle.tdes_cbc(key, iv, data, decrypt).tobytes() == _crypto_tdes_cbc(key, iv, data, decrypt)


@pytest.mark.skipif(shutil.which("openssl") is None, reason="openssl CLI not installed")
def test_cbc_matches_openssl_cli():
    key, iv, data = inputs.key_triple(1400), _rand_bytes(1401, 8), _rand_bytes(1402, 8 * 77)
    res = subprocess.run(["openssl", "enc", "-des-ede3-cbc", "-nopad", "-K", key.hex(), "-iv", iv.hex()],
                         input=data, capture_output=True)
    if res.returncode != 0:
        pytest.skip("openssl des-ede3-cbc unavailable")
    assert oracle.tdes_cbc(key, iv, data).tobytes() == res.stdout


def test_cbc_round_trip_and_first_block_is_ecb_of_xor():
    key, iv, data = inputs.key_triple(1500), _rand_bytes(1501, 8), _rand_bytes(1502, 8 * 50)
    ct = oracle.tdes_cbc(key, iv, data)
    assert oracle.tdes_cbc(key, iv, ct, decrypt=True).tobytes() == data
    x = bytes(a ^ b for a, b in zip(data[:8], iv))
    assert ct[:8].tobytes() == oracle.tdes_ecb(key, x).tobytes()


def _counter_blocks(ctr0: bytes, n: int) -> bytes:
    t0 = int.from_bytes(ctr0, "big")
    return b"".join(((t0 + i) % (1 << 64)).to_bytes(8, "big") for i in range(n))


@pytest.mark.parametrize("start", [0, 12345, (1 << 64) - 5, (1 << 32) - 3])
def test_ctr_is_xor_with_library_ecb_of_counter_blocks(start):
    """CTR reduces to ECB of the counter sequence (computed here with the
    independent library), XORed into the data; includes the 2^32 and 2^64
    carries of the big-endian increment."""
    key = inputs.key_triple(1600)
    ctr0 = start.to_bytes(8, "big")
    data = _rand_bytes(1601, 8 * 40)
    ks = _crypto_tdes(key, _counter_blocks(ctr0, 40), False)
    want = bytes(a ^ b for a, b in zip(data, ks))
    assert oracle.tdes_ctr(key, ctr0, data).tobytes() == want


def test_ctr_is_an_involution():
    key, ctr0, data = inputs.key_triple(1700), _rand_bytes(1701, 8), _rand_bytes(1702, 8 * 999)
    once = oracle.tdes_ctr(key, ctr0, data)
    assert once.tobytes() != data
    assert oracle.tdes_ctr(key, ctr0, once).tobytes() == data
