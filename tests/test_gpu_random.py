"""Seeded random cases across the entry points, each against the oracle:
sizes from one block to 40 000 blocks, buffer offsets on every 8-byte
boundary of a 128-byte window, in place and out of place, 3-key / 2-key /
single-DES keys, both directions, every kernel choice, CTR counters and CBC
IVs drawn at random, and random batches.  The cases are drawn from one
SplitMix64 stream, so a failure names a reproducible case index."""
import numpy as np
import pytest

import oracle
from paper_1305_4376_gb300 import des3, inputs

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NCASES = 120


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1305_4376_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    des3.lib()


def _case(i):
    w = inputs.splitmix64(0x5EED0000 + i, 0, 16)
    nblocks = int(1 + (w[0] % 40000 if w[1] % 4 else w[0] % 70))
    return {
        "nblocks": nblocks,
        "off_in": int(8 * (w[2] % 16)),
        "off_out": int(8 * (w[3] % 16)),
        "in_place": bool(w[4] % 3 == 0),
        "keying": ["3key", "2key", "1key", "des"][int(w[5] % 4)],
        "decrypt": bool(w[6] & 1),
        "kernel": ["auto", "bitslice", "sptable"][int(w[7] % 3)],
        "mode": ["ecb", "ecb", "ctr", "cbc"][int(w[8] % 4)],
        "seed": int(w[9] % (1 << 30)),
    }


def _device(a, offset):
    buf = torch.zeros(a.size + offset + 64, dtype=torch.uint8, device="cuda")
    view = buf[offset:offset + a.size]
    view.copy_(torch.from_numpy(a))
    return buf, view


@pytest.mark.parametrize("i", range(NCASES))
def test_random_case_matches_the_oracle(i):
    c = _case(i)
    data = inputs.data_bytes(c["seed"], 8 * c["nblocks"])
    if c["keying"] == "des":
        key = inputs.key_triple(c["seed"] + 1)[:8]
        ks = des3.des3_key_schedule_des(key)
        key24 = key * 3
    else:
        key24 = inputs.key_triple(c["seed"] + 1, c["keying"])
        ks = des3.des3_key_schedule(key24)
    iv = inputs.data_bytes(c["seed"] + 2, 8).tobytes()
    _bi, src = _device(data, c["off_in"])
    if c["in_place"] and c["mode"] != "cbc":
        dst = src
    else:
        _bo, dst = _device(np.zeros_like(data), c["off_out"])
    if c["mode"] == "ecb":
        des3.des3_ecb_crypt_ex(ks, src, dst, src.numel(), c["decrypt"], c["kernel"])
        ref = oracle.tdes_ecb(key24, data, c["decrypt"])
    elif c["mode"] == "ctr":
        des3.des3_ctr_crypt(ks, iv, src, dst)
        ref = oracle.tdes_ctr(key24, iv, data)
    else:
        des3.des3_cbc_decrypt(ks, iv, src, dst)
        ref = oracle.tdes_cbc(key24, iv, data, decrypt=True)
    torch.cuda.synchronize()
    assert np.array_equal(dst.cpu().numpy(), ref), c


@pytest.mark.parametrize("i", range(12))
def test_random_batch_matches_the_oracle(i):
    """Random batches: 1 to 64 jobs, sizes 0 to 200 000 bytes, a random key
    each from a small pool, random directions, some jobs in place."""
    w = inputs.splitmix64(0xBA7C0000 + i, 0, 4 + 4 * 64)
    njobs = int(1 + w[0] % 64)
    nkeys = int(1 + w[1] % 5)
    keys = inputs.key_triples(int(w[2] % (1 << 30)), nkeys)
    kss = [des3.des3_key_schedule(k) for k in keys]
    specs, pos = [], 0
    for j in range(njobs):
        n = int(8 * (w[4 + 4 * j] % 25000))
        specs.append((pos, n, int(w[5 + 4 * j] % nkeys), bool(w[6 + 4 * j] & 1), bool(w[7 + 4 * j] % 4 == 0)))
        pos += (n + 8 + 255) // 256 * 256
    data = inputs.data_bytes(int(w[3] % (1 << 30)), pos)
    src = torch.from_numpy(data).cuda()
    out = torch.zeros_like(src)
    jobs = []
    for o, n, k, d, inplace in specs:
        dst = src[o:o + n] if inplace else out[o:o + n]
        jobs.append((src[o:o + n], dst, n, k, d))
    des3.des3_ecb_batch(des3.make_keys(kss), des3.make_jobs(jobs))
    torch.cuda.synchronize()
    s, t = src.cpu().numpy(), out.cpu().numpy()
    for o, n, k, d, inplace in specs:
        got = s[o:o + n] if inplace else t[o:o + n]
        assert np.array_equal(got, oracle.tdes_ecb(keys[k], data[o:o + n], d)), (i, o, n, k, d, inplace)
