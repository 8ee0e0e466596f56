"""Write tests/golden/oracle_4gib_digests.json: the CPU oracle over the whole
4 GiB single-buffer workload (2^29 blocks, SplitMix64 data seed 0xDE5C0DE2,
one parity-adjusted 3-key triple from key seed 0x3DE7), encrypted and
decrypted, as SHA-256 digests of the input and of each output.

With ``--keying 2key`` the key is the 2-key triple K1||K2||K1 drawn from the
same seed (keying option 2 of NIST SP 800-67) and the file written is
tests/golden/oracle_4gib_2key_digests.json.

The oracle runs over the workload in 256 MiB pieces (ECB blocks are
independent, paper abstract and Fig. 2) and the digests are taken over the
concatenated bytes, so the GPU test can compare the full 4 GiB output of the
benchmark's call with the oracle's without holding a second copy.

Only oracle/ and the seeded input generator are called.  It takes a few
minutes on 16 cores.  Run from the repository root:
    python tests/golden/make_full_4gib.py [--keying 2key] [extra copy path ...]
"""
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1305_4376_gb300 import inputs  # noqa: E402

CONFIG_ID = 2
NBYTES = 4 << 30
PIECE = 256 << 20


def main():
    args = sys.argv[1:]
    keying = "3key"
    if args[:1] == ["--keying"]:
        keying, args = args[1], args[2:]
    key = inputs.key_triple(inputs.key_seed(CONFIG_ID), keying)
    h_in = hashlib.sha256()
    h_out = {False: hashlib.sha256(), True: hashlib.sha256()}
    t0 = time.time()
    for off in range(0, NBYTES, PIECE):
        data = inputs.data_bytes(inputs.data_seed(CONFIG_ID), PIECE, start_block=off // 8)
        h_in.update(data.tobytes())
        for decrypt in (False, True):
            h_out[decrypt].update(oracle.tdes_ecb(key, data, decrypt).tobytes())
        print("%d MiB done, %.0f s" % ((off + PIECE) >> 20, time.time() - t0), flush=True)
    doc = {
        "what": "SHA-256 digests of the CPU oracle's 3DES-EDE ECB output over the whole 4 GiB workload",
        "source": "written by tests/golden/make_full_4gib.py, which calls only oracle/ and the seeded input generator",
        "cites": "3DES-EDE composition: paper Sec. II.A; ECB: paper abstract and Fig. 2",
        "data_seed": inputs.data_seed(CONFIG_ID),
        "key_seed": inputs.key_seed(CONFIG_ID),
        "keying": keying,
        "key": key.hex(),
        "nbytes": NBYTES,
        "sha256_in": h_in.hexdigest(),
        "sha256_encrypt": h_out[False].hexdigest(),
        "sha256_decrypt": h_out[True].hexdigest(),
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.max_threads(),
    }
    name = "oracle_4gib_digests.json" if keying == "3key" else "oracle_4gib_%s_digests.json" % keying
    paths = [os.path.join(os.path.dirname(os.path.abspath(__file__)), name)]
    paths += args  # optional extra copies
    for path in paths:
        with open(path, "w") as f:
            json.dump(doc, f, indent=1)
            f.write("\n")
        print("wrote", path)


if __name__ == "__main__":
    main()
