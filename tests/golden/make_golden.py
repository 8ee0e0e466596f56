"""Write tests/golden/oracle_digests.json from the CPU oracle alone.

Each case names its seeded input (SplitMix64 data seed, size, key) and stores
SHA-256 digests of the input and of the oracle's output.  The digests freeze
the oracle's results so a later change to it is noticed; the tests also check
them against an independent crypto library where one is installed.

Run from the repository root:  python tests/golden/make_golden.py
"""
import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1305_4376_gb300 import inputs  # noqa: E402


def main():
    cases = []
    specs = [
        # (label, config id, nbytes, keying, decrypt)
        ("1 MiB, 3-key, encrypt", 1, 1 << 20, "3key", False),
        ("1 MiB, 3-key, decrypt", 1, 1 << 20, "3key", True),
        ("64 KiB, 2-key, encrypt", 3, 64 << 10, "2key", False),
        ("64 KiB, 2-key, decrypt", 3, 64 << 10, "2key", True),
        ("8 bytes, 3-key, encrypt", 1, 8, "3key", False),
        ("1016 bytes (127 blocks), 3-key, encrypt", 2, 1016, "3key", False),
    ]
    for label, cid, nbytes, keying, decrypt in specs:
        key = inputs.key_triple(inputs.key_seed(cid), keying)
        data = inputs.data_bytes(inputs.data_seed(cid), nbytes)
        out = oracle.tdes_ecb(key, data, decrypt)
        cases.append({
            "label": label,
            "data_seed": inputs.data_seed(cid),
            "key_seed": inputs.key_seed(cid),
            "keying": keying,
            "key": key.hex(),
            "nbytes": nbytes,
            "decrypt": decrypt,
            "sha256_in": hashlib.sha256(data.tobytes()).hexdigest(),
            "sha256_out": hashlib.sha256(out.tobytes()).hexdigest(),
        })
    doc = {
        "what": "SHA-256 digests of the CPU oracle's 3DES-EDE ECB output on seeded inputs",
        "source": "written by tests/golden/make_golden.py, which calls only oracle/ and the seeded input generator",
        "cites": "3DES-EDE composition: paper Sec. II.A; ECB: paper abstract and Fig. 2",
        "cases": cases,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_digests.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
