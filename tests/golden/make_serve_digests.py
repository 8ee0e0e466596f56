"""Write tests/golden/oracle_serve_digests.json: the CPU oracle over the
serving test's sample of the serving workload, every request in order.

The sample: 2000 requests whose sizes (log-normal, median 256 KiB, sigma 1.5,
clamped to [4 KiB, 64 MiB], rounded down to 8 bytes), key indices (uniform
over 10000 cached triples) and directions (Bernoulli(0.5)) come from
inputs.serve_recipe with data seed 0xDE5C0DE5; the 10000 parity-adjusted
3-key triples from key seed 0x3DEA.  Request i reads its bytes from one
arena of SplitMix64 words (seed 0xDE5C0DE5 + 7) at the 256-byte-aligned
offsets of inputs.arena_offsets.  Its result is 3DES-EDE ECB encryption, or
decryption when its flag is set, under its triple (paper Sec. II.A; ECB:
abstract and Fig. 2).

Stored: SHA-256 of every request's input and of every request's output,
concatenated in request order, and of the outputs of each run of 100
requests.  tests/test_gpu_serve.py serves the same sample through the
continuous-batching server and hashes the results the same way.

Only oracle/ and the seeded input generator are called.  Run from the
repository root:
    python tests/golden/make_serve_digests.py
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

CONFIG_ID = 5
NREQ = 2000
NKEYS = 10000
GROUP = 100


def main():
    sizes, kidx, dec, _ = inputs.serve_recipe(inputs.data_seed(CONFIG_ID), NREQ)
    keys = inputs.key_triples(inputs.key_seed(CONFIG_ID), NKEYS)
    offs, arena_bytes = inputs.arena_offsets(sizes)
    seed = inputs.data_seed(CONFIG_ID) + 7
    h_in, h_out = hashlib.sha256(), hashlib.sha256()
    groups = []
    g = hashlib.sha256()
    t0 = time.time()
    for i, (n, o) in enumerate(zip(sizes, offs)):
        data = inputs.data_bytes(seed, int(n), start_block=o // 8)
        out = oracle.tdes_ecb(keys[int(kidx[i])], data, bool(dec[i])).tobytes()
        h_in.update(data.tobytes())
        h_out.update(out)
        g.update(out)
        if (i + 1) % GROUP == 0 or i + 1 == NREQ:
            groups.append(g.hexdigest())
            g = hashlib.sha256()
    doc = {
        "what": "SHA-256 digests of the CPU oracle's 3DES-EDE ECB output over the serving test's 2000 requests",
        "source": "written by tests/golden/make_serve_digests.py, which calls only oracle/ and the seeded input "
                  "generator",
        "cites": "3DES-EDE composition: paper Sec. II.A; ECB: paper abstract and Fig. 2",
        "data_seed": inputs.data_seed(CONFIG_ID),
        "arena_seed": seed,
        "key_seed": inputs.key_seed(CONFIG_ID),
        "nreq": NREQ,
        "nkeys": NKEYS,
        "total_bytes": int(sizes.sum()),
        "arena_bytes": arena_bytes,
        "sha256_in": h_in.hexdigest(),
        "sha256_out": h_out.hexdigest(),
        "group_requests": GROUP,
        "sha256_out_groups": groups,
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.max_threads(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_serve_digests.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
