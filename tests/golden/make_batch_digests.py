"""Write tests/golden/oracle_batch_digests.json: the CPU oracle over the whole
batched workload, 4096 buffers in job order.

The workload: sizes log-uniform on [512 B, 16 MiB] rounded down to 8 bytes
and directions Bernoulli(0.5), both from data seed 0xDE5C0DE4; one
parity-adjusted 3-key triple per buffer from key seed 0x3DE9; buffers laid out
back to back in one arena at 256-byte boundaries, each holding the arena's
SplitMix64 words (inputs.batch_recipe, inputs.key_triples,
inputs.arena_offsets).  Job i is 3DES-EDE ECB encryption, or decryption when
its flag is set, of buffer i under triple i (paper Sec. II.A; ECB: abstract and
Fig. 2).

Stored: SHA-256 of every job's input concatenated in job order, of every
job's output concatenated in job order, and of the outputs of each run of 256
consecutive jobs (to name the failing range).  The GPU test hashes the
batched plan's outputs the same way.

Only oracle/ and the seeded input generator are called.  About 9 minutes on 8
x86 cores.  Run from the repository root:
    python tests/golden/make_batch_digests.py
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

CONFIG_ID = 4
GROUP = 256


def main():
    seed = inputs.data_seed(CONFIG_ID)
    sizes, dec = inputs.batch_recipe(seed)
    keys = inputs.key_triples(inputs.key_seed(CONFIG_ID), len(sizes))
    offs, arena_bytes = inputs.arena_offsets(sizes)
    h_in, h_out = hashlib.sha256(), hashlib.sha256()
    groups = []
    g = hashlib.sha256()
    t0 = time.time()
    for i, (n, o) in enumerate(zip(sizes, offs)):
        data = inputs.data_bytes(seed, int(n), start_block=o // 8)
        out = oracle.tdes_ecb(keys[i], data, bool(dec[i])).tobytes()
        h_in.update(data.tobytes())
        h_out.update(out)
        g.update(out)
        if (i + 1) % GROUP == 0 or i + 1 == len(sizes):
            groups.append(g.hexdigest())
            g = hashlib.sha256()
            print("%d jobs done, %.0f s" % (i + 1, time.time() - t0), flush=True)
    doc = {
        "what": "SHA-256 digests of the CPU oracle's 3DES-EDE ECB output over the whole batched workload, job order",
        "source": "written by tests/golden/make_batch_digests.py, which calls only oracle/ and the seeded input "
                  "generator",
        "cites": "3DES-EDE composition: paper Sec. II.A; ECB: paper abstract and Fig. 2",
        "data_seed": seed,
        "key_seed": inputs.key_seed(CONFIG_ID),
        "njobs": len(sizes),
        "total_bytes": int(sizes.sum()),
        "arena_bytes": arena_bytes,
        "decrypt_jobs": int(dec.sum()),
        "sha256_in": h_in.hexdigest(),
        "sha256_out": h_out.hexdigest(),
        "group_jobs": GROUP,
        "sha256_out_groups": groups,
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.max_threads(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_batch_digests.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
        f.write("\n")
    print("wrote", path)


if __name__ == "__main__":
    main()
