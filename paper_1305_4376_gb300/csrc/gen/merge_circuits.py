"""Keep the smallest verified LOP3 circuit per S-box over several sboxgen runs.

Each input is a JSON list of {"sbox", "gates", "outputs"} objects written by
sboxgen (a run may cover all eight S-boxes or one).  Every candidate is
re-verified here on all 64 inputs against the S-box table of des_tables.h
before it can win; the winners go to sbox_circuits.json.

    python merge_circuits.py run1.json run2.json ... [--out sbox_circuits.json]
"""
import json
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def sbox_table():
    src = open(os.path.join(HERE, "..", "des_tables.h")).read()
    body = re.search(r"constexpr uint8_t kS\[8\]\[4\]\[16\] = \{(.*?)\};", src, re.S).group(1)
    nums = [int(x) for x in re.findall(r"\d+", body)]
    assert len(nums) == 512
    return [[nums[64 * j + 16 * r:64 * j + 16 * r + 16] for r in range(4)] for j in range(8)]


def verify(c, S):
    j = c["sbox"] - 1
    for x in range(64):
        val = [(x >> (5 - m)) & 1 for m in range(6)]
        for a, b, cc, imm in c["gates"]:
            val.append((imm >> (4 * val[a] + 2 * val[b] + val[cc])) & 1)
        s = S[j][((x >> 5) & 1) * 2 + (x & 1)][(x >> 1) & 15]
        for t, r in enumerate(c["outputs"]):
            if val[r >> 1] ^ (r & 1) != (s >> (3 - t)) & 1:
                return False
    return True


def main(argv):
    out = os.path.join(HERE, "sbox_circuits.json")
    files = []
    i = 0
    while i < len(argv):
        if argv[i] == "--out":
            out = argv[i + 1]
            i += 2
        else:
            files.append(argv[i])
            i += 1
    S = sbox_table()
    best = {}
    for f in files:
        try:
            cands = json.load(open(f))
        except (OSError, ValueError):
            continue
        for c in cands:
            if not verify(c, S):
                raise SystemExit("%s: circuit for S%d fails verification" % (f, c["sbox"]))
            k = c["sbox"]
            if k not in best or len(c["gates"]) < len(best[k]["gates"]):
                best[k] = c
    missing = [k for k in range(1, 9) if k not in best]
    if missing:
        raise SystemExit("no circuit for S-boxes %s" % missing)
    res = [best[k] for k in range(1, 9)]
    with open(out, "w") as fh:
        fh.write("[\n" + ",\n".join(" " + json.dumps(c) for c in res) + "\n]\n")
    print("S-box gate counts:", [len(c["gates"]) for c in res], "total", sum(len(c["gates"]) for c in res))


if __name__ == "__main__":
    main(sys.argv[1:])
