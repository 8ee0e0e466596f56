"""Keep the smallest verified LOP3 circuit per S-box over several sboxgen runs.

Each input is a JSON list of {"sbox", "gates", "outputs"} objects written by
sboxgen (a run may cover all eight S-boxes or one).  Every candidate is first
polished by resubstitution (a gate that three other nodes outside its fanout
also compute is redefined on them, and gates that no longer feed an output
are dropped), then re-verified on all 64 inputs against the S-box table of
des_tables.h; the smallest per S-box go to sbox_circuits.json.

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


ALL = (1 << 64) - 1


def _input_tt(m):
    return sum(1 << p for p in range(64) if (p >> (5 - m)) & 1)


def _eval_lut(a, b, c, imm):
    r = 0
    for k in range(8):
        if (imm >> k) & 1:
            r |= (a if k & 4 else ~a & ALL) & (b if k & 2 else ~b & ALL) & (c if k & 1 else ~c & ALL)
    return r


def _lut_fit(a, b, c, target):
    imm = 0
    for k in range(8):
        sel = (a if k & 4 else ~a & ALL) & (b if k & 2 else ~b & ALL) & (c if k & 1 else ~c & ALL)
        if sel & target:
            if sel & ~target & ALL:
                return -1
            imm |= 1 << k
    return imm


def _normalise(gates, outs):
    """Topological order and dead-gate removal; None on a cycle."""
    ins = {6 + i: g[:3] for i, g in enumerate(gates)}
    imm = {6 + i: g[3] for i, g in enumerate(gates)}
    stack = [r >> 1 for r in outs]
    need = set()
    while stack:
        x = stack.pop()
        if x in need or x < 6:
            continue
        need.add(x)
        stack.extend(ins[x])
    order, done = list(range(6)), set(range(6))
    pending = sorted(need)
    while pending:
        nxt = [x for x in pending if all(i in done for i in ins[x])]
        if not nxt:
            return None
        for x in nxt:
            order.append(x)
            done.add(x)
        pending = [x for x in pending if x not in done]
    pos = {x: i for i, x in enumerate(order)}
    new_gates = [[pos[i] for i in ins[x]] + [imm[x]] for x in order[6:]]
    new_outs = [2 * pos[r >> 1] + (r & 1) for r in outs]
    return new_gates, new_outs


def polish(c):
    """Resubstitution to a fixpoint; returns a circuit no larger than c."""
    gates, outs = [list(g) for g in c["gates"]], list(c["outputs"])
    improved = True
    while improved:
        improved = False
        tt = [_input_tt(m) for m in range(6)]
        for g in gates:
            tt.append(_eval_lut(tt[g[0]], tt[g[1]], tt[g[2]], g[3]))
        n = len(tt)
        for gi in range(len(gates)):
            node = 6 + gi
            tfo = {node}
            for x in range(node + 1, n):
                if any(i in tfo for i in gates[x - 6][:3]):
                    tfo.add(x)
            cand = [x for x in range(n) if x not in tfo]
            found = None
            for i in range(len(cand)):
                for j in range(i, len(cand)):
                    for k in range(j, len(cand)):
                        a, b, cc = cand[i], cand[j], cand[k]
                        if [a, b, cc] == gates[gi][:3]:
                            continue
                        imm = _lut_fit(tt[a], tt[b], tt[cc], tt[node])
                        if imm < 0:
                            continue
                        trial = [list(g) for g in gates]
                        trial[gi] = [a, b, cc, imm]
                        res = _normalise(trial, outs)
                        if res and len(res[0]) < len(gates):
                            found = res
                            break
                    if found:
                        break
                if found:
                    break
            if found:
                gates, outs = found
                improved = True
                break
    return {"sbox": c["sbox"], "gates": gates, "outputs": outs}


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
            p = polish(c)
            if len(p["gates"]) < len(c["gates"]) and verify(p, S):
                print("%s: S%d polished %d -> %d gates" % (f, c["sbox"], len(c["gates"]), len(p["gates"])))
                c = p
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
