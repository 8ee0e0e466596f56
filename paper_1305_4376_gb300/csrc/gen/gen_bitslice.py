"""Generate bs_generated.cuh, the straight-line round code of the bitsliced kernel.

Inputs:
  * ../des_tables.h      -- the library's copy of the DES tables (IP, FP, E, P)
  * sbox_circuits.json   -- LOP3 circuits for S1..S8, found by this project's
                            circuit search (a working tool kept outside the
                            library); each is checked here against the
                            S-box table on all 64 inputs before any code is
                            written (and again by des3_self_test()).  An
                            S-box may carry a second circuit under "fold",
                            used by the folded rounds (below) where it needs
                            fewer instructions once its folds are counted.

Bitsliced layout (one CUDA thread = 32 blocks):
  w[p], p = 0..63, is the bit plane of little-endian bit p of the 64-bit
  block word (byte p/8, bit p%8 counted from the least significant end); bit m
  of w[p] belongs to the thread's m-th block.  DES numbers bits 1..64 from the
  most significant bit of byte 0, so DES bit n lives in plane
  slot(n) = 8*((n-1)//8) + 7 - (n-1)%8.

IP and FP are therefore free: L0[i] is the plane slot(IP[i]) and R0[i] is
slot(IP[32+i]).  The rounds update those planes in place:
  round_A:  L ^= f(R, K)      round_B:  R ^= f(L, K)
and the 3DES pipeline is stage 1 = (A B) x 8, stage 2 = (B A) x 8,
stage 3 = (A B) x 8 (after each DES the halves swap, and FP followed by the
next IP cancels; paper Sec. II.A composes the three DES operations).  The
result R16||L16 goes through FP, which again is only a renaming of planes,
emitted as bs_final_perm().

f(R, K) = P(S(E(R) xor K)): E and P are renamings as well, so the only
instructions are the key XORs, the S-box circuits and the XOR of each S-box
output into its destination plane.

Key absorption: the key bits of a round are all-ones or all-zeros words (one
key for all 32 blocks), so instead of XORing 48 key words into the S-box
inputs every round, every plane is STORED XORed with the key bit of its next
use as an S-box input (its first E position).  The 16 bits E duplicates need
one XOR at their second position (with k_first ^ k_second), and the update
of a destination plane becomes one 3-input XOR that also swaps its stored
mask for the one of its next use: new = old ^ out ^ (mask_old ^ mask_new).
Per round: 16 + gates + 32 instructions instead of 48 + gates + 32.  The
masks are a fixed function of the round keys (bs_mask_bits(), host side):
per round 16 corrections then 32 deltas, and five 32-word remasks at the
start of each DES (the half used as source in two rounds in a row) and at
the end (unmask; the R-planes' unmask is always zero, since the last round
writes them with no later use, so the kernel applies only the L-planes').

The 16 corrections are x ^ c with c all-ones or all-zeros, which equals
x * s + c with s = c | 1 (s = 1 or -1); with --imad they are emitted as
that multiply-add, which runs on the FMA pipe and so leaves the ALU pipe,
the kernel's bottleneck, 16 instructions per round lighter.

Folded outputs: where an S-box output's circuit has a gate with an input its
truth table ignores, on a chain of single-reader gates that are XOR-linear
in it up to the output (find_folds), the destination plane enters that
input and the output node becomes out ^ old.  The update is then only the
mask change, x ^ delta, which runs as the multiply-add x * s + delta on the
FMA pipe: one ALU instruction per folded output and round fewer.  Its
multiplier s = delta | 1 is an extra mask word per round, expanded from the
delta's own key bit, so the key masks the host packs do not change.  Every
fold is checked on all 64 inputs and both values of each plane (--no-fold
emits none).  Both variants are emitted: bs_round_A/B unfolded (the batched
kernel) and bs_round_A_f/B_f folded (the single-buffer kernel), each with
its mask layout.

The round code lists the eight circuits' gates interleaved by depth (all
depth-1 gates of S1..S8, then all depth-2 gates, ...), which measured 0.4 %
faster on a single buffer and 1.2 % faster in the batched kernel than one
S-box after another (--sequential).

Run:  python gen_bitslice.py [--imad] [--sequential] [--no-fold]   (writes ../bs_generated.cuh)
"""
import json
import os
import re
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(HERE, "..", "des_tables.h")
CIRCUITS = os.path.join(HERE, "sbox_circuits.json")
OUT = os.path.join(HERE, "..", "bs_generated.cuh")


def read_table(src, name):
    m = re.search(r"constexpr int %s\[\d+\] = \{([^}]*)\};" % re.escape(name), src)
    return [int(x) for x in m.group(1).replace("\n", " ").split(",") if x.strip()]


def read_sboxes(src):
    """kS[8][4][16] of des_tables.h: S-box j, row b1 b6, column b2 b3 b4 b5."""
    m = re.search(r"constexpr uint8_t kS\[8\]\[4\]\[16\] = \{(.*?)\};", src, re.S)
    vals = [int(x) for x in re.findall(r"\d+", m.group(1))]
    assert len(vals) == 8 * 4 * 16
    return [[vals[(j * 4 + r) * 16:(j * 4 + r + 1) * 16] for r in range(4)] for j in range(8)]


def check_circuit(c, sbox):
    """Evaluates the circuit on all 64 inputs against the table; raises on a mismatch.
    Node m < 6 is input bit b(m+1) (b1 = the input's bit 5); gate g is node 6 + g;
    an output is node*2 + complement, output t the S-box's bit 3 - t."""
    for x in range(64):
        val = [(x >> (5 - m)) & 1 for m in range(6)]
        for a, b, cc, imm in c["gates"]:
            val.append((imm >> (4 * val[a] + 2 * val[b] + val[cc])) & 1)
        s = sbox[((x >> 5) & 1) * 2 + (x & 1)][(x >> 1) & 15]
        for t, o in enumerate(c["outputs"]):
            if (val[o >> 1] ^ (o & 1)) != ((s >> (3 - t)) & 1):
                raise SystemExit("S%d circuit is wrong for input %d, output %d" % (c["sbox"], x, t))


COLUMN = (0xF0, 0xCC, 0xAA)  # truth table of a gate's input a, b, c alone


def depends(imm, k):
    """whether the 3-input truth table imm depends on its input k (0 = a)"""
    sh = 2 - k
    return any(((imm >> x) & 1) != ((imm >> (x ^ (1 << sh))) & 1) for x in range(8))


def xor_linear(imm, k):
    """whether imm(a, b, c) = input k ^ (a function of the other two)"""
    sh = 2 - k
    return all(((imm >> x) & 1) != ((imm >> (x ^ (1 << sh))) & 1) for x in range(8))


def find_folds(c):
    """Outputs whose XOR into the destination plane the circuit can absorb:
    for output t, a gate with an input slot its truth table ignores, whose
    value reaches the output node through gates that each have it as their
    only reader and are XOR-linear in it (the output node itself read by no
    gate and no other output).  The destination plane then enters that slot
    (the gate's table XORed with the slot's column), every gate on the way
    carries it along, and the output node holds S-box bit ^ plane.  Returns
    {t: (gate index, slot)}; the first such gate in a fixed search order."""
    gates = c["gates"]
    readers = {}
    for gi, (a, b, cc, imm) in enumerate(gates):
        for k, s in enumerate((a, b, cc)):
            if depends(imm, k):
                readers[s] = readers.get(s, 0) + 1
    outs = [o >> 1 for o in c["outputs"]]
    folds = {}
    for t, node in enumerate(outs):
        if node < 6 or readers.get(node, 0) or outs.count(node) > 1:
            continue
        stack = [node]
        while stack:
            n = stack.pop()
            a, b, cc, imm = gates[n - 6]
            free = [k for k in range(3) if not depends(imm, k)]
            if free:
                folds[t] = (n - 6, free[0])
                break
            for k, s in enumerate((a, b, cc)):
                if s >= 6 and s not in outs and readers.get(s, 0) == 1 and xor_linear(imm, k):
                    stack.append(s)
    return folds


def folded_gates(c, folds):
    """The gate list with the folds applied: gate -> (inputs, imm), where an
    input is a node number or ("d", t), the destination plane of output t.
    A complemented folded output gets its node's table complemented (the
    node has no other reader), so that the node holds bit ^ plane exactly."""
    gates = [([a, b, cc], imm) for a, b, cc, imm in c["gates"]]
    for t, (gi, k) in folds.items():
        ins, imm = gates[gi]
        ins = list(ins)
        ins[k] = ("d", t)
        gates[gi] = (ins, imm ^ COLUMN[k])
    for t in folds:
        node, neg = c["outputs"][t] >> 1, c["outputs"][t] & 1
        if neg:
            ins, imm = gates[node - 6]
            gates[node - 6] = (ins, ~imm & 0xFF)
    return gates


def check_folds(c, sbox, folds):
    """On all 64 inputs and every value of the folded outputs' planes: a
    folded output node equals S-box bit ^ plane, and every other output is
    unchanged."""
    gates = folded_gates(c, folds)
    ts = sorted(folds)
    for x in range(64):
        s = sbox[((x >> 5) & 1) * 2 + (x & 1)][(x >> 1) & 15]
        for dv in range(1 << len(ts)):
            d = {t: (dv >> i) & 1 for i, t in enumerate(ts)}
            val = [(x >> (5 - m)) & 1 for m in range(6)]
            for ins, imm in gates:
                v = [d[i[1]] if isinstance(i, tuple) else val[i] for i in ins]
                val.append((imm >> (4 * v[0] + 2 * v[1] + v[2])) & 1)
            for t, o in enumerate(c["outputs"]):
                want = (s >> (3 - t)) & 1
                got = val[o >> 1] ^ d[t] if t in folds else val[o >> 1] ^ (o & 1)
                if got != want:
                    raise SystemExit("S%d fold of output %d is wrong for input %d" % (c["sbox"], t, x))


def slot(n):
    return 8 * ((n - 1) // 8) + 7 - (n - 1) % 8


IMAD = "--imad" in sys.argv
INTERLEAVE = "--sequential" not in sys.argv
FOLD = "--no-fold" not in sys.argv


def main():
    src = open(TABLES).read()
    IP = read_table(src, "kIP")
    FP = read_table(src, "kFP")
    E = read_table(src, "kE")
    P = read_table(src, "kP")
    circuits = json.load(open(CIRCUITS))
    assert len(circuits) == 8
    sboxes = read_sboxes(src)
    for c in circuits:
        check_circuit(c, sboxes[c["sbox"] - 1])
    # The folded rounds may use another circuit per S-box (its "fold" entry):
    # the fewest gates serve the unfolded rounds, the fewest gates plus
    # outputs that cannot fold serve the folded ones.
    fold_circuits = []
    for c in circuits:
        fc = dict(c["fold"], sbox=c["sbox"]) if FOLD and "fold" in c else c
        check_circuit(fc, sboxes[c["sbox"] - 1])
        fold_circuits.append(fc)
    # folded outputs, numbered f = 0.. in S-box order: (j, t) -> f
    folds = [find_folds(c) if FOLD else {} for c in fold_circuits]
    for c, fd in zip(fold_circuits, folds):
        check_folds(c, sboxes[c["sbox"] - 1], fd)
    fold_index = {}
    for j, fd in enumerate(folds):
        for t in sorted(fd):
            fold_index[(j, t)] = len(fold_index)
    nfold = len(fold_index)
    mapL = [None] + [slot(IP[i - 1]) for i in range(1, 33)]
    mapR = [None] + [slot(IP[32 + i - 1]) for i in range(1, 33)]
    Pinv = [None] * 33
    for i in range(1, 33):
        Pinv[P[i - 1]] = i
    # first E position of every R bit, and the 16 duplicated bits' second positions
    first_pos = [None] * 33
    dups = []  # (bit, first position, second position)
    for q, e in enumerate(E):
        if first_pos[e] is None:
            first_pos[e] = q
        else:
            dups.append((e, first_pos[e], q))
    assert len(dups) == 16 and all(x is not None for x in first_pos[1:])
    dup_index = {q2: d for d, (_, _, q2) in enumerate(dups)}

    total_gates = sum(len(c["gates"]) for c in circuits)
    total_gates_f = sum(len(c["gates"]) for c in fold_circuits)
    lines = []
    emit = lines.append
    emit("// Generated by gen/gen_bitslice.py from des_tables.h and gen/sbox_circuits.json.")
    emit("// Do not edit by hand.  Straight-line bitsliced DES round code (see the")
    emit("// generator's docstring for the plane layout and the key absorption).")
    emit("#pragma once")
    emit("")
    emit("#define DES3_BS_SBOX_GATES %d  // LOP3 gates of S1..S8 together (unfolded rounds)" % total_gates)
    emit("#define DES3_BS_SBOX_GATES_F %d  // the same in the folded rounds" % total_gates_f)
    for c in circuits:
        emit("#define DES3_BS_S%d_GATES %d" % (c["sbox"], len(c["gates"])))
    emit("// S-box outputs whose XOR into the destination plane their circuit absorbs")
    emit("// (the plane enters a free gate input; the update's mask change then runs as")
    emit("// a multiply-add); the other outputs keep the 3-input XOR")
    emit("#define DES3_BS_FOLDS %d" % nfold)
    emit("// integer instructions per round for 32 blocks: 16 key corrections + gates + 32 state")
    emit("// updates (of which DES3_BS_FOLDS are multiply-adds)")
    emit("#define DES3_BS_OPS_PER_ROUND (16 + DES3_BS_SBOX_GATES + 32)")
    emit("#define DES3_BS_OPS_PER_ROUND_F (16 + DES3_BS_SBOX_GATES_F + 32)")
    emit("// Key masks as the host builds them (one bit each, bs_mask_bits): 48 rounds x")
    emit("// (16 corrections, 32 deltas, 16 copies of the corrections), then remasks of the")
    emit("// source half before rounds 0, 16 and 32 (32 each), then the final unmask of")
    emit("// L-planes and R-planes (32 each)")
    emit("#define DES3_BS_KEY_ROUND_WORDS 64")
    emit("#define DES3_BS_KEY_WORDS (48 * DES3_BS_KEY_ROUND_WORDS + 5 * 32)")
    emit("#define DES3_BS_KEY_PRE0 (48 * DES3_BS_KEY_ROUND_WORDS)")
    emit("#define DES3_BS_KEY_PRE16 (48 * DES3_BS_KEY_ROUND_WORDS + 32)")
    emit("#define DES3_BS_KEY_PRE32 (48 * DES3_BS_KEY_ROUND_WORDS + 64)")
    emit("#define DES3_BS_KEY_POST_L (48 * DES3_BS_KEY_ROUND_WORDS + 96)")
    emit("#define DES3_BS_KEY_POST_R (48 * DES3_BS_KEY_ROUND_WORDS + 128)")
    emit("// Mask words as the rounds read them (bs_mask_from_bits expands the bits).  Two")
    emit("// layouts: the unfolded rounds (bs_round_A/B) read per round [0,16) corrections c,")
    emit("// [16,48) deltas, [48,64) multipliers s = c | 1 of the corrections; the folded")
    emit("// rounds (bs_round_A_f/B_f) read those and [64, 64 + DES3_BS_FOLDS) multipliers of")
    emit("// the folded outputs' deltas; then the remasks and unmasks as above")
    emit("#define DES3_BS_ROUND_WORDS 64")
    emit("#define DES3_BS_MASK_WORDS (48 * DES3_BS_ROUND_WORDS + 5 * 32)")
    emit("#define DES3_BS_PRE0 (48 * DES3_BS_ROUND_WORDS)")
    emit("#define DES3_BS_PRE16 (48 * DES3_BS_ROUND_WORDS + 32)")
    emit("#define DES3_BS_PRE32 (48 * DES3_BS_ROUND_WORDS + 64)")
    emit("#define DES3_BS_POST_L (48 * DES3_BS_ROUND_WORDS + 96)")
    emit("#define DES3_BS_POST_R (48 * DES3_BS_ROUND_WORDS + 128)")
    emit("#define DES3_BS_ROUND_WORDS_F (64 + DES3_BS_FOLDS)")
    emit("#define DES3_BS_MASK_WORDS_F (48 * DES3_BS_ROUND_WORDS_F + 5 * 32)")
    emit("// 1: the 16 corrections run as x * s + c on the FMA pipe (mad.lo); 0: x ^ c on the ALU")
    emit("#define DES3_BS_IMAD_CORR %d" % (1 if IMAD else 0))
    emit("")
    emit("// E position (0..47) of the first use of R bit i (1..32); index 0 unused.")
    emit("static constexpr int kBsFirstPos[33] = {-1, %s};" % ", ".join(str(first_pos[i]) for i in range(1, 33)))
    emit("// The 16 bits E uses twice: {bit, first position, second position}.")
    emit("static constexpr int kBsDup[16][3] = {%s};" % ", ".join("{%d, %d, %d}" % d for d in dups))
    emit("// Round mask word (16..47) of the delta whose multiplier is round mask word 64 + f.")
    emit("__host__ __device__ __forceinline__ int bs_fold_delta(int f) {")
    emit("  switch (f) {")
    for (j, t), f in sorted(fold_index.items(), key=lambda kv: kv[1]):
        emit("    case %d: return %d;  // S%d output %d" % (f, 16 + Pinv[4 * j + t + 1] - 1, circuits[j]["sbox"], t))
    emit("    default: return 16;")
    emit("  }")
    emit("}")
    emit("")

    def round_fn(name, dst_map, src_map, fold):
        emit("// %s: %s ^= f(%s, K).  m[0..15]: corrections of the duplicated E inputs," % (
            name, "L" if dst_map is mapL else "R", "R" if src_map is mapR else "L"))
        emit("// m[16 + i - 1]: mask change of destination plane i (see the generator)%s." % (
            "; m[64 + f]: multiplier of fold f's mask change" if fold else ""))
        emit("__host__ __device__ __forceinline__ void %s(uint32_t (&w)[64], const uint32_t* __restrict__ m) {" % name)
        fx = folds if fold else [{} for _ in circuits]
        fi = fold_index if fold else {}
        cs = fold_circuits if fold else circuits
        if INTERLEAVE:
            round_body_interleaved(dst_map, src_map, fx, fi, cs)
            emit("}")
            emit("")
            return
        for j, c in enumerate(cs):
            emit("  {  // S%d" % c["sbox"])
            for mm in range(6):
                q = 6 * j + mm
                if q in dup_index:
                    emit("    const uint32_t n%d = bs_correct(w[%d], m[%d], m[%d]);" % (
                        mm, src_map[E[q]], dup_index[q], 48 + dup_index[q]))
                else:
                    emit("    const uint32_t n%d = w[%d];" % (mm, src_map[E[q]]))
            def ref(x):
                return "w[%d]" % dst_map[Pinv[4 * j + x[1] + 1]] if isinstance(x, tuple) else "n%d" % x
            for gi, (ins, imm) in enumerate(folded_gates(c, fx[j])):
                emit("    const uint32_t n%d = lop3<0x%02x>(%s, %s, %s);" % ((gi + 6, imm) + tuple(ref(x) for x in ins)))
            for t, r in enumerate(c["outputs"]):
                node, neg = r >> 1, r & 1
                i = Pinv[4 * j + t + 1]
                dst = dst_map[i]
                if (j, t) in fi:  # node = out ^ old: only the mask change, on the FMA pipe
                    emit("    w[%d] = bs_correct(n%d, m[%d], m[%d]);" % (dst, node, 16 + i - 1, 64 + fi[(j, t)]))
                    continue
                imm = 0x96 if not neg else 0x69  # a ^ b ^ c  /  a ^ ~b ^ c
                emit("    w[%d] = lop3<0x%02x>(w[%d], n%d, m[%d]);" % (dst, imm, dst, node, 16 + i - 1))
            emit("  }")
        emit("}")
        emit("")

    def round_body_interleaved(dst_map, src_map, fx, fi, circuits):
        # all eight S-boxes at once, gate by gate in order of depth, so that
        # independent instructions sit next to each other in the source
        depth = {}
        for j, c in enumerate(circuits):
            for mm in range(6):
                q = 6 * j + mm
                if q in dup_index:
                    emit("  const uint32_t s%d_%d = bs_correct(w[%d], m[%d], m[%d]);" % (
                        j, mm, src_map[E[q]], dup_index[q], 48 + dup_index[q]))
                else:
                    emit("  const uint32_t s%d_%d = w[%d];" % (j, mm, src_map[E[q]]))
                depth[(j, mm)] = 0
            for gi, (ins, imm) in enumerate(folded_gates(c, fx[j])):
                depth[(j, gi + 6)] = 1 + max(0 if isinstance(x, tuple) else depth[(j, x)] for x in ins)
        maxd = max(depth.values())
        for d in range(1, maxd + 1):
            for j, c in enumerate(circuits):
                def ref(x):
                    return "w[%d]" % dst_map[Pinv[4 * j + x[1] + 1]] if isinstance(x, tuple) else "s%d_%d" % (j, x)
                for gi, (ins, imm) in enumerate(folded_gates(c, fx[j])):
                    if depth[(j, gi + 6)] == d:
                        emit("  const uint32_t s%d_%d = lop3<0x%02x>(%s, %s, %s);" % (
                            (j, gi + 6, imm) + tuple(ref(x) for x in ins)))
        for j, c in enumerate(circuits):
            for t, r in enumerate(c["outputs"]):
                node, neg = r >> 1, r & 1
                i = Pinv[4 * j + t + 1]
                dst = dst_map[i]
                if (j, t) in fi:  # node = out ^ old: only the mask change, on the FMA pipe
                    emit("  w[%d] = bs_correct(s%d_%d, m[%d], m[%d]);" % (
                        dst, j, node, 16 + i - 1, 64 + fi[(j, t)]))
                    continue
                imm = 0x96 if not neg else 0x69
                emit("  w[%d] = lop3<0x%02x>(w[%d], s%d_%d, m[%d]);" % (dst, imm, dst, j, node, 16 + i - 1))

    round_fn("bs_round_A", mapL, mapR, False)
    round_fn("bs_round_B", mapR, mapL, False)
    round_fn("bs_round_A_f", mapL, mapR, True)
    round_fn("bs_round_B_f", mapR, mapL, True)

    for name, mp in (("bs_remask_L", mapL), ("bs_remask_R", mapR)):
        emit("// %s: XOR every %s-plane i with m[i - 1]." % (name, name[-1]))
        emit("__host__ __device__ __forceinline__ void %s(uint32_t (&w)[64], const uint32_t* __restrict__ m) {" % name)
        for i in range(1, 33):
            emit("  w[%d] ^= m[%d];" % (mp[i], i - 1))
        emit("}")
        emit("")

    emit("// bs_swap_halves: exchange the L-planes and the R-planes (so that one loop")
    emit("// body of (round_A, round_B) can run all three DES of the pipeline).")
    emit("__host__ __device__ __forceinline__ void bs_swap_halves(uint32_t (&w)[64]) {")
    for i in range(1, 33):
        emit("  { const uint32_t t = w[%d]; w[%d] = w[%d]; w[%d] = t; }" % (mapL[i], mapL[i], mapR[i], mapR[i]))
    emit("}")
    emit("")
    # final: output DES bit n sits in plane src(n); move it to slot(n)
    emit("// After 48 rounds the pre-output is R16||L16 (R = the planes that started as")
    emit("// R0).  Output bit n of FP is pre-output bit FP[n]; o[slot(n)] receives it.")
    emit("__host__ __device__ __forceinline__ void bs_final_perm(const uint32_t (&w)[64], uint32_t (&o)[64]) {")
    for n in range(1, 65):
        q = FP[n - 1]
        src_slot = mapR[q] if q <= 32 else mapL[q - 32]
        emit("  o[%d] = w[%d];" % (slot(n), src_slot))
    emit("}")
    emit("")
    # the LOP3 gate list as data, for the host self test
    emit("// The circuits as data (inputs are nodes 0..5 = b1..b6; node 6+i is gate i;")
    emit("// an output reference is 2*node + complement).  Used by the self test.")
    emit("struct BsCircuit { int ngates; unsigned char g[64][4]; int out[4]; };")
    emit("static const BsCircuit kBsCircuits[8] = {")
    for c in circuits:
        gl = ", ".join("{%d, %d, %d, 0x%02x}" % tuple(g) for g in c["gates"])
        emit("  {%d, {%s}, {%s}}," % (len(c["gates"]), gl, ", ".join(str(x) for x in c["outputs"])))
    emit("};")
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")
    if IMAD:
        print("wrote %s: unfolded rounds %d gates, %d ALU + 16 FMA ops; folded rounds %d gates, %d folded "
              "outputs, %d ALU + %d FMA ops (per round)" % (OUT, total_gates, 32 + total_gates, total_gates_f, nfold,
                                                          32 + total_gates_f - nfold, 16 + nfold))
    else:
        print("wrote %s: unfolded rounds %d gates; folded rounds %d gates, %d folded outputs" % (
            OUT, total_gates, total_gates_f, nfold))


if __name__ == "__main__":
    main()
