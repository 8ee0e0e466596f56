"""Generate bs_generated.cuh, the straight-line round code of the bitsliced kernel.

Inputs:
  * ../des_tables.h      -- the library's copy of the DES tables (IP, FP, E, P)
  * sbox_circuits.json   -- LOP3 circuits for S1..S8, found by this project's
                            circuit search (a working tool kept outside the
                            library); each is checked here against the
                            S-box table on all 64 inputs before any code is
                            written (and again by des3_self_test())

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

The round code lists the eight circuits' gates interleaved by depth (all
depth-1 gates of S1..S8, then all depth-2 gates, ...), which measured 0.4 %
faster on a single buffer and 1.2 % faster in the batched kernel than one
S-box after another (--sequential).

Run:  python gen_bitslice.py [--imad] [--sequential]   (writes ../bs_generated.cuh)
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


def slot(n):
    return 8 * ((n - 1) // 8) + 7 - (n - 1) % 8


IMAD = "--imad" in sys.argv
INTERLEAVE = "--sequential" not in sys.argv


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
    lines = []
    emit = lines.append
    emit("// Generated by gen/gen_bitslice.py from des_tables.h and gen/sbox_circuits.json.")
    emit("// Do not edit by hand.  Straight-line bitsliced DES round code (see the")
    emit("// generator's docstring for the plane layout and the key absorption).")
    emit("#pragma once")
    emit("")
    emit("#define DES3_BS_SBOX_GATES %d  // LOP3 gates of S1..S8 together" % total_gates)
    for c in circuits:
        emit("#define DES3_BS_S%d_GATES %d" % (c["sbox"], len(c["gates"])))
    emit("// integer instructions per round for 32 blocks: 16 key corrections + gates + 32 state XORs")
    emit("#define DES3_BS_OPS_PER_ROUND (16 + DES3_BS_SBOX_GATES + 32)")
    emit("// mask words: 48 rounds x (16 corrections, 32 deltas), then remasks of the")
    emit("// source half before rounds 0, 16 and 32 (32 words each), then the final unmask of")
    emit("// L-planes and R-planes (32 words each)")
    emit("// per round: [0,16) corrections c, [16,48) deltas, [48,64) multipliers s = c | 1")
    emit("#define DES3_BS_ROUND_WORDS 64")
    emit("#define DES3_BS_MASK_WORDS (48 * DES3_BS_ROUND_WORDS + 5 * 32)")
    emit("#define DES3_BS_PRE0 (48 * DES3_BS_ROUND_WORDS)")
    emit("#define DES3_BS_PRE16 (48 * DES3_BS_ROUND_WORDS + 32)")
    emit("#define DES3_BS_PRE32 (48 * DES3_BS_ROUND_WORDS + 64)")
    emit("#define DES3_BS_POST_L (48 * DES3_BS_ROUND_WORDS + 96)")
    emit("#define DES3_BS_POST_R (48 * DES3_BS_ROUND_WORDS + 128)")
    emit("// 1: the 16 corrections run as x * s + c on the FMA pipe (mad.lo); 0: x ^ c on the ALU")
    emit("#define DES3_BS_IMAD_CORR %d" % (1 if IMAD else 0))
    emit("")
    emit("// E position (0..47) of the first use of R bit i (1..32); index 0 unused.")
    emit("static constexpr int kBsFirstPos[33] = {-1, %s};" % ", ".join(str(first_pos[i]) for i in range(1, 33)))
    emit("// The 16 bits E uses twice: {bit, first position, second position}.")
    emit("static constexpr int kBsDup[16][3] = {%s};" % ", ".join("{%d, %d, %d}" % d for d in dups))
    emit("")

    def round_fn(name, dst_map, src_map):
        emit("// %s: %s ^= f(%s, K).  m[0..15]: corrections of the duplicated E inputs," % (
            name, "L" if dst_map is mapL else "R", "R" if src_map is mapR else "L"))
        emit("// m[16 + i - 1]: mask change of destination plane i (see the generator).")
        emit("__host__ __device__ __forceinline__ void %s(uint32_t (&w)[64], const uint32_t* __restrict__ m) {" % name)
        if INTERLEAVE:
            round_body_interleaved(dst_map, src_map)
            emit("}")
            emit("")
            return
        for j, c in enumerate(circuits):
            emit("  {  // S%d" % c["sbox"])
            for mm in range(6):
                q = 6 * j + mm
                if q in dup_index:
                    emit("    const uint32_t n%d = bs_correct(w[%d], m[%d], m[%d]);" % (
                        mm, src_map[E[q]], dup_index[q], 48 + dup_index[q]))
                else:
                    emit("    const uint32_t n%d = w[%d];" % (mm, src_map[E[q]]))
            gates = c["gates"]
            for gi, g in enumerate(gates):
                a, b, cc, imm = g
                emit("    const uint32_t n%d = lop3<0x%02x>(n%d, n%d, n%d);" % (gi + 6, imm, a, b, cc))
            for t, r in enumerate(c["outputs"]):
                node, neg = r >> 1, r & 1
                i = Pinv[4 * j + t + 1]
                dst = dst_map[i]
                imm = 0x96 if not neg else 0x69  # a ^ b ^ c  /  a ^ ~b ^ c
                emit("    w[%d] = lop3<0x%02x>(w[%d], n%d, m[%d]);" % (dst, imm, dst, node, 16 + i - 1))
            emit("  }")
        emit("}")
        emit("")

    def round_body_interleaved(dst_map, src_map):
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
            for gi, g in enumerate(c["gates"]):
                depth[(j, gi + 6)] = 1 + max(depth[(j, x)] for x in g[:3])
        maxd = max(depth.values())
        for d in range(1, maxd + 1):
            for j, c in enumerate(circuits):
                for gi, g in enumerate(c["gates"]):
                    if depth[(j, gi + 6)] == d:
                        a, b, cc, imm = g
                        emit("  const uint32_t s%d_%d = lop3<0x%02x>(s%d_%d, s%d_%d, s%d_%d);" % (
                            j, gi + 6, imm, j, a, j, b, j, cc))
        for j, c in enumerate(circuits):
            for t, r in enumerate(c["outputs"]):
                node, neg = r >> 1, r & 1
                i = Pinv[4 * j + t + 1]
                dst = dst_map[i]
                imm = 0x96 if not neg else 0x69
                emit("  w[%d] = lop3<0x%02x>(w[%d], s%d_%d, m[%d]);" % (dst, imm, dst, j, node, 16 + i - 1))

    round_fn("bs_round_A", mapL, mapR)
    round_fn("bs_round_B", mapR, mapL)

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
    print("wrote %s: %d gates, %d ALU + 16 %s ops per round" % (OUT, total_gates, 32 + total_gates,
                                                              "FMA" if IMAD else "ALU"))


if __name__ == "__main__":
    main()
