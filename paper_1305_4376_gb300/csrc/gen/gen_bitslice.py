"""Generate bs_generated.cuh, the straight-line round code of the bitsliced kernel.

Inputs:
  * ../des_tables.h      -- the library's copy of the DES tables (IP, FP, E, P)
  * sbox_circuits.json   -- LOP3 circuits for S1..S8 written by sboxgen.c

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
instructions are the 48 key XORs, the S-box circuits and the XOR of each S-box
output into its destination plane, which is folded into the circuit's last
gate when that gate has at most two distinct inputs.

Run:  python gen_bitslice.py   (writes ../bs_generated.cuh)
"""
import json
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
TABLES = os.path.join(HERE, "..", "des_tables.h")
CIRCUITS = os.path.join(HERE, "sbox_circuits.json")
OUT = os.path.join(HERE, "..", "bs_generated.cuh")


def read_table(src, name):
    m = re.search(r"constexpr int %s\[\d+\] = \{([^}]*)\};" % re.escape(name), src)
    return [int(x) for x in m.group(1).replace("\n", " ").split(",") if x.strip()]


def slot(n):
    return 8 * ((n - 1) // 8) + 7 - (n - 1) % 8


def flip_input(imm, pos):
    """Truth table of LUT(a,b,c) with input `pos` (0=a,1=b,2=c) complemented."""
    bit = {0: 4, 1: 2, 2: 1}[pos]
    return sum(((imm >> (k ^ bit)) & 1) << k for k in range(8))


def lut_eval(imm, a, b, c):
    return (imm >> (4 * a + 2 * b + c)) & 1


def main():
    src = open(TABLES).read()
    IP = read_table(src, "kIP")
    FP = read_table(src, "kFP")
    E = read_table(src, "kE")
    P = read_table(src, "kP")
    circuits = json.load(open(CIRCUITS))
    assert len(circuits) == 8
    mapL = [None] + [slot(IP[i - 1]) for i in range(1, 33)]
    mapR = [None] + [slot(IP[32 + i - 1]) for i in range(1, 33)]
    Pinv = [None] * 33
    for i in range(1, 33):
        Pinv[P[i - 1]] = i

    total_gates = sum(len(c["gates"]) for c in circuits)
    lines = []
    emit = lines.append
    emit("// Generated by gen/gen_bitslice.py from des_tables.h and gen/sbox_circuits.json.")
    emit("// Do not edit by hand.  Straight-line bitsliced DES round code (see the")
    emit("// generator's docstring for the plane layout).")
    emit("#pragma once")
    emit("")
    emit("#define DES3_BS_SBOX_GATES %d  // LOP3 gates of S1..S8 together" % total_gates)
    for c in circuits:
        emit("#define DES3_BS_S%d_GATES %d" % (c["sbox"], len(c["gates"])))
    emit("")

    def round_fn(name, dst_map, src_map):
        emit("// %s: %s ^= f(%s, K) with the 48 key masks k[0..47] of this round." % (
            name, "L" if dst_map is mapL else "R", "R" if src_map is mapR else "L"))
        emit("__host__ __device__ __forceinline__ void %s(uint32_t (&w)[64], const uint32_t* __restrict__ k) {" % name)
        nfold = 0
        nxor = 0
        for j, c in enumerate(circuits):
            emit("  {  // S%d" % c["sbox"])
            for m in range(6):
                emit("    const uint32_t n%d = w[%d] ^ k[%d];" % (m, src_map[E[6 * j + m]], 6 * j + m))
            gates = c["gates"]
            outs = c["outputs"]
            # which nodes are outputs and how many gate uses each node has
            uses = {}
            for g in gates:
                for x in set(g[:3]):
                    uses[x] = uses.get(x, 0) + 1
            out_nodes = {}
            for t, r in enumerate(outs):
                out_nodes.setdefault(r >> 1, []).append(t)
            foldable = {}
            for t, r in enumerate(outs):
                node = r >> 1
                if node < 6:
                    continue
                g = gates[node - 6]
                distinct = sorted(set(g[:3]))
                if len(distinct) <= 2 and uses.get(node, 0) == 0 and len(out_nodes[node]) == 1:
                    foldable[node] = t
            for gi, g in enumerate(gates):
                node = gi + 6
                a, b, cc, imm = g
                if node in foldable:
                    continue
                emit("    const uint32_t n%d = lop3<0x%02x>(n%d, n%d, n%d);" % (node, imm, a, b, cc))
            for t, r in enumerate(outs):
                node, neg = r >> 1, r & 1
                dst = dst_map[Pinv[4 * j + t + 1]]
                if node in foldable:
                    a, b, cc, imm = gates[node - 6]
                    distinct = sorted(set([a, b, cc]))
                    while len(distinct) < 2:
                        distinct.append(distinct[0])
                    u, v = distinct
                    # new = w ^ G(u, v) ^ neg, as a LUT of (w, u, v)
                    tt = 0
                    for k in range(8):
                        wv, uv, vv = (k >> 2) & 1, (k >> 1) & 1, k & 1
                        val = {u: uv, v: vv}
                        gv = lut_eval(imm, val[a], val[b], val[cc])
                        tt |= (wv ^ gv ^ neg) << k
                    emit("    w[%d] = lop3<0x%02x>(w[%d], n%d, n%d);" % (dst, tt, dst, u, v))
                    nfold += 1
                else:
                    imm = 0x96 if False else (0x3C if not neg else 0xC3)  # a ^ b  /  a ^ ~b
                    emit("    w[%d] = lop3<0x%02x>(w[%d], n%d, n%d);" % (dst, imm, dst, node, node))
                    nxor += 1
            emit("  }")
        emit("}")
        emit("")
        return nfold, nxor

    nfold, nxor = round_fn("bs_round_A", mapL, mapR)
    round_fn("bs_round_B", mapR, mapL)
    emit("#define DES3_BS_FOLDED_OUTPUTS %d  // S-box outputs whose XOR into the state is free" % nfold)
    emit("#define DES3_BS_XOR_OUTPUTS %d     // S-box outputs needing one extra XOR" % nxor)
    emit("// ALU instructions per round for 32 blocks: key XORs + gates + extra output XORs")
    emit("#define DES3_BS_OPS_PER_ROUND (48 + DES3_BS_SBOX_GATES - DES3_BS_FOLDED_OUTPUTS + DES3_BS_XOR_OUTPUTS)")
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
    print("wrote %s: %d gates, %d folded outputs, %d extra XORs per round" % (OUT, total_gates, nfold, nxor))


if __name__ == "__main__":
    main()
