// sptable.cuh -- the table kernel's round function: combined S+P tables and
// the rotated form the kernel runs, for the device and for the host self test.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace des3 {

// ---- table kernel: combined S-box + P tables ---------------------------
//
// f(R, K) = P(S(E(R) xor K)) = XOR over j of SP_j[E_j(R) xor K_j], where
// SP_j[x] is P applied to S_j(x) placed at S-box j's output nibble.  E_j(R),
// S-box j's 6-bit window of R, is a rotation: rotr(R, (27 - 4j) mod 32) & 63.
// The kernel keeps the window at bits 7..12 (a byte offset into a table
// whose 64 entries are 128 bytes apart, one 4-byte slot per lane), so it
// rotates by 7 less.
struct SpTable {
    uint32_t v[8][64];
};

constexpr SpTable make_sp_table() {
    SpTable t{};
    for (int j = 0; j < 8; j++)
        for (uint32_t x = 0; x < 64; x++) {
            uint32_t sout = fips::sbox(j, x) << (28 - 4 * j);  // S output bit q at bit 32-q
            uint32_t f = 0;
            for (int i = 1; i <= 32; i++)
                if ((sout >> (32 - fips::kP[i - 1])) & 1u) f |= 1u << (32 - i);
            t.v[j][x] = f;
        }
    return t;
}

// rotr amount that brings S-box j's window to bits 7..12: (20 - 4j) mod 32.
DES3_HD constexpr int sp_rot(int j) { return (20 - 4 * j) & 31; }

// Key words of the table kernel: for round r and S-box j, the 6 key bits
// K_r[6j+1..6j+6] shifted to bits 7..12.
DES3_HD uint32_t sp_key_word(uint64_t rk, int j) {
    return (uint32_t)((rk >> (42 - 6 * j)) & 63u) << 7;
}

// f(R, K) with a table lookup functor lk(j, byte_offset).
template <class Lookup>
DES3_HD uint32_t sp_f(uint32_t r, const uint32_t* k8, const Lookup& lk) {
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < 8; j++) s ^= lk(j, (rotr32(r, sp_rot(j)) & 0x1F80u) ^ k8[j]);
    return s;
}

// ---- table kernel, rotated form (what sptable_kernel runs) ---------------
//
// Both halves are kept rotated right by one bit, R' = rotr(R, 1).  In that
// form every S-box window of E(R) is a fixed field of R', its first input bit
// b1 on top:
//   S1 bits 26..31, S3 18..23, S5 10..15, S7 2..7         (disjoint)
//   S2 bits 22..27, S4 14..19, S6 6..11, S8 3..0 then 31,30 (disjoint; wraps)
// The six key bits of each S-box sit in the same field of one of two words
// per round, ke (S1, S3, S5, S7) and ko (S2, S4, S6, S8), so a single LOP3
// gives (R' ^ k) & field.  A shift then moves the field to bits 10..15 of the
// shared-memory address (S8's wrapped field: a rotation by 12, which brings
// bits 30, 31 to 10, 11 and bits 0..3 to 12..15) and the lane's base is
// added.  The tables hold rotr(P(S_j(x)), 1), so the XOR of the eight
// lookups updates the other rotated half directly.  (Doing the shifts as
// multiply-adds on the FMA pipe, a right shift as the high half of a product,
// ran 19 % slower: the high-half multiply-add is a two-pass instruction and
// stalled dispatch.)
//
// Shared-memory layout: entry x of S-box j (0-based) for lane l at byte
// x * 1024 + j * 128 + 4 l (64 KiB); the 32 lanes of a warp always read 32
// distinct banks.
constexpr SpTable make_sp_rot_table() {
    SpTable t = make_sp_table();
    for (int j = 0; j < 8; j++)
        for (int x = 0; x < 64; x++) t.v[j][x] = (t.v[j][x] >> 1) | (t.v[j][x] << 31);
    return t;
}

// (ke, ko) of one round key (round-key bit 1 at bit 47, S-box j's six bits
// at 42 - 6j .. 47 - 6j).
inline void sp_rot_key(uint64_t rk, uint32_t* ke, uint32_t* ko) {
    uint32_t c[8];
    for (int j = 0; j < 8; j++) c[j] = (uint32_t)(rk >> (42 - 6 * j)) & 63u;
    *ke = (c[0] << 26) | (c[2] << 18) | (c[4] << 10) | (c[6] << 2);
    *ko = (c[1] << 22) | (c[3] << 14) | (c[5] << 6) | (c[7] >> 2) | ((c[7] & 3u) << 30);
}

// One round in the rotated form: returns l' ^ f'(r'), where f' = rotr(f, 1).
// tb: the lane's table base address; lk.template at<J>(addr) reads the
// table word at addr + 128 J.
template <class Lookup>
DES3_HD uint32_t sp_round_rot(uint32_t l, uint32_t r, uint32_t ke, uint32_t ko, uint32_t tb, const Lookup& lk) {
    constexpr uint32_t kAndXor = 0x48;  // (a ^ c) & b
    const uint32_t v0 = lk.template at<0>((lop3<kAndXor>(r, 0xFC000000u, ke) >> 16) + tb);
    const uint32_t v1 = lk.template at<1>((lop3<kAndXor>(r, 0x0FC00000u, ko) >> 12) + tb);
    const uint32_t v2 = lk.template at<2>((lop3<kAndXor>(r, 0x00FC0000u, ke) >> 8) + tb);
    const uint32_t v3 = lk.template at<3>((lop3<kAndXor>(r, 0x000FC000u, ko) >> 4) + tb);
    const uint32_t v4 = lk.template at<4>(lop3<kAndXor>(r, 0x0000FC00u, ke) + tb);
    const uint32_t v5 = lk.template at<5>((lop3<kAndXor>(r, 0x00000FC0u, ko) << 4) + tb);
    const uint32_t v6 = lk.template at<6>((lop3<kAndXor>(r, 0x000000FCu, ke) << 8) + tb);
    const uint32_t v7 = lk.template at<7>(rotl32(lop3<kAndXor>(r, 0xC000000Fu, ko), 12) + tb);
    return lop3<0x96>(lop3<0x96>(v0, v1, v2), lop3<0x96>(v3, v4, v5), lop3<0x96>(v6, v7, l));
}

// 3DES (NS = 3) or single DES (NS = 1) on NB blocks held as big-endian (hi,
// lo) word pairs, in place.  k4[i] = (ke, ko) of rounds 2i and 2i + 1 in
// application order.
template <int NB, int NS, class Lookup>
DES3_HD void sp_tdes_rot(uint32_t (&hi)[NB], uint32_t (&lo)[NB], const uint4* k4, uint32_t tb, const Lookup& lk) {
    uint32_t a[NB], b[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) {
        initial_perm(hi[i], lo[i]);
        a[i] = rotr32(hi[i], 1);  // L0'
        b[i] = rotr32(lo[i], 1);  // R0'
    }
    // Within a DES the halves alternate as the updated one; between DES
    // operations FP and the next IP cancel, so the second DES starts by
    // updating the half the first one updated last.
#pragma unroll 1
    for (int d = 0; d < NS; d++) {
#pragma unroll 1
        for (int r = 0; r < 8; r++, k4++) {
            const uint4 k = *k4;
            if (d == 1) {
#pragma unroll
                for (int i = 0; i < NB; i++) b[i] = sp_round_rot(b[i], a[i], k.x, k.y, tb, lk);
#pragma unroll
                for (int i = 0; i < NB; i++) a[i] = sp_round_rot(a[i], b[i], k.z, k.w, tb, lk);
            } else {
#pragma unroll
                for (int i = 0; i < NB; i++) a[i] = sp_round_rot(a[i], b[i], k.x, k.y, tb, lk);
#pragma unroll
                for (int i = 0; i < NB; i++) b[i] = sp_round_rot(b[i], a[i], k.z, k.w, tb, lk);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
        // after an odd number of DES the last update went to b (R16 of the
        // last DES), after NS = 3 likewise: the pre-output is R16 || L16
        hi[i] = rotl32(b[i], 1);
        lo[i] = rotl32(a[i], 1);
        final_perm(hi[i], lo[i]);
    }
}

}  // namespace des3
