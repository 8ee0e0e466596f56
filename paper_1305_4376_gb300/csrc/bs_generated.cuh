// Generated by gen/gen_bitslice.py from des_tables.h and gen/sbox_circuits.json.
// Do not edit by hand.  Straight-line bitsliced DES round code (see the
// generator's docstring for the plane layout and the key absorption).
#pragma once

#define DES3_BS_SBOX_GATES 194  // LOP3 gates of S1..S8 together (unfolded rounds)
#define DES3_BS_SBOX_GATES_F 195  // the same in the folded rounds
#define DES3_BS_S1_GATES 26
#define DES3_BS_S2_GATES 24
#define DES3_BS_S3_GATES 25
#define DES3_BS_S4_GATES 19
#define DES3_BS_S5_GATES 26
#define DES3_BS_S6_GATES 26
#define DES3_BS_S7_GATES 25
#define DES3_BS_S8_GATES 23
// S-box outputs whose XOR into the destination plane their circuit absorbs
// (the plane enters a free gate input; the update's mask change then runs as
// a multiply-add); the other outputs keep the 3-input XOR
#define DES3_BS_FOLDS 3
// integer instructions per round for 32 blocks: 16 key corrections + gates + 32 state
// updates (of which DES3_BS_FOLDS are multiply-adds)
#define DES3_BS_OPS_PER_ROUND (16 + DES3_BS_SBOX_GATES + 32)
#define DES3_BS_OPS_PER_ROUND_F (16 + DES3_BS_SBOX_GATES_F + 32)
// Key masks as the host builds them (one bit each, bs_mask_bits): 48 rounds x
// (16 corrections, 32 deltas, 16 copies of the corrections), then remasks of the
// source half before rounds 0, 16 and 32 (32 each), then the final unmask of
// L-planes and R-planes (32 each)
#define DES3_BS_KEY_ROUND_WORDS 64
#define DES3_BS_KEY_WORDS (48 * DES3_BS_KEY_ROUND_WORDS + 5 * 32)
#define DES3_BS_KEY_PRE0 (48 * DES3_BS_KEY_ROUND_WORDS)
#define DES3_BS_KEY_PRE16 (48 * DES3_BS_KEY_ROUND_WORDS + 32)
#define DES3_BS_KEY_PRE32 (48 * DES3_BS_KEY_ROUND_WORDS + 64)
#define DES3_BS_KEY_POST_L (48 * DES3_BS_KEY_ROUND_WORDS + 96)
#define DES3_BS_KEY_POST_R (48 * DES3_BS_KEY_ROUND_WORDS + 128)
// Mask words as the rounds read them (bs_mask_from_bits expands the bits).  Two
// layouts: the unfolded rounds (bs_round_A/B) read per round [0,16) corrections c,
// [16,48) deltas, [48,64) multipliers s = c | 1 of the corrections; the folded
// rounds (bs_round_A_f/B_f) read those and [64, 64 + DES3_BS_FOLDS) multipliers of
// the folded outputs' deltas; then the remasks and unmasks as above
#define DES3_BS_ROUND_WORDS 64
#define DES3_BS_MASK_WORDS (48 * DES3_BS_ROUND_WORDS + 5 * 32)
#define DES3_BS_PRE0 (48 * DES3_BS_ROUND_WORDS)
#define DES3_BS_PRE16 (48 * DES3_BS_ROUND_WORDS + 32)
#define DES3_BS_PRE32 (48 * DES3_BS_ROUND_WORDS + 64)
#define DES3_BS_POST_L (48 * DES3_BS_ROUND_WORDS + 96)
#define DES3_BS_POST_R (48 * DES3_BS_ROUND_WORDS + 128)
#define DES3_BS_ROUND_WORDS_F (64 + DES3_BS_FOLDS)
#define DES3_BS_MASK_WORDS_F (48 * DES3_BS_ROUND_WORDS_F + 5 * 32)
// 1: the 16 corrections run as x * s + c on the FMA pipe (mad.lo); 0: x ^ c on the ALU
#define DES3_BS_IMAD_CORR 1

// E position (0..47) of the first use of R bit i (1..32); index 0 unused.
static constexpr int kBsFirstPos[33] = {-1, 1, 2, 3, 4, 5, 8, 9, 10, 11, 14, 15, 16, 17, 20, 21, 22, 23, 26, 27, 28, 29, 32, 33, 34, 35, 38, 39, 40, 41, 44, 45, 0};
// The 16 bits E uses twice: {bit, first position, second position}.
static constexpr int kBsDup[16][3] = {{4, 4, 6}, {5, 5, 7}, {8, 10, 12}, {9, 11, 13}, {12, 16, 18}, {13, 17, 19}, {16, 22, 24}, {17, 23, 25}, {20, 28, 30}, {21, 29, 31}, {24, 34, 36}, {25, 35, 37}, {28, 40, 42}, {29, 41, 43}, {32, 0, 46}, {1, 1, 47}};
// Round mask word (16..47) of the delta whose multiplier is round mask word 64 + f.
__host__ __device__ __forceinline__ int bs_fold_delta(int f) {
  switch (f) {
    case 0: return 25;  // S4 output 2
    case 1: return 16;  // S4 output 3
    case 2: return 34;  // S6 output 3
    default: return 16;
  }
}

// bs_round_A: L ^= f(R, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator).
__host__ __device__ __forceinline__ void bs_round_A(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  const uint32_t s0_0 = w[1];
  const uint32_t s0_1 = w[63];
  const uint32_t s0_2 = w[55];
  const uint32_t s0_3 = w[47];
  const uint32_t s0_4 = w[39];
  const uint32_t s0_5 = w[31];
  const uint32_t s1_0 = bs_correct(w[39], m[0], m[48]);
  const uint32_t s1_1 = bs_correct(w[31], m[1], m[49]);
  const uint32_t s1_2 = w[23];
  const uint32_t s1_3 = w[15];
  const uint32_t s1_4 = w[7];
  const uint32_t s1_5 = w[61];
  const uint32_t s2_0 = bs_correct(w[7], m[2], m[50]);
  const uint32_t s2_1 = bs_correct(w[61], m[3], m[51]);
  const uint32_t s2_2 = w[53];
  const uint32_t s2_3 = w[45];
  const uint32_t s2_4 = w[37];
  const uint32_t s2_5 = w[29];
  const uint32_t s3_0 = bs_correct(w[37], m[4], m[52]);
  const uint32_t s3_1 = bs_correct(w[29], m[5], m[53]);
  const uint32_t s3_2 = w[21];
  const uint32_t s3_3 = w[13];
  const uint32_t s3_4 = w[5];
  const uint32_t s3_5 = w[59];
  const uint32_t s4_0 = bs_correct(w[5], m[6], m[54]);
  const uint32_t s4_1 = bs_correct(w[59], m[7], m[55]);
  const uint32_t s4_2 = w[51];
  const uint32_t s4_3 = w[43];
  const uint32_t s4_4 = w[35];
  const uint32_t s4_5 = w[27];
  const uint32_t s5_0 = bs_correct(w[35], m[8], m[56]);
  const uint32_t s5_1 = bs_correct(w[27], m[9], m[57]);
  const uint32_t s5_2 = w[19];
  const uint32_t s5_3 = w[11];
  const uint32_t s5_4 = w[3];
  const uint32_t s5_5 = w[57];
  const uint32_t s6_0 = bs_correct(w[3], m[10], m[58]);
  const uint32_t s6_1 = bs_correct(w[57], m[11], m[59]);
  const uint32_t s6_2 = w[49];
  const uint32_t s6_3 = w[41];
  const uint32_t s6_4 = w[33];
  const uint32_t s6_5 = w[25];
  const uint32_t s7_0 = bs_correct(w[33], m[12], m[60]);
  const uint32_t s7_1 = bs_correct(w[25], m[13], m[61]);
  const uint32_t s7_2 = w[17];
  const uint32_t s7_3 = w[9];
  const uint32_t s7_4 = bs_correct(w[1], m[14], m[62]);
  const uint32_t s7_5 = bs_correct(w[63], m[15], m[63]);
  const uint32_t s0_6 = lop3<0x1b>(s0_2, s0_1, s0_0);
  const uint32_t s0_7 = lop3<0x86>(s0_3, s0_4, s0_5);
  const uint32_t s0_8 = lop3<0xda>(s0_0, s0_4, s0_3);
  const uint32_t s1_6 = lop3<0x69>(s1_4, s1_3, s1_0);
  const uint32_t s1_7 = lop3<0x39>(s1_5, s1_2, s1_3);
  const uint32_t s1_8 = lop3<0x6e>(s1_4, s1_2, s1_5);
  const uint32_t s2_6 = lop3<0x96>(s2_5, s2_1, s2_3);
  const uint32_t s2_10 = lop3<0xd5>(s2_1, s2_2, s2_5);
  const uint32_t s3_6 = lop3<0x86>(s3_3, s3_4, s3_1);
  const uint32_t s3_8 = lop3<0xc1>(s3_1, s3_2, s3_4);
  const uint32_t s3_9 = lop3<0x3d>(s3_1, s3_2, s3_4);
  const uint32_t s4_6 = lop3<0x4a>(s4_0, s4_2, s4_5);
  const uint32_t s4_8 = lop3<0xb9>(s4_0, s4_1, s4_2);
  const uint32_t s4_10 = lop3<0xca>(s4_5, s4_1, s4_2);
  const uint32_t s4_12 = lop3<0x96>(s4_1, s4_3, s4_5);
  const uint32_t s4_15 = lop3<0x86>(s4_1, s4_2, s4_4);
  const uint32_t s4_23 = lop3<0xb6>(s4_0, s4_2, s4_4);
  const uint32_t s5_6 = lop3<0x63>(s5_1, s5_0, s5_3);
  const uint32_t s6_6 = lop3<0x69>(s6_3, s6_0, s6_4);
  const uint32_t s6_7 = lop3<0x39>(s6_4, s6_1, s6_3);
  const uint32_t s6_16 = lop3<0x6d>(s6_2, s6_0, s6_3);
  const uint32_t s7_6 = lop3<0xf2>(s7_2, s7_0, s7_4);
  const uint32_t s7_8 = lop3<0xd0>(s7_0, s7_5, s7_3);
  const uint32_t s7_9 = lop3<0xa9>(s7_3, s7_4, s7_2);
  const uint32_t s0_9 = lop3<0xd2>(s0_7, s0_1, s0_8);
  const uint32_t s1_9 = lop3<0x6a>(s1_5, s1_2, s1_6);
  const uint32_t s1_10 = lop3<0x5e>(s1_5, s1_0, s1_6);
  const uint32_t s1_11 = lop3<0x56>(s1_6, s1_5, s1_7);
  const uint32_t s2_7 = lop3<0x96>(s2_3, s2_2, s2_6);
  const uint32_t s2_27 = lop3<0x96>(s2_2, s2_4, s2_6);
  const uint32_t s3_7 = lop3<0xc6>(s3_1, s3_6, s3_2);
  const uint32_t s3_10 = lop3<0xe2>(s3_4, s3_6, s3_8);
  const uint32_t s3_12 = lop3<0xc6>(s3_6, s3_9, s3_3);
  const uint32_t s4_7 = lop3<0x9c>(s4_1, s4_6, s4_2);
  const uint32_t s4_11 = lop3<0x5c>(s4_3, s4_10, s4_8);
  const uint32_t s4_16 = lop3<0x7c>(s4_12, s4_1, s4_4);
  const uint32_t s4_30 = lop3<0xb6>(s4_1, s4_4, s4_6);
  const uint32_t s5_7 = lop3<0x82>(s5_6, s5_1, s5_3);
  const uint32_t s5_8 = lop3<0x96>(s5_3, s5_5, s5_6);
  const uint32_t s6_8 = lop3<0xc6>(s6_2, s6_6, s6_7);
  const uint32_t s7_7 = lop3<0xb6>(s7_5, s7_6, s7_4);
  const uint32_t s7_10 = lop3<0xc5>(s7_1, s7_3, s7_6);
  const uint32_t s7_11 = lop3<0xd6>(s7_1, s7_0, s7_9);
  const uint32_t s7_12 = lop3<0x6d>(s7_3, s7_8, s7_0);
  const uint32_t s7_16 = lop3<0x2a>(s7_4, s7_5, s7_8);
  const uint32_t s0_10 = lop3<0x76>(s0_7, s0_5, s0_9);
  const uint32_t s1_12 = lop3<0x78>(s1_9, s1_8, s1_0);
  const uint32_t s1_14 = lop3<0x65>(s1_3, s1_10, s1_9);
  const uint32_t s1_15 = lop3<0x74>(s1_11, s1_6, s1_8);
  const uint32_t s2_8 = lop3<0xac>(s2_4, s2_6, s2_7);
  const uint32_t s2_9 = lop3<0x46>(s2_1, s2_4, s2_7);
  const uint32_t s2_19 = lop3<0x76>(s2_3, s2_4, s2_7);
  const uint32_t s3_11 = lop3<0xac>(s3_0, s3_10, s3_7);
  const uint32_t s3_13 = lop3<0x61>(s3_4, s3_10, s3_12);
  const uint32_t s3_16 = lop3<0xa3>(s3_0, s3_6, s3_10);
  const uint32_t s4_9 = lop3<0x6c>(s4_3, s4_7, s4_8);
  const uint32_t s4_13 = lop3<0x2c>(s4_0, s4_11, s4_12);
  const uint32_t s4_17 = lop3<0xc6>(s4_3, s4_15, s4_16);
  const uint32_t s4_19 = lop3<0x3e>(s4_2, s4_5, s4_16);
  const uint32_t s5_9 = lop3<0xda>(s5_4, s5_7, s5_8);
  const uint32_t s5_12 = lop3<0xe3>(s5_0, s5_4, s5_8);
  const uint32_t s6_9 = lop3<0x97>(s6_7, s6_1, s6_8);
  const uint32_t s6_23 = lop3<0x67>(s6_8, s6_3, s6_4);
  const uint32_t s7_13 = lop3<0x2e>(s7_1, s7_11, s7_8);
  const uint32_t s7_14 = lop3<0x32>(s7_8, s7_12, s7_4);
  const uint32_t s7_17 = lop3<0x9c>(s7_0, s7_11, s7_2);
  const uint32_t s0_11 = lop3<0x6d>(s0_1, s0_0, s0_10);
  const uint32_t s0_12 = lop3<0xda>(s0_9, s0_2, s0_10);
  const uint32_t s1_13 = lop3<0xe2>(s1_12, s1_0, s1_7);
  const uint32_t s1_16 = lop3<0x36>(s1_1, s1_12, s1_2);
  const uint32_t s1_17 = lop3<0xbc>(s1_12, s1_5, s1_0);
  const uint32_t s2_11 = lop3<0xc6>(s2_3, s2_9, s2_10);
  const uint32_t s2_13 = lop3<0x1a>(s2_8, s2_1, s2_2);
  const uint32_t s2_15 = lop3<0xb2>(s2_1, s2_4, s2_8);
  const uint32_t s3_14 = lop3<0xac>(s3_0, s3_12, s3_13);
  const uint32_t s3_17 = lop3<0xa9>(s3_11, s3_4, s3_12);
  const uint32_t s4_14 = lop3<0xca>(s4_4, s4_9, s4_13);
  const uint32_t s4_28 = lop3<0x6e>(s4_6, s4_1, s4_13);
  const uint32_t s5_10 = lop3<0xb7>(s5_1, s5_0, s5_9);
  const uint32_t s6_10 = lop3<0xb1>(s6_9, s6_2, s6_7);
  const uint32_t s7_15 = lop3<0x96>(s7_14, s7_7, s7_13);
  const uint32_t s7_18 = lop3<0x6c>(s7_10, s7_17, s7_4);
  const uint32_t s7_23 = lop3<0x36>(s7_16, s7_6, s7_14);
  const uint32_t s7_24 = lop3<0xbf>(s7_12, s7_7, s7_17);
  const uint32_t s0_13 = lop3<0x7b>(s0_12, s0_8, s0_3);
  const uint32_t s0_16 = lop3<0x76>(s0_11, s0_9, s0_3);
  const uint32_t s0_19 = lop3<0xdc>(s0_12, s0_4, s0_6);
  const uint32_t s1_18 = lop3<0xba>(s1_0, s1_17, s1_7);
  const uint32_t s1_19 = lop3<0x2d>(s1_13, s1_3, s1_10);
  const uint32_t s1_20 = lop3<0x2d>(s1_11, s1_4, s1_17);
  const uint32_t s1_21 = lop3<0xe2>(s1_14, s1_4, s1_16);
  const uint32_t s2_12 = lop3<0xac>(s2_0, s2_8, s2_11);
  const uint32_t s2_14 = lop3<0xac>(s2_4, s2_13, s2_6);
  const uint32_t s3_15 = lop3<0xca>(s3_5, s3_14, s3_11);
  const uint32_t s3_18 = lop3<0x74>(s3_14, s3_5, s3_11);
  const uint32_t s3_19 = lop3<0x9c>(s3_17, s3_16, s3_1);
  const uint32_t s3_20 = lop3<0x49>(s3_4, s3_16, s3_14);
  const uint32_t s3_21 = lop3<0xe3>(s3_2, s3_10, s3_14);
  const uint32_t s4_18 = lop3<0x83>(s4_9, s4_14, s4_15);
  const uint32_t s5_11 = lop3<0x6c>(s5_0, s5_10, s5_4);
  const uint32_t s6_11 = lop3<0xac>(s6_0, s6_9, s6_10);
  const uint32_t s6_20 = lop3<0x65>(s6_10, s6_0, s6_6);
  const uint32_t s7_19 = lop3<0x96>(s7_9, s7_8, s7_15);
  const uint32_t s7_20 = lop3<0xac>(s7_4, s7_18, s7_10);
  const uint32_t s7_25 = lop3<0x78>(s7_23, s7_1, s7_24);
  const uint32_t s0_14 = lop3<0x39>(s0_11, s0_4, s0_13);
  const uint32_t s0_17 = lop3<0xe2>(s0_13, s0_7, s0_1);
  const uint32_t s1_22 = lop3<0x72>(s1_21, s1_20, s1_1);
  const uint32_t s1_23 = lop3<0x24>(s1_4, s1_19, s1_18);
  const uint32_t s1_27 = lop3<0xe2>(s1_12, s1_1, s1_19);
  const uint32_t s2_16 = lop3<0x6c>(s2_3, s2_14, s2_15);
  const uint32_t s2_17 = lop3<0xfd>(s2_14, s2_2, s2_8);
  const uint32_t s3_22 = lop3<0xd8>(s3_20, s3_21, s3_3);
  const uint32_t s4_20 = lop3<0xac>(s4_1, s4_18, s4_19);
  const uint32_t s5_13 = lop3<0xcb>(s5_3, s5_11, s5_12);
  const uint32_t s6_12 = lop3<0xac>(s6_5, s6_8, s6_11);
  const uint32_t s6_14 = lop3<0xbd>(s6_11, s6_0, s6_5);
  const uint32_t s6_21 = lop3<0xac>(s6_5, s6_11, s6_20);
  const uint32_t s7_21 = lop3<0x6a>(s7_3, s7_20, s7_19);
  const uint32_t s0_15 = lop3<0xc6>(s0_2, s0_9, s0_14);
  const uint32_t s0_18 = lop3<0xc5>(s0_0, s0_17, s0_16);
  const uint32_t s0_21 = lop3<0x27>(s0_8, s0_9, s0_14);
  const uint32_t s1_24 = lop3<0xd2>(s1_23, s1_15, s1_0);
  const uint32_t s1_25 = lop3<0x67>(s1_14, s1_16, s1_23);
  const uint32_t s1_28 = lop3<0x39>(s1_23, s1_1, s1_5);
  const uint32_t s2_18 = lop3<0x6c>(s2_0, s2_16, s2_17);
  const uint32_t s2_20 = lop3<0x87>(s2_14, s2_2, s2_16);
  const uint32_t s2_29 = lop3<0xde>(s2_16, s2_11, s2_27);
  const uint32_t s3_23 = lop3<0xb4>(s3_19, s3_22, s3_5);
  const uint32_t s4_21 = lop3<0xc6>(s4_0, s4_17, s4_20);
  const uint32_t s4_25 = lop3<0x21>(s4_13, s4_18, s4_20);
  const uint32_t s5_14 = lop3<0x6a>(s5_2, s5_13, s5_9);
  const uint32_t s5_17 = lop3<0xa9>(s5_2, s5_13, s5_8);
  const uint32_t s6_13 = lop3<0x47>(s6_4, s6_0, s6_12);
  const uint32_t s6_17 = lop3<0xad>(s6_14, s6_2, s6_8);
  const uint32_t s6_26 = lop3<0xd6>(s6_3, s6_10, s6_21);
  const uint32_t s7_22 = lop3<0xb8>(s7_18, s7_5, s7_21);
  const uint32_t s0_20 = lop3<0x6a>(s0_19, s0_2, s0_18);
  const uint32_t s0_30 = lop3<0x7d>(s0_15, s0_10, s0_7);
  const uint32_t s1_26 = lop3<0xd6>(s1_1, s1_24, s1_25);
  const uint32_t s1_29 = lop3<0xc6>(s1_28, s1_6, s1_18);
  const uint32_t s2_21 = lop3<0xc6>(s2_0, s2_19, s2_20);
  const uint32_t s2_22 = lop3<0x76>(s2_18, s2_4, s2_6);
  const uint32_t s3_24 = lop3<0x69>(s3_22, s3_23, s3_5);
  const uint32_t s4_22 = lop3<0x97>(s4_6, s4_18, s4_21);
  const uint32_t s4_27 = lop3<0x16>(s4_17, s4_12, s4_25);
  const uint32_t s5_15 = lop3<0xc6>(s5_14, s5_3, s5_10);
  const uint32_t s5_16 = lop3<0x78>(s5_8, s5_3, s5_14);
  const uint32_t s5_19 = lop3<0x97>(s5_9, s5_14, s5_5);
  const uint32_t s6_15 = lop3<0x6c>(s6_3, s6_13, s6_14);
  const uint32_t s6_18 = lop3<0xbc>(s6_5, s6_16, s6_17);
  const uint32_t s7_26 = lop3<0x95>(s7_22, s7_4, s7_23);
  const uint32_t s0_22 = lop3<0x97>(s0_0, s0_20, s0_21);
  const uint32_t s0_24 = lop3<0x7e>(s0_0, s0_1, s0_20);
  const uint32_t s2_23 = lop3<0x7e>(s2_4, s2_0, s2_21);
  const uint32_t s4_24 = lop3<0xac>(s4_3, s4_22, s4_23);
  const uint32_t s4_29 = lop3<0xc6>(s4_4, s4_27, s4_28);
  const uint32_t s5_18 = lop3<0x87>(s5_15, s5_17, s5_4);
  const uint32_t s5_20 = lop3<0x93>(s5_19, s5_17, s5_4);
  const uint32_t s5_21 = lop3<0x7a>(s5_3, s5_19, s5_2);
  const uint32_t s6_19 = lop3<0x6c>(s6_1, s6_15, s6_18);
  const uint32_t s6_22 = lop3<0x69>(s6_10, s6_3, s6_18);
  const uint32_t s7_27 = lop3<0x2e>(s7_21, s7_3, s7_26);
  const uint32_t s0_23 = lop3<0xe2>(s0_22, s0_2, s0_21);
  const uint32_t s0_25 = lop3<0xd3>(s0_24, s0_5, s0_6);
  const uint32_t s2_24 = lop3<0xc6>(s2_2, s2_22, s2_23);
  const uint32_t s4_26 = lop3<0xbc>(s4_12, s4_24, s4_25);
  const uint32_t s4_31 = lop3<0xc6>(s4_22, s4_29, s4_30);
  const uint32_t s5_22 = lop3<0x95>(s5_1, s5_21, s5_8);
  const uint32_t s5_27 = lop3<0xac>(s5_1, s5_20, s5_18);
  const uint32_t s5_30 = lop3<0x97>(s5_1, s5_13, s5_20);
  const uint32_t s6_24 = lop3<0xc6>(s6_2, s6_22, s6_23);
  const uint32_t s7_28 = lop3<0x2e>(s7_18, s7_5, s7_27);
  const uint32_t s0_26 = lop3<0x6c>(s0_3, s0_23, s0_25);
  const uint32_t s2_25 = lop3<0xca>(s2_1, s2_21, s2_24);
  const uint32_t s5_23 = lop3<0x5c>(s5_12, s5_3, s5_22);
  const uint32_t s6_25 = lop3<0xca>(s6_1, s6_21, s6_24);
  const uint32_t s0_27 = lop3<0x96>(s0_20, s0_26, s0_15);
  const uint32_t s0_28 = lop3<0x98>(s0_26, s0_5, s0_15);
  const uint32_t s2_26 = lop3<0x85>(s2_25, s2_4, s2_8);
  const uint32_t s5_24 = lop3<0x1b>(s5_23, s5_1, s5_5);
  const uint32_t s6_27 = lop3<0x2e>(s6_14, s6_21, s6_25);
  const uint32_t s6_29 = lop3<0x69>(s6_10, s6_19, s6_25);
  const uint32_t s0_29 = lop3<0x6a>(s0_4, s0_28, s0_27);
  const uint32_t s2_28 = lop3<0x2c>(s2_1, s2_26, s2_27);
  const uint32_t s5_25 = lop3<0xe2>(s5_23, s5_2, s5_24);
  const uint32_t s6_28 = lop3<0xc6>(s6_2, s6_26, s6_27);
  const uint32_t s0_31 = lop3<0xb4>(s0_29, s0_30, s0_1);
  const uint32_t s2_30 = lop3<0xc2>(s2_0, s2_28, s2_29);
  const uint32_t s5_26 = lop3<0xb8>(s5_25, s5_4, s5_22);
  const uint32_t s6_30 = lop3<0xc6>(s6_20, s6_28, s6_29);
  const uint32_t s5_28 = lop3<0xbe>(s5_26, s5_7, s5_0);
  const uint32_t s5_29 = lop3<0x99>(s5_22, s5_28, s5_16);
  const uint32_t s5_31 = lop3<0xd2>(s5_29, s5_2, s5_30);
  w[60] = lop3<0x96>(w[60], s0_15, m[24]);
  w[58] = lop3<0x96>(w[58], s0_31, m[32]);
  w[10] = lop3<0x96>(w[10], s0_26, m[38]);
  w[8] = lop3<0x96>(w[8], s0_20, m[46]);
  w[28] = lop3<0x96>(w[28], s1_27, m[28]);
  w[32] = lop3<0x96>(w[32], s1_29, m[43]);
  w[54] = lop3<0x96>(w[54], s1_26, m[17]);
  w[50] = lop3<0x96>(w[50], s1_22, m[33]);
  w[2] = lop3<0x96>(w[2], s2_30, m[39]);
  w[4] = lop3<0x96>(w[4], s2_18, m[31]);
  w[16] = lop3<0x96>(w[16], s2_25, m[45]);
  w[22] = lop3<0x96>(w[22], s2_12, m[21]);
  w[48] = lop3<0x69>(w[48], s3_18, m[41]);
  w[34] = lop3<0x96>(w[34], s3_15, m[35]);
  w[52] = lop3<0x96>(w[52], s3_23, m[25]);
  w[62] = lop3<0x96>(w[62], s3_24, m[16]);
  w[6] = lop3<0x96>(w[6], s4_31, m[23]);
  w[20] = lop3<0x96>(w[20], s4_26, m[29]);
  w[56] = lop3<0x96>(w[56], s4_21, m[40]);
  w[46] = lop3<0x96>(w[46], s4_14, m[18]);
  w[38] = lop3<0x96>(w[38], s5_26, m[19]);
  w[24] = lop3<0x96>(w[24], s5_14, m[44]);
  w[44] = lop3<0x96>(w[44], s5_27, m[26]);
  w[42] = lop3<0x96>(w[42], s5_31, m[34]);
  w[0] = lop3<0x96>(w[0], s6_25, m[47]);
  w[36] = lop3<0x96>(w[36], s6_19, m[27]);
  w[18] = lop3<0x96>(w[18], s6_30, m[37]);
  w[14] = lop3<0x96>(w[14], s6_12, m[22]);
  w[30] = lop3<0x96>(w[30], s7_28, m[20]);
  w[40] = lop3<0x96>(w[40], s7_15, m[42]);
  w[12] = lop3<0x96>(w[12], s7_25, m[30]);
  w[26] = lop3<0x96>(w[26], s7_22, m[36]);
}

// bs_round_B: R ^= f(L, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator).
__host__ __device__ __forceinline__ void bs_round_B(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  const uint32_t s0_0 = w[0];
  const uint32_t s0_1 = w[62];
  const uint32_t s0_2 = w[54];
  const uint32_t s0_3 = w[46];
  const uint32_t s0_4 = w[38];
  const uint32_t s0_5 = w[30];
  const uint32_t s1_0 = bs_correct(w[38], m[0], m[48]);
  const uint32_t s1_1 = bs_correct(w[30], m[1], m[49]);
  const uint32_t s1_2 = w[22];
  const uint32_t s1_3 = w[14];
  const uint32_t s1_4 = w[6];
  const uint32_t s1_5 = w[60];
  const uint32_t s2_0 = bs_correct(w[6], m[2], m[50]);
  const uint32_t s2_1 = bs_correct(w[60], m[3], m[51]);
  const uint32_t s2_2 = w[52];
  const uint32_t s2_3 = w[44];
  const uint32_t s2_4 = w[36];
  const uint32_t s2_5 = w[28];
  const uint32_t s3_0 = bs_correct(w[36], m[4], m[52]);
  const uint32_t s3_1 = bs_correct(w[28], m[5], m[53]);
  const uint32_t s3_2 = w[20];
  const uint32_t s3_3 = w[12];
  const uint32_t s3_4 = w[4];
  const uint32_t s3_5 = w[58];
  const uint32_t s4_0 = bs_correct(w[4], m[6], m[54]);
  const uint32_t s4_1 = bs_correct(w[58], m[7], m[55]);
  const uint32_t s4_2 = w[50];
  const uint32_t s4_3 = w[42];
  const uint32_t s4_4 = w[34];
  const uint32_t s4_5 = w[26];
  const uint32_t s5_0 = bs_correct(w[34], m[8], m[56]);
  const uint32_t s5_1 = bs_correct(w[26], m[9], m[57]);
  const uint32_t s5_2 = w[18];
  const uint32_t s5_3 = w[10];
  const uint32_t s5_4 = w[2];
  const uint32_t s5_5 = w[56];
  const uint32_t s6_0 = bs_correct(w[2], m[10], m[58]);
  const uint32_t s6_1 = bs_correct(w[56], m[11], m[59]);
  const uint32_t s6_2 = w[48];
  const uint32_t s6_3 = w[40];
  const uint32_t s6_4 = w[32];
  const uint32_t s6_5 = w[24];
  const uint32_t s7_0 = bs_correct(w[32], m[12], m[60]);
  const uint32_t s7_1 = bs_correct(w[24], m[13], m[61]);
  const uint32_t s7_2 = w[16];
  const uint32_t s7_3 = w[8];
  const uint32_t s7_4 = bs_correct(w[0], m[14], m[62]);
  const uint32_t s7_5 = bs_correct(w[62], m[15], m[63]);
  const uint32_t s0_6 = lop3<0x1b>(s0_2, s0_1, s0_0);
  const uint32_t s0_7 = lop3<0x86>(s0_3, s0_4, s0_5);
  const uint32_t s0_8 = lop3<0xda>(s0_0, s0_4, s0_3);
  const uint32_t s1_6 = lop3<0x69>(s1_4, s1_3, s1_0);
  const uint32_t s1_7 = lop3<0x39>(s1_5, s1_2, s1_3);
  const uint32_t s1_8 = lop3<0x6e>(s1_4, s1_2, s1_5);
  const uint32_t s2_6 = lop3<0x96>(s2_5, s2_1, s2_3);
  const uint32_t s2_10 = lop3<0xd5>(s2_1, s2_2, s2_5);
  const uint32_t s3_6 = lop3<0x86>(s3_3, s3_4, s3_1);
  const uint32_t s3_8 = lop3<0xc1>(s3_1, s3_2, s3_4);
  const uint32_t s3_9 = lop3<0x3d>(s3_1, s3_2, s3_4);
  const uint32_t s4_6 = lop3<0x4a>(s4_0, s4_2, s4_5);
  const uint32_t s4_8 = lop3<0xb9>(s4_0, s4_1, s4_2);
  const uint32_t s4_10 = lop3<0xca>(s4_5, s4_1, s4_2);
  const uint32_t s4_12 = lop3<0x96>(s4_1, s4_3, s4_5);
  const uint32_t s4_15 = lop3<0x86>(s4_1, s4_2, s4_4);
  const uint32_t s4_23 = lop3<0xb6>(s4_0, s4_2, s4_4);
  const uint32_t s5_6 = lop3<0x63>(s5_1, s5_0, s5_3);
  const uint32_t s6_6 = lop3<0x69>(s6_3, s6_0, s6_4);
  const uint32_t s6_7 = lop3<0x39>(s6_4, s6_1, s6_3);
  const uint32_t s6_16 = lop3<0x6d>(s6_2, s6_0, s6_3);
  const uint32_t s7_6 = lop3<0xf2>(s7_2, s7_0, s7_4);
  const uint32_t s7_8 = lop3<0xd0>(s7_0, s7_5, s7_3);
  const uint32_t s7_9 = lop3<0xa9>(s7_3, s7_4, s7_2);
  const uint32_t s0_9 = lop3<0xd2>(s0_7, s0_1, s0_8);
  const uint32_t s1_9 = lop3<0x6a>(s1_5, s1_2, s1_6);
  const uint32_t s1_10 = lop3<0x5e>(s1_5, s1_0, s1_6);
  const uint32_t s1_11 = lop3<0x56>(s1_6, s1_5, s1_7);
  const uint32_t s2_7 = lop3<0x96>(s2_3, s2_2, s2_6);
  const uint32_t s2_27 = lop3<0x96>(s2_2, s2_4, s2_6);
  const uint32_t s3_7 = lop3<0xc6>(s3_1, s3_6, s3_2);
  const uint32_t s3_10 = lop3<0xe2>(s3_4, s3_6, s3_8);
  const uint32_t s3_12 = lop3<0xc6>(s3_6, s3_9, s3_3);
  const uint32_t s4_7 = lop3<0x9c>(s4_1, s4_6, s4_2);
  const uint32_t s4_11 = lop3<0x5c>(s4_3, s4_10, s4_8);
  const uint32_t s4_16 = lop3<0x7c>(s4_12, s4_1, s4_4);
  const uint32_t s4_30 = lop3<0xb6>(s4_1, s4_4, s4_6);
  const uint32_t s5_7 = lop3<0x82>(s5_6, s5_1, s5_3);
  const uint32_t s5_8 = lop3<0x96>(s5_3, s5_5, s5_6);
  const uint32_t s6_8 = lop3<0xc6>(s6_2, s6_6, s6_7);
  const uint32_t s7_7 = lop3<0xb6>(s7_5, s7_6, s7_4);
  const uint32_t s7_10 = lop3<0xc5>(s7_1, s7_3, s7_6);
  const uint32_t s7_11 = lop3<0xd6>(s7_1, s7_0, s7_9);
  const uint32_t s7_12 = lop3<0x6d>(s7_3, s7_8, s7_0);
  const uint32_t s7_16 = lop3<0x2a>(s7_4, s7_5, s7_8);
  const uint32_t s0_10 = lop3<0x76>(s0_7, s0_5, s0_9);
  const uint32_t s1_12 = lop3<0x78>(s1_9, s1_8, s1_0);
  const uint32_t s1_14 = lop3<0x65>(s1_3, s1_10, s1_9);
  const uint32_t s1_15 = lop3<0x74>(s1_11, s1_6, s1_8);
  const uint32_t s2_8 = lop3<0xac>(s2_4, s2_6, s2_7);
  const uint32_t s2_9 = lop3<0x46>(s2_1, s2_4, s2_7);
  const uint32_t s2_19 = lop3<0x76>(s2_3, s2_4, s2_7);
  const uint32_t s3_11 = lop3<0xac>(s3_0, s3_10, s3_7);
  const uint32_t s3_13 = lop3<0x61>(s3_4, s3_10, s3_12);
  const uint32_t s3_16 = lop3<0xa3>(s3_0, s3_6, s3_10);
  const uint32_t s4_9 = lop3<0x6c>(s4_3, s4_7, s4_8);
  const uint32_t s4_13 = lop3<0x2c>(s4_0, s4_11, s4_12);
  const uint32_t s4_17 = lop3<0xc6>(s4_3, s4_15, s4_16);
  const uint32_t s4_19 = lop3<0x3e>(s4_2, s4_5, s4_16);
  const uint32_t s5_9 = lop3<0xda>(s5_4, s5_7, s5_8);
  const uint32_t s5_12 = lop3<0xe3>(s5_0, s5_4, s5_8);
  const uint32_t s6_9 = lop3<0x97>(s6_7, s6_1, s6_8);
  const uint32_t s6_23 = lop3<0x67>(s6_8, s6_3, s6_4);
  const uint32_t s7_13 = lop3<0x2e>(s7_1, s7_11, s7_8);
  const uint32_t s7_14 = lop3<0x32>(s7_8, s7_12, s7_4);
  const uint32_t s7_17 = lop3<0x9c>(s7_0, s7_11, s7_2);
  const uint32_t s0_11 = lop3<0x6d>(s0_1, s0_0, s0_10);
  const uint32_t s0_12 = lop3<0xda>(s0_9, s0_2, s0_10);
  const uint32_t s1_13 = lop3<0xe2>(s1_12, s1_0, s1_7);
  const uint32_t s1_16 = lop3<0x36>(s1_1, s1_12, s1_2);
  const uint32_t s1_17 = lop3<0xbc>(s1_12, s1_5, s1_0);
  const uint32_t s2_11 = lop3<0xc6>(s2_3, s2_9, s2_10);
  const uint32_t s2_13 = lop3<0x1a>(s2_8, s2_1, s2_2);
  const uint32_t s2_15 = lop3<0xb2>(s2_1, s2_4, s2_8);
  const uint32_t s3_14 = lop3<0xac>(s3_0, s3_12, s3_13);
  const uint32_t s3_17 = lop3<0xa9>(s3_11, s3_4, s3_12);
  const uint32_t s4_14 = lop3<0xca>(s4_4, s4_9, s4_13);
  const uint32_t s4_28 = lop3<0x6e>(s4_6, s4_1, s4_13);
  const uint32_t s5_10 = lop3<0xb7>(s5_1, s5_0, s5_9);
  const uint32_t s6_10 = lop3<0xb1>(s6_9, s6_2, s6_7);
  const uint32_t s7_15 = lop3<0x96>(s7_14, s7_7, s7_13);
  const uint32_t s7_18 = lop3<0x6c>(s7_10, s7_17, s7_4);
  const uint32_t s7_23 = lop3<0x36>(s7_16, s7_6, s7_14);
  const uint32_t s7_24 = lop3<0xbf>(s7_12, s7_7, s7_17);
  const uint32_t s0_13 = lop3<0x7b>(s0_12, s0_8, s0_3);
  const uint32_t s0_16 = lop3<0x76>(s0_11, s0_9, s0_3);
  const uint32_t s0_19 = lop3<0xdc>(s0_12, s0_4, s0_6);
  const uint32_t s1_18 = lop3<0xba>(s1_0, s1_17, s1_7);
  const uint32_t s1_19 = lop3<0x2d>(s1_13, s1_3, s1_10);
  const uint32_t s1_20 = lop3<0x2d>(s1_11, s1_4, s1_17);
  const uint32_t s1_21 = lop3<0xe2>(s1_14, s1_4, s1_16);
  const uint32_t s2_12 = lop3<0xac>(s2_0, s2_8, s2_11);
  const uint32_t s2_14 = lop3<0xac>(s2_4, s2_13, s2_6);
  const uint32_t s3_15 = lop3<0xca>(s3_5, s3_14, s3_11);
  const uint32_t s3_18 = lop3<0x74>(s3_14, s3_5, s3_11);
  const uint32_t s3_19 = lop3<0x9c>(s3_17, s3_16, s3_1);
  const uint32_t s3_20 = lop3<0x49>(s3_4, s3_16, s3_14);
  const uint32_t s3_21 = lop3<0xe3>(s3_2, s3_10, s3_14);
  const uint32_t s4_18 = lop3<0x83>(s4_9, s4_14, s4_15);
  const uint32_t s5_11 = lop3<0x6c>(s5_0, s5_10, s5_4);
  const uint32_t s6_11 = lop3<0xac>(s6_0, s6_9, s6_10);
  const uint32_t s6_20 = lop3<0x65>(s6_10, s6_0, s6_6);
  const uint32_t s7_19 = lop3<0x96>(s7_9, s7_8, s7_15);
  const uint32_t s7_20 = lop3<0xac>(s7_4, s7_18, s7_10);
  const uint32_t s7_25 = lop3<0x78>(s7_23, s7_1, s7_24);
  const uint32_t s0_14 = lop3<0x39>(s0_11, s0_4, s0_13);
  const uint32_t s0_17 = lop3<0xe2>(s0_13, s0_7, s0_1);
  const uint32_t s1_22 = lop3<0x72>(s1_21, s1_20, s1_1);
  const uint32_t s1_23 = lop3<0x24>(s1_4, s1_19, s1_18);
  const uint32_t s1_27 = lop3<0xe2>(s1_12, s1_1, s1_19);
  const uint32_t s2_16 = lop3<0x6c>(s2_3, s2_14, s2_15);
  const uint32_t s2_17 = lop3<0xfd>(s2_14, s2_2, s2_8);
  const uint32_t s3_22 = lop3<0xd8>(s3_20, s3_21, s3_3);
  const uint32_t s4_20 = lop3<0xac>(s4_1, s4_18, s4_19);
  const uint32_t s5_13 = lop3<0xcb>(s5_3, s5_11, s5_12);
  const uint32_t s6_12 = lop3<0xac>(s6_5, s6_8, s6_11);
  const uint32_t s6_14 = lop3<0xbd>(s6_11, s6_0, s6_5);
  const uint32_t s6_21 = lop3<0xac>(s6_5, s6_11, s6_20);
  const uint32_t s7_21 = lop3<0x6a>(s7_3, s7_20, s7_19);
  const uint32_t s0_15 = lop3<0xc6>(s0_2, s0_9, s0_14);
  const uint32_t s0_18 = lop3<0xc5>(s0_0, s0_17, s0_16);
  const uint32_t s0_21 = lop3<0x27>(s0_8, s0_9, s0_14);
  const uint32_t s1_24 = lop3<0xd2>(s1_23, s1_15, s1_0);
  const uint32_t s1_25 = lop3<0x67>(s1_14, s1_16, s1_23);
  const uint32_t s1_28 = lop3<0x39>(s1_23, s1_1, s1_5);
  const uint32_t s2_18 = lop3<0x6c>(s2_0, s2_16, s2_17);
  const uint32_t s2_20 = lop3<0x87>(s2_14, s2_2, s2_16);
  const uint32_t s2_29 = lop3<0xde>(s2_16, s2_11, s2_27);
  const uint32_t s3_23 = lop3<0xb4>(s3_19, s3_22, s3_5);
  const uint32_t s4_21 = lop3<0xc6>(s4_0, s4_17, s4_20);
  const uint32_t s4_25 = lop3<0x21>(s4_13, s4_18, s4_20);
  const uint32_t s5_14 = lop3<0x6a>(s5_2, s5_13, s5_9);
  const uint32_t s5_17 = lop3<0xa9>(s5_2, s5_13, s5_8);
  const uint32_t s6_13 = lop3<0x47>(s6_4, s6_0, s6_12);
  const uint32_t s6_17 = lop3<0xad>(s6_14, s6_2, s6_8);
  const uint32_t s6_26 = lop3<0xd6>(s6_3, s6_10, s6_21);
  const uint32_t s7_22 = lop3<0xb8>(s7_18, s7_5, s7_21);
  const uint32_t s0_20 = lop3<0x6a>(s0_19, s0_2, s0_18);
  const uint32_t s0_30 = lop3<0x7d>(s0_15, s0_10, s0_7);
  const uint32_t s1_26 = lop3<0xd6>(s1_1, s1_24, s1_25);
  const uint32_t s1_29 = lop3<0xc6>(s1_28, s1_6, s1_18);
  const uint32_t s2_21 = lop3<0xc6>(s2_0, s2_19, s2_20);
  const uint32_t s2_22 = lop3<0x76>(s2_18, s2_4, s2_6);
  const uint32_t s3_24 = lop3<0x69>(s3_22, s3_23, s3_5);
  const uint32_t s4_22 = lop3<0x97>(s4_6, s4_18, s4_21);
  const uint32_t s4_27 = lop3<0x16>(s4_17, s4_12, s4_25);
  const uint32_t s5_15 = lop3<0xc6>(s5_14, s5_3, s5_10);
  const uint32_t s5_16 = lop3<0x78>(s5_8, s5_3, s5_14);
  const uint32_t s5_19 = lop3<0x97>(s5_9, s5_14, s5_5);
  const uint32_t s6_15 = lop3<0x6c>(s6_3, s6_13, s6_14);
  const uint32_t s6_18 = lop3<0xbc>(s6_5, s6_16, s6_17);
  const uint32_t s7_26 = lop3<0x95>(s7_22, s7_4, s7_23);
  const uint32_t s0_22 = lop3<0x97>(s0_0, s0_20, s0_21);
  const uint32_t s0_24 = lop3<0x7e>(s0_0, s0_1, s0_20);
  const uint32_t s2_23 = lop3<0x7e>(s2_4, s2_0, s2_21);
  const uint32_t s4_24 = lop3<0xac>(s4_3, s4_22, s4_23);
  const uint32_t s4_29 = lop3<0xc6>(s4_4, s4_27, s4_28);
  const uint32_t s5_18 = lop3<0x87>(s5_15, s5_17, s5_4);
  const uint32_t s5_20 = lop3<0x93>(s5_19, s5_17, s5_4);
  const uint32_t s5_21 = lop3<0x7a>(s5_3, s5_19, s5_2);
  const uint32_t s6_19 = lop3<0x6c>(s6_1, s6_15, s6_18);
  const uint32_t s6_22 = lop3<0x69>(s6_10, s6_3, s6_18);
  const uint32_t s7_27 = lop3<0x2e>(s7_21, s7_3, s7_26);
  const uint32_t s0_23 = lop3<0xe2>(s0_22, s0_2, s0_21);
  const uint32_t s0_25 = lop3<0xd3>(s0_24, s0_5, s0_6);
  const uint32_t s2_24 = lop3<0xc6>(s2_2, s2_22, s2_23);
  const uint32_t s4_26 = lop3<0xbc>(s4_12, s4_24, s4_25);
  const uint32_t s4_31 = lop3<0xc6>(s4_22, s4_29, s4_30);
  const uint32_t s5_22 = lop3<0x95>(s5_1, s5_21, s5_8);
  const uint32_t s5_27 = lop3<0xac>(s5_1, s5_20, s5_18);
  const uint32_t s5_30 = lop3<0x97>(s5_1, s5_13, s5_20);
  const uint32_t s6_24 = lop3<0xc6>(s6_2, s6_22, s6_23);
  const uint32_t s7_28 = lop3<0x2e>(s7_18, s7_5, s7_27);
  const uint32_t s0_26 = lop3<0x6c>(s0_3, s0_23, s0_25);
  const uint32_t s2_25 = lop3<0xca>(s2_1, s2_21, s2_24);
  const uint32_t s5_23 = lop3<0x5c>(s5_12, s5_3, s5_22);
  const uint32_t s6_25 = lop3<0xca>(s6_1, s6_21, s6_24);
  const uint32_t s0_27 = lop3<0x96>(s0_20, s0_26, s0_15);
  const uint32_t s0_28 = lop3<0x98>(s0_26, s0_5, s0_15);
  const uint32_t s2_26 = lop3<0x85>(s2_25, s2_4, s2_8);
  const uint32_t s5_24 = lop3<0x1b>(s5_23, s5_1, s5_5);
  const uint32_t s6_27 = lop3<0x2e>(s6_14, s6_21, s6_25);
  const uint32_t s6_29 = lop3<0x69>(s6_10, s6_19, s6_25);
  const uint32_t s0_29 = lop3<0x6a>(s0_4, s0_28, s0_27);
  const uint32_t s2_28 = lop3<0x2c>(s2_1, s2_26, s2_27);
  const uint32_t s5_25 = lop3<0xe2>(s5_23, s5_2, s5_24);
  const uint32_t s6_28 = lop3<0xc6>(s6_2, s6_26, s6_27);
  const uint32_t s0_31 = lop3<0xb4>(s0_29, s0_30, s0_1);
  const uint32_t s2_30 = lop3<0xc2>(s2_0, s2_28, s2_29);
  const uint32_t s5_26 = lop3<0xb8>(s5_25, s5_4, s5_22);
  const uint32_t s6_30 = lop3<0xc6>(s6_20, s6_28, s6_29);
  const uint32_t s5_28 = lop3<0xbe>(s5_26, s5_7, s5_0);
  const uint32_t s5_29 = lop3<0x99>(s5_22, s5_28, s5_16);
  const uint32_t s5_31 = lop3<0xd2>(s5_29, s5_2, s5_30);
  w[61] = lop3<0x96>(w[61], s0_15, m[24]);
  w[59] = lop3<0x96>(w[59], s0_31, m[32]);
  w[11] = lop3<0x96>(w[11], s0_26, m[38]);
  w[9] = lop3<0x96>(w[9], s0_20, m[46]);
  w[29] = lop3<0x96>(w[29], s1_27, m[28]);
  w[33] = lop3<0x96>(w[33], s1_29, m[43]);
  w[55] = lop3<0x96>(w[55], s1_26, m[17]);
  w[51] = lop3<0x96>(w[51], s1_22, m[33]);
  w[3] = lop3<0x96>(w[3], s2_30, m[39]);
  w[5] = lop3<0x96>(w[5], s2_18, m[31]);
  w[17] = lop3<0x96>(w[17], s2_25, m[45]);
  w[23] = lop3<0x96>(w[23], s2_12, m[21]);
  w[49] = lop3<0x69>(w[49], s3_18, m[41]);
  w[35] = lop3<0x96>(w[35], s3_15, m[35]);
  w[53] = lop3<0x96>(w[53], s3_23, m[25]);
  w[63] = lop3<0x96>(w[63], s3_24, m[16]);
  w[7] = lop3<0x96>(w[7], s4_31, m[23]);
  w[21] = lop3<0x96>(w[21], s4_26, m[29]);
  w[57] = lop3<0x96>(w[57], s4_21, m[40]);
  w[47] = lop3<0x96>(w[47], s4_14, m[18]);
  w[39] = lop3<0x96>(w[39], s5_26, m[19]);
  w[25] = lop3<0x96>(w[25], s5_14, m[44]);
  w[45] = lop3<0x96>(w[45], s5_27, m[26]);
  w[43] = lop3<0x96>(w[43], s5_31, m[34]);
  w[1] = lop3<0x96>(w[1], s6_25, m[47]);
  w[37] = lop3<0x96>(w[37], s6_19, m[27]);
  w[19] = lop3<0x96>(w[19], s6_30, m[37]);
  w[15] = lop3<0x96>(w[15], s6_12, m[22]);
  w[31] = lop3<0x96>(w[31], s7_28, m[20]);
  w[41] = lop3<0x96>(w[41], s7_15, m[42]);
  w[13] = lop3<0x96>(w[13], s7_25, m[30]);
  w[27] = lop3<0x96>(w[27], s7_22, m[36]);
}

// bs_round_A_f: L ^= f(R, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator); m[64 + f]: multiplier of fold f's mask change.
__host__ __device__ __forceinline__ void bs_round_A_f(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  const uint32_t s0_0 = w[1];
  const uint32_t s0_1 = w[63];
  const uint32_t s0_2 = w[55];
  const uint32_t s0_3 = w[47];
  const uint32_t s0_4 = w[39];
  const uint32_t s0_5 = w[31];
  const uint32_t s1_0 = bs_correct(w[39], m[0], m[48]);
  const uint32_t s1_1 = bs_correct(w[31], m[1], m[49]);
  const uint32_t s1_2 = w[23];
  const uint32_t s1_3 = w[15];
  const uint32_t s1_4 = w[7];
  const uint32_t s1_5 = w[61];
  const uint32_t s2_0 = bs_correct(w[7], m[2], m[50]);
  const uint32_t s2_1 = bs_correct(w[61], m[3], m[51]);
  const uint32_t s2_2 = w[53];
  const uint32_t s2_3 = w[45];
  const uint32_t s2_4 = w[37];
  const uint32_t s2_5 = w[29];
  const uint32_t s3_0 = bs_correct(w[37], m[4], m[52]);
  const uint32_t s3_1 = bs_correct(w[29], m[5], m[53]);
  const uint32_t s3_2 = w[21];
  const uint32_t s3_3 = w[13];
  const uint32_t s3_4 = w[5];
  const uint32_t s3_5 = w[59];
  const uint32_t s4_0 = bs_correct(w[5], m[6], m[54]);
  const uint32_t s4_1 = bs_correct(w[59], m[7], m[55]);
  const uint32_t s4_2 = w[51];
  const uint32_t s4_3 = w[43];
  const uint32_t s4_4 = w[35];
  const uint32_t s4_5 = w[27];
  const uint32_t s5_0 = bs_correct(w[35], m[8], m[56]);
  const uint32_t s5_1 = bs_correct(w[27], m[9], m[57]);
  const uint32_t s5_2 = w[19];
  const uint32_t s5_3 = w[11];
  const uint32_t s5_4 = w[3];
  const uint32_t s5_5 = w[57];
  const uint32_t s6_0 = bs_correct(w[3], m[10], m[58]);
  const uint32_t s6_1 = bs_correct(w[57], m[11], m[59]);
  const uint32_t s6_2 = w[49];
  const uint32_t s6_3 = w[41];
  const uint32_t s6_4 = w[33];
  const uint32_t s6_5 = w[25];
  const uint32_t s7_0 = bs_correct(w[33], m[12], m[60]);
  const uint32_t s7_1 = bs_correct(w[25], m[13], m[61]);
  const uint32_t s7_2 = w[17];
  const uint32_t s7_3 = w[9];
  const uint32_t s7_4 = bs_correct(w[1], m[14], m[62]);
  const uint32_t s7_5 = bs_correct(w[63], m[15], m[63]);
  const uint32_t s0_6 = lop3<0x1b>(s0_2, s0_1, s0_0);
  const uint32_t s0_7 = lop3<0x86>(s0_3, s0_4, s0_5);
  const uint32_t s0_8 = lop3<0xda>(s0_0, s0_4, s0_3);
  const uint32_t s1_6 = lop3<0x69>(s1_4, s1_3, s1_0);
  const uint32_t s1_7 = lop3<0x39>(s1_5, s1_2, s1_3);
  const uint32_t s1_8 = lop3<0x6e>(s1_4, s1_2, s1_5);
  const uint32_t s2_6 = lop3<0x96>(s2_5, s2_1, s2_3);
  const uint32_t s2_10 = lop3<0xd5>(s2_1, s2_2, s2_5);
  const uint32_t s3_6 = lop3<0x3d>(s3_2, s3_1, s3_4);
  const uint32_t s3_7 = lop3<0x3e>(s3_2, s3_1, s3_4);
  const uint32_t s3_8 = lop3<0x86>(s3_3, s3_4, s3_1);
  const uint32_t s4_6 = lop3<0x4a>(s4_0, s4_2, s4_5);
  const uint32_t s4_8 = lop3<0xb9>(s4_0, s4_1, s4_2);
  const uint32_t s4_10 = lop3<0xca>(s4_5, s4_1, s4_2);
  const uint32_t s4_12 = lop3<0x96>(s4_1, s4_3, s4_5);
  const uint32_t s4_15 = lop3<0x86>(s4_1, s4_2, s4_4);
  const uint32_t s4_23 = lop3<0xb6>(s4_0, s4_2, s4_4);
  const uint32_t s5_6 = lop3<0x63>(s5_1, s5_0, s5_3);
  const uint32_t s6_6 = lop3<0x69>(s6_3, s6_0, s6_4);
  const uint32_t s6_7 = lop3<0x39>(s6_4, s6_1, s6_3);
  const uint32_t s6_16 = lop3<0x6d>(s6_2, s6_0, s6_3);
  const uint32_t s7_6 = lop3<0xf2>(s7_2, s7_0, s7_4);
  const uint32_t s7_8 = lop3<0xd0>(s7_0, s7_5, s7_3);
  const uint32_t s7_9 = lop3<0xa9>(s7_3, s7_4, s7_2);
  const uint32_t s0_9 = lop3<0xd2>(s0_7, s0_1, s0_8);
  const uint32_t s1_9 = lop3<0x6a>(s1_5, s1_2, s1_6);
  const uint32_t s1_10 = lop3<0x5e>(s1_5, s1_0, s1_6);
  const uint32_t s1_11 = lop3<0x56>(s1_6, s1_5, s1_7);
  const uint32_t s2_7 = lop3<0x96>(s2_3, s2_2, s2_6);
  const uint32_t s2_27 = lop3<0x96>(s2_2, s2_4, s2_6);
  const uint32_t s3_9 = lop3<0x68>(s3_2, s3_8, s3_7);
  const uint32_t s3_10 = lop3<0xb1>(s3_4, s3_7, s3_8);
  const uint32_t s3_12 = lop3<0x9a>(s3_3, s3_8, s3_6);
  const uint32_t s4_7 = lop3<0x9c>(s4_1, s4_6, s4_2);
  const uint32_t s4_11 = lop3<0x5c>(s4_3, s4_10, s4_8);
  const uint32_t s4_16 = lop3<0x7c>(s4_12, s4_1, s4_4);
  const uint32_t s4_30 = lop3<0xb6>(s4_1, s4_4, s4_6);
  const uint32_t s5_7 = lop3<0x82>(s5_6, s5_1, s5_3);
  const uint32_t s5_8 = lop3<0x96>(s5_3, s5_5, s5_6);
  const uint32_t s6_8 = lop3<0xc6>(s6_2, s6_6, s6_7);
  const uint32_t s7_7 = lop3<0xb6>(s7_5, s7_6, s7_4);
  const uint32_t s7_10 = lop3<0xc5>(s7_1, s7_3, s7_6);
  const uint32_t s7_11 = lop3<0xd6>(s7_1, s7_0, s7_9);
  const uint32_t s7_12 = lop3<0x6d>(s7_3, s7_8, s7_0);
  const uint32_t s7_16 = lop3<0x2a>(s7_4, s7_5, s7_8);
  const uint32_t s0_10 = lop3<0x76>(s0_7, s0_5, s0_9);
  const uint32_t s1_12 = lop3<0x78>(s1_9, s1_8, s1_0);
  const uint32_t s1_14 = lop3<0x65>(s1_3, s1_10, s1_9);
  const uint32_t s1_15 = lop3<0x74>(s1_11, s1_6, s1_8);
  const uint32_t s2_8 = lop3<0xac>(s2_4, s2_6, s2_7);
  const uint32_t s2_9 = lop3<0x46>(s2_1, s2_4, s2_7);
  const uint32_t s2_19 = lop3<0x76>(s2_3, s2_4, s2_7);
  const uint32_t s3_11 = lop3<0xb8>(s3_10, s3_0, s3_9);
  const uint32_t s3_13 = lop3<0x49>(s3_12, s3_4, s3_10);
  const uint32_t s3_19 = lop3<0x8d>(s3_8, s3_10, s3_0);
  const uint32_t s4_9 = lop3<0x6c>(s4_3, s4_7, s4_8);
  const uint32_t s4_13 = lop3<0x2c>(s4_0, s4_11, s4_12);
  const uint32_t s4_17 = lop3<0xc6>(s4_3, s4_15, s4_16);
  const uint32_t s4_19 = lop3<0x3e>(s4_2, s4_5, s4_16);
  const uint32_t s5_9 = lop3<0xda>(s5_4, s5_7, s5_8);
  const uint32_t s5_12 = lop3<0xe3>(s5_0, s5_4, s5_8);
  const uint32_t s6_9 = lop3<0x97>(s6_7, s6_1, s6_8);
  const uint32_t s6_23 = lop3<0x67>(s6_8, s6_3, s6_4);
  const uint32_t s7_13 = lop3<0x2e>(s7_1, s7_11, s7_8);
  const uint32_t s7_14 = lop3<0x32>(s7_8, s7_12, s7_4);
  const uint32_t s7_17 = lop3<0x9c>(s7_0, s7_11, s7_2);
  const uint32_t s0_11 = lop3<0x6d>(s0_1, s0_0, s0_10);
  const uint32_t s0_12 = lop3<0xda>(s0_9, s0_2, s0_10);
  const uint32_t s1_13 = lop3<0xe2>(s1_12, s1_0, s1_7);
  const uint32_t s1_16 = lop3<0x36>(s1_1, s1_12, s1_2);
  const uint32_t s1_17 = lop3<0xbc>(s1_12, s1_5, s1_0);
  const uint32_t s2_11 = lop3<0xc6>(s2_3, s2_9, s2_10);
  const uint32_t s2_13 = lop3<0x1a>(s2_8, s2_1, s2_2);
  const uint32_t s2_15 = lop3<0xb2>(s2_1, s2_4, s2_8);
  const uint32_t s3_14 = lop3<0xe2>(s3_13, s3_0, s3_12);
  const uint32_t s3_18 = lop3<0xc9>(s3_11, s3_12, s3_4);
  const uint32_t s4_14 = lop3<0xca>(s4_4, s4_9, s4_13);
  const uint32_t s4_28 = lop3<0x6e>(s4_6, s4_1, s4_13);
  const uint32_t s5_10 = lop3<0xb7>(s5_1, s5_0, s5_9);
  const uint32_t s6_10 = lop3<0xb1>(s6_9, s6_2, s6_7);
  const uint32_t s7_15 = lop3<0x96>(s7_14, s7_7, s7_13);
  const uint32_t s7_18 = lop3<0x6c>(s7_10, s7_17, s7_4);
  const uint32_t s7_23 = lop3<0x36>(s7_16, s7_6, s7_14);
  const uint32_t s7_24 = lop3<0xbf>(s7_12, s7_7, s7_17);
  const uint32_t s0_13 = lop3<0x7b>(s0_12, s0_8, s0_3);
  const uint32_t s0_16 = lop3<0x76>(s0_11, s0_9, s0_3);
  const uint32_t s0_19 = lop3<0xdc>(s0_12, s0_4, s0_6);
  const uint32_t s1_18 = lop3<0xba>(s1_0, s1_17, s1_7);
  const uint32_t s1_19 = lop3<0x2d>(s1_13, s1_3, s1_10);
  const uint32_t s1_20 = lop3<0x2d>(s1_11, s1_4, s1_17);
  const uint32_t s1_21 = lop3<0xe2>(s1_14, s1_4, s1_16);
  const uint32_t s2_12 = lop3<0xac>(s2_0, s2_8, s2_11);
  const uint32_t s2_14 = lop3<0xac>(s2_4, s2_13, s2_6);
  const uint32_t s3_15 = lop3<0xd9>(s3_14, s3_2, s3_10);
  const uint32_t s3_16 = lop3<0x74>(s3_14, s3_5, s3_11);
  const uint32_t s3_17 = lop3<0xac>(s3_5, s3_11, s3_14);
  const uint32_t s3_20 = lop3<0xb4>(s3_19, s3_18, s3_1);
  const uint32_t s3_21 = lop3<0x49>(s3_4, s3_19, s3_14);
  const uint32_t s4_18 = lop3<0x83>(s4_9, s4_14, s4_15);
  const uint32_t s5_11 = lop3<0x6c>(s5_0, s5_10, s5_4);
  const uint32_t s6_11 = lop3<0xac>(s6_0, s6_9, s6_10);
  const uint32_t s6_20 = lop3<0x65>(s6_10, s6_0, s6_6);
  const uint32_t s7_19 = lop3<0x96>(s7_9, s7_8, s7_15);
  const uint32_t s7_20 = lop3<0xac>(s7_4, s7_18, s7_10);
  const uint32_t s7_25 = lop3<0x78>(s7_23, s7_1, s7_24);
  const uint32_t s0_14 = lop3<0x39>(s0_11, s0_4, s0_13);
  const uint32_t s0_17 = lop3<0xe2>(s0_13, s0_7, s0_1);
  const uint32_t s1_22 = lop3<0x72>(s1_21, s1_20, s1_1);
  const uint32_t s1_23 = lop3<0x24>(s1_4, s1_19, s1_18);
  const uint32_t s1_27 = lop3<0xe2>(s1_12, s1_1, s1_19);
  const uint32_t s2_16 = lop3<0x6c>(s2_3, s2_14, s2_15);
  const uint32_t s2_17 = lop3<0xfd>(s2_14, s2_2, s2_8);
  const uint32_t s3_22 = lop3<0xca>(s3_3, s3_15, s3_21);
  const uint32_t s4_20 = lop3<0xac>(s4_1, s4_18, s4_19);
  const uint32_t s5_13 = lop3<0xcb>(s5_3, s5_11, s5_12);
  const uint32_t s6_12 = lop3<0xac>(s6_5, s6_8, s6_11);
  const uint32_t s6_14 = lop3<0xbd>(s6_11, s6_0, s6_5);
  const uint32_t s6_21 = lop3<0xac>(s6_5, s6_11, s6_20);
  const uint32_t s7_21 = lop3<0x6a>(s7_3, s7_20, s7_19);
  const uint32_t s0_15 = lop3<0xc6>(s0_2, s0_9, s0_14);
  const uint32_t s0_18 = lop3<0xc5>(s0_0, s0_17, s0_16);
  const uint32_t s0_21 = lop3<0x27>(s0_8, s0_9, s0_14);
  const uint32_t s1_24 = lop3<0xd2>(s1_23, s1_15, s1_0);
  const uint32_t s1_25 = lop3<0x67>(s1_14, s1_16, s1_23);
  const uint32_t s1_28 = lop3<0x39>(s1_23, s1_1, s1_5);
  const uint32_t s2_18 = lop3<0x6c>(s2_0, s2_16, s2_17);
  const uint32_t s2_20 = lop3<0x87>(s2_14, s2_2, s2_16);
  const uint32_t s2_29 = lop3<0xde>(s2_16, s2_11, s2_27);
  const uint32_t s3_23 = lop3<0x36>(s3_22, s3_20, s3_5);
  const uint32_t s4_21 = lop3<0xc6>(s4_0, s4_17, s4_20);
  const uint32_t s4_25 = lop3<0x21>(s4_13, s4_18, s4_20);
  const uint32_t s5_14 = lop3<0x6a>(s5_2, s5_13, s5_9);
  const uint32_t s5_17 = lop3<0xa9>(s5_2, s5_13, s5_8);
  const uint32_t s6_13 = lop3<0x47>(s6_4, s6_0, s6_12);
  const uint32_t s6_17 = lop3<0xad>(s6_14, s6_2, s6_8);
  const uint32_t s6_26 = lop3<0xd6>(s6_3, s6_10, s6_21);
  const uint32_t s7_22 = lop3<0xb8>(s7_18, s7_5, s7_21);
  const uint32_t s0_20 = lop3<0x6a>(s0_19, s0_2, s0_18);
  const uint32_t s0_30 = lop3<0x7d>(s0_15, s0_10, s0_7);
  const uint32_t s1_26 = lop3<0xd6>(s1_1, s1_24, s1_25);
  const uint32_t s1_29 = lop3<0xc6>(s1_28, s1_6, s1_18);
  const uint32_t s2_21 = lop3<0xc6>(s2_0, s2_19, s2_20);
  const uint32_t s2_22 = lop3<0x76>(s2_18, s2_4, s2_6);
  const uint32_t s3_24 = lop3<0x69>(s3_22, w[62], s3_23);
  const uint32_t s3_25 = lop3<0x96>(s3_5, w[52], s3_23);
  const uint32_t s4_22 = lop3<0x97>(s4_6, s4_18, s4_21);
  const uint32_t s4_27 = lop3<0x16>(s4_17, s4_12, s4_25);
  const uint32_t s5_15 = lop3<0xc6>(s5_14, s5_3, s5_10);
  const uint32_t s5_16 = lop3<0x78>(s5_8, s5_3, s5_14);
  const uint32_t s5_19 = lop3<0x97>(s5_9, s5_14, s5_5);
  const uint32_t s6_15 = lop3<0x6c>(s6_3, s6_13, s6_14);
  const uint32_t s6_18 = lop3<0xbc>(s6_5, s6_16, s6_17);
  const uint32_t s7_26 = lop3<0x95>(s7_22, s7_4, s7_23);
  const uint32_t s0_22 = lop3<0x97>(s0_0, s0_20, s0_21);
  const uint32_t s0_24 = lop3<0x7e>(s0_0, s0_1, s0_20);
  const uint32_t s2_23 = lop3<0x7e>(s2_4, s2_0, s2_21);
  const uint32_t s4_24 = lop3<0xac>(s4_3, s4_22, s4_23);
  const uint32_t s4_29 = lop3<0xc6>(s4_4, s4_27, s4_28);
  const uint32_t s5_18 = lop3<0x87>(s5_15, s5_17, s5_4);
  const uint32_t s5_20 = lop3<0x93>(s5_19, s5_17, s5_4);
  const uint32_t s5_21 = lop3<0x7a>(s5_3, s5_19, s5_2);
  const uint32_t s6_19 = lop3<0x6c>(s6_1, s6_15, s6_18);
  const uint32_t s6_22 = lop3<0x69>(s6_10, s6_3, s6_18);
  const uint32_t s7_27 = lop3<0x2e>(s7_21, s7_3, s7_26);
  const uint32_t s0_23 = lop3<0xe2>(s0_22, s0_2, s0_21);
  const uint32_t s0_25 = lop3<0xd3>(s0_24, s0_5, s0_6);
  const uint32_t s2_24 = lop3<0xc6>(s2_2, s2_22, s2_23);
  const uint32_t s4_26 = lop3<0xbc>(s4_12, s4_24, s4_25);
  const uint32_t s4_31 = lop3<0xc6>(s4_22, s4_29, s4_30);
  const uint32_t s5_22 = lop3<0x95>(s5_1, s5_21, s5_8);
  const uint32_t s5_27 = lop3<0xac>(s5_1, s5_20, s5_18);
  const uint32_t s5_30 = lop3<0x97>(s5_1, s5_13, s5_20);
  const uint32_t s6_24 = lop3<0xc6>(s6_2, s6_22, s6_23);
  const uint32_t s7_28 = lop3<0x2e>(s7_18, s7_5, s7_27);
  const uint32_t s0_26 = lop3<0x6c>(s0_3, s0_23, s0_25);
  const uint32_t s2_25 = lop3<0xca>(s2_1, s2_21, s2_24);
  const uint32_t s5_23 = lop3<0x5c>(s5_12, s5_3, s5_22);
  const uint32_t s6_25 = lop3<0xca>(s6_1, s6_21, s6_24);
  const uint32_t s0_27 = lop3<0x96>(s0_20, s0_26, s0_15);
  const uint32_t s0_28 = lop3<0x98>(s0_26, s0_5, s0_15);
  const uint32_t s2_26 = lop3<0x85>(s2_25, s2_4, s2_8);
  const uint32_t s5_24 = lop3<0x1b>(s5_23, s5_1, s5_5);
  const uint32_t s6_27 = lop3<0x2e>(s6_14, s6_21, s6_25);
  const uint32_t s6_29 = lop3<0x69>(s6_10, s6_19, s6_25);
  const uint32_t s0_29 = lop3<0x6a>(s0_4, s0_28, s0_27);
  const uint32_t s2_28 = lop3<0x2c>(s2_1, s2_26, s2_27);
  const uint32_t s5_25 = lop3<0xe2>(s5_23, s5_2, s5_24);
  const uint32_t s6_28 = lop3<0xc6>(s6_2, s6_26, s6_27);
  const uint32_t s0_31 = lop3<0xb4>(s0_29, s0_30, s0_1);
  const uint32_t s2_30 = lop3<0xc2>(s2_0, s2_28, s2_29);
  const uint32_t s5_26 = lop3<0xb8>(s5_25, s5_4, s5_22);
  const uint32_t s6_30 = lop3<0xc6>(s6_20, s6_28, s6_29);
  const uint32_t s5_28 = lop3<0xbe>(s5_26, s5_7, s5_0);
  const uint32_t s5_29 = lop3<0x69>(w[42], s5_28, s5_16);
  const uint32_t s5_31 = lop3<0xd2>(s5_29, s5_2, s5_30);
  w[60] = lop3<0x96>(w[60], s0_15, m[24]);
  w[58] = lop3<0x96>(w[58], s0_31, m[32]);
  w[10] = lop3<0x96>(w[10], s0_26, m[38]);
  w[8] = lop3<0x96>(w[8], s0_20, m[46]);
  w[28] = lop3<0x96>(w[28], s1_27, m[28]);
  w[32] = lop3<0x96>(w[32], s1_29, m[43]);
  w[54] = lop3<0x96>(w[54], s1_26, m[17]);
  w[50] = lop3<0x96>(w[50], s1_22, m[33]);
  w[2] = lop3<0x96>(w[2], s2_30, m[39]);
  w[4] = lop3<0x96>(w[4], s2_18, m[31]);
  w[16] = lop3<0x96>(w[16], s2_25, m[45]);
  w[22] = lop3<0x96>(w[22], s2_12, m[21]);
  w[48] = lop3<0x69>(w[48], s3_16, m[41]);
  w[34] = lop3<0x96>(w[34], s3_17, m[35]);
  w[52] = bs_correct(s3_25, m[25], m[64]);
  w[62] = bs_correct(s3_24, m[16], m[65]);
  w[6] = lop3<0x96>(w[6], s4_31, m[23]);
  w[20] = lop3<0x96>(w[20], s4_26, m[29]);
  w[56] = lop3<0x96>(w[56], s4_21, m[40]);
  w[46] = lop3<0x96>(w[46], s4_14, m[18]);
  w[38] = lop3<0x96>(w[38], s5_26, m[19]);
  w[24] = lop3<0x96>(w[24], s5_14, m[44]);
  w[44] = lop3<0x96>(w[44], s5_27, m[26]);
  w[42] = bs_correct(s5_31, m[34], m[66]);
  w[0] = lop3<0x96>(w[0], s6_25, m[47]);
  w[36] = lop3<0x96>(w[36], s6_19, m[27]);
  w[18] = lop3<0x96>(w[18], s6_30, m[37]);
  w[14] = lop3<0x96>(w[14], s6_12, m[22]);
  w[30] = lop3<0x96>(w[30], s7_28, m[20]);
  w[40] = lop3<0x96>(w[40], s7_15, m[42]);
  w[12] = lop3<0x96>(w[12], s7_25, m[30]);
  w[26] = lop3<0x96>(w[26], s7_22, m[36]);
}

// bs_round_B_f: R ^= f(L, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator); m[64 + f]: multiplier of fold f's mask change.
__host__ __device__ __forceinline__ void bs_round_B_f(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  const uint32_t s0_0 = w[0];
  const uint32_t s0_1 = w[62];
  const uint32_t s0_2 = w[54];
  const uint32_t s0_3 = w[46];
  const uint32_t s0_4 = w[38];
  const uint32_t s0_5 = w[30];
  const uint32_t s1_0 = bs_correct(w[38], m[0], m[48]);
  const uint32_t s1_1 = bs_correct(w[30], m[1], m[49]);
  const uint32_t s1_2 = w[22];
  const uint32_t s1_3 = w[14];
  const uint32_t s1_4 = w[6];
  const uint32_t s1_5 = w[60];
  const uint32_t s2_0 = bs_correct(w[6], m[2], m[50]);
  const uint32_t s2_1 = bs_correct(w[60], m[3], m[51]);
  const uint32_t s2_2 = w[52];
  const uint32_t s2_3 = w[44];
  const uint32_t s2_4 = w[36];
  const uint32_t s2_5 = w[28];
  const uint32_t s3_0 = bs_correct(w[36], m[4], m[52]);
  const uint32_t s3_1 = bs_correct(w[28], m[5], m[53]);
  const uint32_t s3_2 = w[20];
  const uint32_t s3_3 = w[12];
  const uint32_t s3_4 = w[4];
  const uint32_t s3_5 = w[58];
  const uint32_t s4_0 = bs_correct(w[4], m[6], m[54]);
  const uint32_t s4_1 = bs_correct(w[58], m[7], m[55]);
  const uint32_t s4_2 = w[50];
  const uint32_t s4_3 = w[42];
  const uint32_t s4_4 = w[34];
  const uint32_t s4_5 = w[26];
  const uint32_t s5_0 = bs_correct(w[34], m[8], m[56]);
  const uint32_t s5_1 = bs_correct(w[26], m[9], m[57]);
  const uint32_t s5_2 = w[18];
  const uint32_t s5_3 = w[10];
  const uint32_t s5_4 = w[2];
  const uint32_t s5_5 = w[56];
  const uint32_t s6_0 = bs_correct(w[2], m[10], m[58]);
  const uint32_t s6_1 = bs_correct(w[56], m[11], m[59]);
  const uint32_t s6_2 = w[48];
  const uint32_t s6_3 = w[40];
  const uint32_t s6_4 = w[32];
  const uint32_t s6_5 = w[24];
  const uint32_t s7_0 = bs_correct(w[32], m[12], m[60]);
  const uint32_t s7_1 = bs_correct(w[24], m[13], m[61]);
  const uint32_t s7_2 = w[16];
  const uint32_t s7_3 = w[8];
  const uint32_t s7_4 = bs_correct(w[0], m[14], m[62]);
  const uint32_t s7_5 = bs_correct(w[62], m[15], m[63]);
  const uint32_t s0_6 = lop3<0x1b>(s0_2, s0_1, s0_0);
  const uint32_t s0_7 = lop3<0x86>(s0_3, s0_4, s0_5);
  const uint32_t s0_8 = lop3<0xda>(s0_0, s0_4, s0_3);
  const uint32_t s1_6 = lop3<0x69>(s1_4, s1_3, s1_0);
  const uint32_t s1_7 = lop3<0x39>(s1_5, s1_2, s1_3);
  const uint32_t s1_8 = lop3<0x6e>(s1_4, s1_2, s1_5);
  const uint32_t s2_6 = lop3<0x96>(s2_5, s2_1, s2_3);
  const uint32_t s2_10 = lop3<0xd5>(s2_1, s2_2, s2_5);
  const uint32_t s3_6 = lop3<0x3d>(s3_2, s3_1, s3_4);
  const uint32_t s3_7 = lop3<0x3e>(s3_2, s3_1, s3_4);
  const uint32_t s3_8 = lop3<0x86>(s3_3, s3_4, s3_1);
  const uint32_t s4_6 = lop3<0x4a>(s4_0, s4_2, s4_5);
  const uint32_t s4_8 = lop3<0xb9>(s4_0, s4_1, s4_2);
  const uint32_t s4_10 = lop3<0xca>(s4_5, s4_1, s4_2);
  const uint32_t s4_12 = lop3<0x96>(s4_1, s4_3, s4_5);
  const uint32_t s4_15 = lop3<0x86>(s4_1, s4_2, s4_4);
  const uint32_t s4_23 = lop3<0xb6>(s4_0, s4_2, s4_4);
  const uint32_t s5_6 = lop3<0x63>(s5_1, s5_0, s5_3);
  const uint32_t s6_6 = lop3<0x69>(s6_3, s6_0, s6_4);
  const uint32_t s6_7 = lop3<0x39>(s6_4, s6_1, s6_3);
  const uint32_t s6_16 = lop3<0x6d>(s6_2, s6_0, s6_3);
  const uint32_t s7_6 = lop3<0xf2>(s7_2, s7_0, s7_4);
  const uint32_t s7_8 = lop3<0xd0>(s7_0, s7_5, s7_3);
  const uint32_t s7_9 = lop3<0xa9>(s7_3, s7_4, s7_2);
  const uint32_t s0_9 = lop3<0xd2>(s0_7, s0_1, s0_8);
  const uint32_t s1_9 = lop3<0x6a>(s1_5, s1_2, s1_6);
  const uint32_t s1_10 = lop3<0x5e>(s1_5, s1_0, s1_6);
  const uint32_t s1_11 = lop3<0x56>(s1_6, s1_5, s1_7);
  const uint32_t s2_7 = lop3<0x96>(s2_3, s2_2, s2_6);
  const uint32_t s2_27 = lop3<0x96>(s2_2, s2_4, s2_6);
  const uint32_t s3_9 = lop3<0x68>(s3_2, s3_8, s3_7);
  const uint32_t s3_10 = lop3<0xb1>(s3_4, s3_7, s3_8);
  const uint32_t s3_12 = lop3<0x9a>(s3_3, s3_8, s3_6);
  const uint32_t s4_7 = lop3<0x9c>(s4_1, s4_6, s4_2);
  const uint32_t s4_11 = lop3<0x5c>(s4_3, s4_10, s4_8);
  const uint32_t s4_16 = lop3<0x7c>(s4_12, s4_1, s4_4);
  const uint32_t s4_30 = lop3<0xb6>(s4_1, s4_4, s4_6);
  const uint32_t s5_7 = lop3<0x82>(s5_6, s5_1, s5_3);
  const uint32_t s5_8 = lop3<0x96>(s5_3, s5_5, s5_6);
  const uint32_t s6_8 = lop3<0xc6>(s6_2, s6_6, s6_7);
  const uint32_t s7_7 = lop3<0xb6>(s7_5, s7_6, s7_4);
  const uint32_t s7_10 = lop3<0xc5>(s7_1, s7_3, s7_6);
  const uint32_t s7_11 = lop3<0xd6>(s7_1, s7_0, s7_9);
  const uint32_t s7_12 = lop3<0x6d>(s7_3, s7_8, s7_0);
  const uint32_t s7_16 = lop3<0x2a>(s7_4, s7_5, s7_8);
  const uint32_t s0_10 = lop3<0x76>(s0_7, s0_5, s0_9);
  const uint32_t s1_12 = lop3<0x78>(s1_9, s1_8, s1_0);
  const uint32_t s1_14 = lop3<0x65>(s1_3, s1_10, s1_9);
  const uint32_t s1_15 = lop3<0x74>(s1_11, s1_6, s1_8);
  const uint32_t s2_8 = lop3<0xac>(s2_4, s2_6, s2_7);
  const uint32_t s2_9 = lop3<0x46>(s2_1, s2_4, s2_7);
  const uint32_t s2_19 = lop3<0x76>(s2_3, s2_4, s2_7);
  const uint32_t s3_11 = lop3<0xb8>(s3_10, s3_0, s3_9);
  const uint32_t s3_13 = lop3<0x49>(s3_12, s3_4, s3_10);
  const uint32_t s3_19 = lop3<0x8d>(s3_8, s3_10, s3_0);
  const uint32_t s4_9 = lop3<0x6c>(s4_3, s4_7, s4_8);
  const uint32_t s4_13 = lop3<0x2c>(s4_0, s4_11, s4_12);
  const uint32_t s4_17 = lop3<0xc6>(s4_3, s4_15, s4_16);
  const uint32_t s4_19 = lop3<0x3e>(s4_2, s4_5, s4_16);
  const uint32_t s5_9 = lop3<0xda>(s5_4, s5_7, s5_8);
  const uint32_t s5_12 = lop3<0xe3>(s5_0, s5_4, s5_8);
  const uint32_t s6_9 = lop3<0x97>(s6_7, s6_1, s6_8);
  const uint32_t s6_23 = lop3<0x67>(s6_8, s6_3, s6_4);
  const uint32_t s7_13 = lop3<0x2e>(s7_1, s7_11, s7_8);
  const uint32_t s7_14 = lop3<0x32>(s7_8, s7_12, s7_4);
  const uint32_t s7_17 = lop3<0x9c>(s7_0, s7_11, s7_2);
  const uint32_t s0_11 = lop3<0x6d>(s0_1, s0_0, s0_10);
  const uint32_t s0_12 = lop3<0xda>(s0_9, s0_2, s0_10);
  const uint32_t s1_13 = lop3<0xe2>(s1_12, s1_0, s1_7);
  const uint32_t s1_16 = lop3<0x36>(s1_1, s1_12, s1_2);
  const uint32_t s1_17 = lop3<0xbc>(s1_12, s1_5, s1_0);
  const uint32_t s2_11 = lop3<0xc6>(s2_3, s2_9, s2_10);
  const uint32_t s2_13 = lop3<0x1a>(s2_8, s2_1, s2_2);
  const uint32_t s2_15 = lop3<0xb2>(s2_1, s2_4, s2_8);
  const uint32_t s3_14 = lop3<0xe2>(s3_13, s3_0, s3_12);
  const uint32_t s3_18 = lop3<0xc9>(s3_11, s3_12, s3_4);
  const uint32_t s4_14 = lop3<0xca>(s4_4, s4_9, s4_13);
  const uint32_t s4_28 = lop3<0x6e>(s4_6, s4_1, s4_13);
  const uint32_t s5_10 = lop3<0xb7>(s5_1, s5_0, s5_9);
  const uint32_t s6_10 = lop3<0xb1>(s6_9, s6_2, s6_7);
  const uint32_t s7_15 = lop3<0x96>(s7_14, s7_7, s7_13);
  const uint32_t s7_18 = lop3<0x6c>(s7_10, s7_17, s7_4);
  const uint32_t s7_23 = lop3<0x36>(s7_16, s7_6, s7_14);
  const uint32_t s7_24 = lop3<0xbf>(s7_12, s7_7, s7_17);
  const uint32_t s0_13 = lop3<0x7b>(s0_12, s0_8, s0_3);
  const uint32_t s0_16 = lop3<0x76>(s0_11, s0_9, s0_3);
  const uint32_t s0_19 = lop3<0xdc>(s0_12, s0_4, s0_6);
  const uint32_t s1_18 = lop3<0xba>(s1_0, s1_17, s1_7);
  const uint32_t s1_19 = lop3<0x2d>(s1_13, s1_3, s1_10);
  const uint32_t s1_20 = lop3<0x2d>(s1_11, s1_4, s1_17);
  const uint32_t s1_21 = lop3<0xe2>(s1_14, s1_4, s1_16);
  const uint32_t s2_12 = lop3<0xac>(s2_0, s2_8, s2_11);
  const uint32_t s2_14 = lop3<0xac>(s2_4, s2_13, s2_6);
  const uint32_t s3_15 = lop3<0xd9>(s3_14, s3_2, s3_10);
  const uint32_t s3_16 = lop3<0x74>(s3_14, s3_5, s3_11);
  const uint32_t s3_17 = lop3<0xac>(s3_5, s3_11, s3_14);
  const uint32_t s3_20 = lop3<0xb4>(s3_19, s3_18, s3_1);
  const uint32_t s3_21 = lop3<0x49>(s3_4, s3_19, s3_14);
  const uint32_t s4_18 = lop3<0x83>(s4_9, s4_14, s4_15);
  const uint32_t s5_11 = lop3<0x6c>(s5_0, s5_10, s5_4);
  const uint32_t s6_11 = lop3<0xac>(s6_0, s6_9, s6_10);
  const uint32_t s6_20 = lop3<0x65>(s6_10, s6_0, s6_6);
  const uint32_t s7_19 = lop3<0x96>(s7_9, s7_8, s7_15);
  const uint32_t s7_20 = lop3<0xac>(s7_4, s7_18, s7_10);
  const uint32_t s7_25 = lop3<0x78>(s7_23, s7_1, s7_24);
  const uint32_t s0_14 = lop3<0x39>(s0_11, s0_4, s0_13);
  const uint32_t s0_17 = lop3<0xe2>(s0_13, s0_7, s0_1);
  const uint32_t s1_22 = lop3<0x72>(s1_21, s1_20, s1_1);
  const uint32_t s1_23 = lop3<0x24>(s1_4, s1_19, s1_18);
  const uint32_t s1_27 = lop3<0xe2>(s1_12, s1_1, s1_19);
  const uint32_t s2_16 = lop3<0x6c>(s2_3, s2_14, s2_15);
  const uint32_t s2_17 = lop3<0xfd>(s2_14, s2_2, s2_8);
  const uint32_t s3_22 = lop3<0xca>(s3_3, s3_15, s3_21);
  const uint32_t s4_20 = lop3<0xac>(s4_1, s4_18, s4_19);
  const uint32_t s5_13 = lop3<0xcb>(s5_3, s5_11, s5_12);
  const uint32_t s6_12 = lop3<0xac>(s6_5, s6_8, s6_11);
  const uint32_t s6_14 = lop3<0xbd>(s6_11, s6_0, s6_5);
  const uint32_t s6_21 = lop3<0xac>(s6_5, s6_11, s6_20);
  const uint32_t s7_21 = lop3<0x6a>(s7_3, s7_20, s7_19);
  const uint32_t s0_15 = lop3<0xc6>(s0_2, s0_9, s0_14);
  const uint32_t s0_18 = lop3<0xc5>(s0_0, s0_17, s0_16);
  const uint32_t s0_21 = lop3<0x27>(s0_8, s0_9, s0_14);
  const uint32_t s1_24 = lop3<0xd2>(s1_23, s1_15, s1_0);
  const uint32_t s1_25 = lop3<0x67>(s1_14, s1_16, s1_23);
  const uint32_t s1_28 = lop3<0x39>(s1_23, s1_1, s1_5);
  const uint32_t s2_18 = lop3<0x6c>(s2_0, s2_16, s2_17);
  const uint32_t s2_20 = lop3<0x87>(s2_14, s2_2, s2_16);
  const uint32_t s2_29 = lop3<0xde>(s2_16, s2_11, s2_27);
  const uint32_t s3_23 = lop3<0x36>(s3_22, s3_20, s3_5);
  const uint32_t s4_21 = lop3<0xc6>(s4_0, s4_17, s4_20);
  const uint32_t s4_25 = lop3<0x21>(s4_13, s4_18, s4_20);
  const uint32_t s5_14 = lop3<0x6a>(s5_2, s5_13, s5_9);
  const uint32_t s5_17 = lop3<0xa9>(s5_2, s5_13, s5_8);
  const uint32_t s6_13 = lop3<0x47>(s6_4, s6_0, s6_12);
  const uint32_t s6_17 = lop3<0xad>(s6_14, s6_2, s6_8);
  const uint32_t s6_26 = lop3<0xd6>(s6_3, s6_10, s6_21);
  const uint32_t s7_22 = lop3<0xb8>(s7_18, s7_5, s7_21);
  const uint32_t s0_20 = lop3<0x6a>(s0_19, s0_2, s0_18);
  const uint32_t s0_30 = lop3<0x7d>(s0_15, s0_10, s0_7);
  const uint32_t s1_26 = lop3<0xd6>(s1_1, s1_24, s1_25);
  const uint32_t s1_29 = lop3<0xc6>(s1_28, s1_6, s1_18);
  const uint32_t s2_21 = lop3<0xc6>(s2_0, s2_19, s2_20);
  const uint32_t s2_22 = lop3<0x76>(s2_18, s2_4, s2_6);
  const uint32_t s3_24 = lop3<0x69>(s3_22, w[63], s3_23);
  const uint32_t s3_25 = lop3<0x96>(s3_5, w[53], s3_23);
  const uint32_t s4_22 = lop3<0x97>(s4_6, s4_18, s4_21);
  const uint32_t s4_27 = lop3<0x16>(s4_17, s4_12, s4_25);
  const uint32_t s5_15 = lop3<0xc6>(s5_14, s5_3, s5_10);
  const uint32_t s5_16 = lop3<0x78>(s5_8, s5_3, s5_14);
  const uint32_t s5_19 = lop3<0x97>(s5_9, s5_14, s5_5);
  const uint32_t s6_15 = lop3<0x6c>(s6_3, s6_13, s6_14);
  const uint32_t s6_18 = lop3<0xbc>(s6_5, s6_16, s6_17);
  const uint32_t s7_26 = lop3<0x95>(s7_22, s7_4, s7_23);
  const uint32_t s0_22 = lop3<0x97>(s0_0, s0_20, s0_21);
  const uint32_t s0_24 = lop3<0x7e>(s0_0, s0_1, s0_20);
  const uint32_t s2_23 = lop3<0x7e>(s2_4, s2_0, s2_21);
  const uint32_t s4_24 = lop3<0xac>(s4_3, s4_22, s4_23);
  const uint32_t s4_29 = lop3<0xc6>(s4_4, s4_27, s4_28);
  const uint32_t s5_18 = lop3<0x87>(s5_15, s5_17, s5_4);
  const uint32_t s5_20 = lop3<0x93>(s5_19, s5_17, s5_4);
  const uint32_t s5_21 = lop3<0x7a>(s5_3, s5_19, s5_2);
  const uint32_t s6_19 = lop3<0x6c>(s6_1, s6_15, s6_18);
  const uint32_t s6_22 = lop3<0x69>(s6_10, s6_3, s6_18);
  const uint32_t s7_27 = lop3<0x2e>(s7_21, s7_3, s7_26);
  const uint32_t s0_23 = lop3<0xe2>(s0_22, s0_2, s0_21);
  const uint32_t s0_25 = lop3<0xd3>(s0_24, s0_5, s0_6);
  const uint32_t s2_24 = lop3<0xc6>(s2_2, s2_22, s2_23);
  const uint32_t s4_26 = lop3<0xbc>(s4_12, s4_24, s4_25);
  const uint32_t s4_31 = lop3<0xc6>(s4_22, s4_29, s4_30);
  const uint32_t s5_22 = lop3<0x95>(s5_1, s5_21, s5_8);
  const uint32_t s5_27 = lop3<0xac>(s5_1, s5_20, s5_18);
  const uint32_t s5_30 = lop3<0x97>(s5_1, s5_13, s5_20);
  const uint32_t s6_24 = lop3<0xc6>(s6_2, s6_22, s6_23);
  const uint32_t s7_28 = lop3<0x2e>(s7_18, s7_5, s7_27);
  const uint32_t s0_26 = lop3<0x6c>(s0_3, s0_23, s0_25);
  const uint32_t s2_25 = lop3<0xca>(s2_1, s2_21, s2_24);
  const uint32_t s5_23 = lop3<0x5c>(s5_12, s5_3, s5_22);
  const uint32_t s6_25 = lop3<0xca>(s6_1, s6_21, s6_24);
  const uint32_t s0_27 = lop3<0x96>(s0_20, s0_26, s0_15);
  const uint32_t s0_28 = lop3<0x98>(s0_26, s0_5, s0_15);
  const uint32_t s2_26 = lop3<0x85>(s2_25, s2_4, s2_8);
  const uint32_t s5_24 = lop3<0x1b>(s5_23, s5_1, s5_5);
  const uint32_t s6_27 = lop3<0x2e>(s6_14, s6_21, s6_25);
  const uint32_t s6_29 = lop3<0x69>(s6_10, s6_19, s6_25);
  const uint32_t s0_29 = lop3<0x6a>(s0_4, s0_28, s0_27);
  const uint32_t s2_28 = lop3<0x2c>(s2_1, s2_26, s2_27);
  const uint32_t s5_25 = lop3<0xe2>(s5_23, s5_2, s5_24);
  const uint32_t s6_28 = lop3<0xc6>(s6_2, s6_26, s6_27);
  const uint32_t s0_31 = lop3<0xb4>(s0_29, s0_30, s0_1);
  const uint32_t s2_30 = lop3<0xc2>(s2_0, s2_28, s2_29);
  const uint32_t s5_26 = lop3<0xb8>(s5_25, s5_4, s5_22);
  const uint32_t s6_30 = lop3<0xc6>(s6_20, s6_28, s6_29);
  const uint32_t s5_28 = lop3<0xbe>(s5_26, s5_7, s5_0);
  const uint32_t s5_29 = lop3<0x69>(w[43], s5_28, s5_16);
  const uint32_t s5_31 = lop3<0xd2>(s5_29, s5_2, s5_30);
  w[61] = lop3<0x96>(w[61], s0_15, m[24]);
  w[59] = lop3<0x96>(w[59], s0_31, m[32]);
  w[11] = lop3<0x96>(w[11], s0_26, m[38]);
  w[9] = lop3<0x96>(w[9], s0_20, m[46]);
  w[29] = lop3<0x96>(w[29], s1_27, m[28]);
  w[33] = lop3<0x96>(w[33], s1_29, m[43]);
  w[55] = lop3<0x96>(w[55], s1_26, m[17]);
  w[51] = lop3<0x96>(w[51], s1_22, m[33]);
  w[3] = lop3<0x96>(w[3], s2_30, m[39]);
  w[5] = lop3<0x96>(w[5], s2_18, m[31]);
  w[17] = lop3<0x96>(w[17], s2_25, m[45]);
  w[23] = lop3<0x96>(w[23], s2_12, m[21]);
  w[49] = lop3<0x69>(w[49], s3_16, m[41]);
  w[35] = lop3<0x96>(w[35], s3_17, m[35]);
  w[53] = bs_correct(s3_25, m[25], m[64]);
  w[63] = bs_correct(s3_24, m[16], m[65]);
  w[7] = lop3<0x96>(w[7], s4_31, m[23]);
  w[21] = lop3<0x96>(w[21], s4_26, m[29]);
  w[57] = lop3<0x96>(w[57], s4_21, m[40]);
  w[47] = lop3<0x96>(w[47], s4_14, m[18]);
  w[39] = lop3<0x96>(w[39], s5_26, m[19]);
  w[25] = lop3<0x96>(w[25], s5_14, m[44]);
  w[45] = lop3<0x96>(w[45], s5_27, m[26]);
  w[43] = bs_correct(s5_31, m[34], m[66]);
  w[1] = lop3<0x96>(w[1], s6_25, m[47]);
  w[37] = lop3<0x96>(w[37], s6_19, m[27]);
  w[19] = lop3<0x96>(w[19], s6_30, m[37]);
  w[15] = lop3<0x96>(w[15], s6_12, m[22]);
  w[31] = lop3<0x96>(w[31], s7_28, m[20]);
  w[41] = lop3<0x96>(w[41], s7_15, m[42]);
  w[13] = lop3<0x96>(w[13], s7_25, m[30]);
  w[27] = lop3<0x96>(w[27], s7_22, m[36]);
}

// bs_remask_L: XOR every L-plane i with m[i - 1].
__host__ __device__ __forceinline__ void bs_remask_L(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  w[62] ^= m[0];
  w[54] ^= m[1];
  w[46] ^= m[2];
  w[38] ^= m[3];
  w[30] ^= m[4];
  w[22] ^= m[5];
  w[14] ^= m[6];
  w[6] ^= m[7];
  w[60] ^= m[8];
  w[52] ^= m[9];
  w[44] ^= m[10];
  w[36] ^= m[11];
  w[28] ^= m[12];
  w[20] ^= m[13];
  w[12] ^= m[14];
  w[4] ^= m[15];
  w[58] ^= m[16];
  w[50] ^= m[17];
  w[42] ^= m[18];
  w[34] ^= m[19];
  w[26] ^= m[20];
  w[18] ^= m[21];
  w[10] ^= m[22];
  w[2] ^= m[23];
  w[56] ^= m[24];
  w[48] ^= m[25];
  w[40] ^= m[26];
  w[32] ^= m[27];
  w[24] ^= m[28];
  w[16] ^= m[29];
  w[8] ^= m[30];
  w[0] ^= m[31];
}

// bs_remask_R: XOR every R-plane i with m[i - 1].
__host__ __device__ __forceinline__ void bs_remask_R(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  w[63] ^= m[0];
  w[55] ^= m[1];
  w[47] ^= m[2];
  w[39] ^= m[3];
  w[31] ^= m[4];
  w[23] ^= m[5];
  w[15] ^= m[6];
  w[7] ^= m[7];
  w[61] ^= m[8];
  w[53] ^= m[9];
  w[45] ^= m[10];
  w[37] ^= m[11];
  w[29] ^= m[12];
  w[21] ^= m[13];
  w[13] ^= m[14];
  w[5] ^= m[15];
  w[59] ^= m[16];
  w[51] ^= m[17];
  w[43] ^= m[18];
  w[35] ^= m[19];
  w[27] ^= m[20];
  w[19] ^= m[21];
  w[11] ^= m[22];
  w[3] ^= m[23];
  w[57] ^= m[24];
  w[49] ^= m[25];
  w[41] ^= m[26];
  w[33] ^= m[27];
  w[25] ^= m[28];
  w[17] ^= m[29];
  w[9] ^= m[30];
  w[1] ^= m[31];
}

// bs_swap_halves: exchange the L-planes and the R-planes (so that one loop
// body of (round_A, round_B) can run all three DES of the pipeline).
__host__ __device__ __forceinline__ void bs_swap_halves(uint32_t (&w)[64]) {
  { const uint32_t t = w[62]; w[62] = w[63]; w[63] = t; }
  { const uint32_t t = w[54]; w[54] = w[55]; w[55] = t; }
  { const uint32_t t = w[46]; w[46] = w[47]; w[47] = t; }
  { const uint32_t t = w[38]; w[38] = w[39]; w[39] = t; }
  { const uint32_t t = w[30]; w[30] = w[31]; w[31] = t; }
  { const uint32_t t = w[22]; w[22] = w[23]; w[23] = t; }
  { const uint32_t t = w[14]; w[14] = w[15]; w[15] = t; }
  { const uint32_t t = w[6]; w[6] = w[7]; w[7] = t; }
  { const uint32_t t = w[60]; w[60] = w[61]; w[61] = t; }
  { const uint32_t t = w[52]; w[52] = w[53]; w[53] = t; }
  { const uint32_t t = w[44]; w[44] = w[45]; w[45] = t; }
  { const uint32_t t = w[36]; w[36] = w[37]; w[37] = t; }
  { const uint32_t t = w[28]; w[28] = w[29]; w[29] = t; }
  { const uint32_t t = w[20]; w[20] = w[21]; w[21] = t; }
  { const uint32_t t = w[12]; w[12] = w[13]; w[13] = t; }
  { const uint32_t t = w[4]; w[4] = w[5]; w[5] = t; }
  { const uint32_t t = w[58]; w[58] = w[59]; w[59] = t; }
  { const uint32_t t = w[50]; w[50] = w[51]; w[51] = t; }
  { const uint32_t t = w[42]; w[42] = w[43]; w[43] = t; }
  { const uint32_t t = w[34]; w[34] = w[35]; w[35] = t; }
  { const uint32_t t = w[26]; w[26] = w[27]; w[27] = t; }
  { const uint32_t t = w[18]; w[18] = w[19]; w[19] = t; }
  { const uint32_t t = w[10]; w[10] = w[11]; w[11] = t; }
  { const uint32_t t = w[2]; w[2] = w[3]; w[3] = t; }
  { const uint32_t t = w[56]; w[56] = w[57]; w[57] = t; }
  { const uint32_t t = w[48]; w[48] = w[49]; w[49] = t; }
  { const uint32_t t = w[40]; w[40] = w[41]; w[41] = t; }
  { const uint32_t t = w[32]; w[32] = w[33]; w[33] = t; }
  { const uint32_t t = w[24]; w[24] = w[25]; w[25] = t; }
  { const uint32_t t = w[16]; w[16] = w[17]; w[17] = t; }
  { const uint32_t t = w[8]; w[8] = w[9]; w[9] = t; }
  { const uint32_t t = w[0]; w[0] = w[1]; w[1] = t; }
}

// After 48 rounds the pre-output is R16||L16 (R = the planes that started as
// R0).  Output bit n of FP is pre-output bit FP[n]; o[slot(n)] receives it.
__host__ __device__ __forceinline__ void bs_final_perm(const uint32_t (&w)[64], uint32_t (&o)[64]) {
  o[7] = w[6];
  o[6] = w[7];
  o[5] = w[4];
  o[4] = w[5];
  o[3] = w[2];
  o[2] = w[3];
  o[1] = w[0];
  o[0] = w[1];
  o[15] = w[14];
  o[14] = w[15];
  o[13] = w[12];
  o[12] = w[13];
  o[11] = w[10];
  o[10] = w[11];
  o[9] = w[8];
  o[8] = w[9];
  o[23] = w[22];
  o[22] = w[23];
  o[21] = w[20];
  o[20] = w[21];
  o[19] = w[18];
  o[18] = w[19];
  o[17] = w[16];
  o[16] = w[17];
  o[31] = w[30];
  o[30] = w[31];
  o[29] = w[28];
  o[28] = w[29];
  o[27] = w[26];
  o[26] = w[27];
  o[25] = w[24];
  o[24] = w[25];
  o[39] = w[38];
  o[38] = w[39];
  o[37] = w[36];
  o[36] = w[37];
  o[35] = w[34];
  o[34] = w[35];
  o[33] = w[32];
  o[32] = w[33];
  o[47] = w[46];
  o[46] = w[47];
  o[45] = w[44];
  o[44] = w[45];
  o[43] = w[42];
  o[42] = w[43];
  o[41] = w[40];
  o[40] = w[41];
  o[55] = w[54];
  o[54] = w[55];
  o[53] = w[52];
  o[52] = w[53];
  o[51] = w[50];
  o[50] = w[51];
  o[49] = w[48];
  o[48] = w[49];
  o[63] = w[62];
  o[62] = w[63];
  o[61] = w[60];
  o[60] = w[61];
  o[59] = w[58];
  o[58] = w[59];
  o[57] = w[56];
  o[56] = w[57];
}

// The circuits as data (inputs are nodes 0..5 = b1..b6; node 6+i is gate i;
// an output reference is 2*node + complement).  Used by the self test.
struct BsCircuit { int ngates; unsigned char g[64][4]; int out[4]; };
static const BsCircuit kBsCircuits[8] = {
  {26, {{2, 1, 0, 0x1b}, {3, 4, 5, 0x86}, {0, 4, 3, 0xda}, {7, 1, 8, 0xd2}, {7, 5, 9, 0x76}, {1, 0, 10, 0x6d}, {9, 2, 10, 0xda}, {12, 8, 3, 0x7b}, {11, 4, 13, 0x39}, {2, 9, 14, 0xc6}, {11, 9, 3, 0x76}, {13, 7, 1, 0xe2}, {0, 17, 16, 0xc5}, {12, 4, 6, 0xdc}, {19, 2, 18, 0x6a}, {8, 9, 14, 0x27}, {0, 20, 21, 0x97}, {22, 2, 21, 0xe2}, {0, 1, 20, 0x7e}, {24, 5, 6, 0xd3}, {3, 23, 25, 0x6c}, {20, 26, 15, 0x96}, {26, 5, 15, 0x98}, {4, 28, 27, 0x6a}, {15, 10, 7, 0x7d}, {29, 30, 1, 0xb4}}, {30, 62, 52, 40}},
  {24, {{4, 3, 0, 0x69}, {5, 2, 3, 0x39}, {4, 2, 5, 0x6e}, {5, 2, 6, 0x6a}, {5, 0, 6, 0x5e}, {6, 5, 7, 0x56}, {9, 8, 0, 0x78}, {12, 0, 7, 0xe2}, {3, 10, 9, 0x65}, {11, 6, 8, 0x74}, {1, 12, 2, 0x36}, {12, 5, 0, 0xbc}, {0, 17, 7, 0xba}, {13, 3, 10, 0x2d}, {11, 4, 17, 0x2d}, {14, 4, 16, 0xe2}, {21, 20, 1, 0x72}, {4, 19, 18, 0x24}, {23, 15, 0, 0xd2}, {14, 16, 23, 0x67}, {1, 24, 25, 0xd6}, {12, 1, 19, 0xe2}, {23, 1, 5, 0x39}, {28, 6, 18, 0xc6}}, {54, 58, 52, 44}},
  {25, {{5, 1, 3, 0x96}, {3, 2, 6, 0x96}, {4, 6, 7, 0xac}, {1, 4, 7, 0x46}, {1, 2, 5, 0xd5}, {3, 9, 10, 0xc6}, {0, 8, 11, 0xac}, {8, 1, 2, 0x1a}, {4, 13, 6, 0xac}, {1, 4, 8, 0xb2}, {3, 14, 15, 0x6c}, {14, 2, 8, 0xfd}, {0, 16, 17, 0x6c}, {3, 4, 7, 0x76}, {14, 2, 16, 0x87}, {0, 19, 20, 0xc6}, {18, 4, 6, 0x76}, {4, 0, 21, 0x7e}, {2, 22, 23, 0xc6}, {1, 21, 24, 0xca}, {25, 4, 8, 0x85}, {2, 4, 6, 0x96}, {1, 26, 27, 0x2c}, {16, 11, 27, 0xde}, {0, 28, 29, 0xc2}}, {60, 36, 50, 24}},
  {19, {{3, 4, 1, 0x86}, {1, 6, 2, 0xc6}, {1, 2, 4, 0xc1}, {1, 2, 4, 0x3d}, {4, 6, 8, 0xe2}, {0, 10, 7, 0xac}, {6, 9, 3, 0xc6}, {4, 10, 12, 0x61}, {0, 12, 13, 0xac}, {5, 14, 11, 0xca}, {0, 6, 10, 0xa3}, {11, 4, 12, 0xa9}, {14, 5, 11, 0x74}, {17, 16, 1, 0x9c}, {4, 16, 14, 0x49}, {2, 10, 14, 0xe3}, {20, 21, 3, 0xd8}, {19, 22, 5, 0xb4}, {22, 23, 5, 0x69}}, {37, 30, 46, 48}},
  {26, {{0, 2, 5, 0x4a}, {1, 6, 2, 0x9c}, {0, 1, 2, 0xb9}, {3, 7, 8, 0x6c}, {5, 1, 2, 0xca}, {3, 10, 8, 0x5c}, {1, 3, 5, 0x96}, {0, 11, 12, 0x2c}, {4, 9, 13, 0xca}, {1, 2, 4, 0x86}, {12, 1, 4, 0x7c}, {3, 15, 16, 0xc6}, {9, 14, 15, 0x83}, {2, 5, 16, 0x3e}, {1, 18, 19, 0xac}, {0, 17, 20, 0xc6}, {6, 18, 21, 0x97}, {0, 2, 4, 0xb6}, {3, 22, 23, 0xac}, {13, 18, 20, 0x21}, {12, 24, 25, 0xbc}, {17, 12, 25, 0x16}, {6, 1, 13, 0x6e}, {4, 27, 28, 0xc6}, {1, 4, 6, 0xb6}, {22, 29, 30, 0xc6}}, {62, 52, 42, 28}},
  {26, {{1, 0, 3, 0x63}, {6, 1, 3, 0x82}, {3, 5, 6, 0x96}, {4, 7, 8, 0xda}, {1, 0, 9, 0xb7}, {0, 10, 4, 0x6c}, {0, 4, 8, 0xe3}, {3, 11, 12, 0xcb}, {2, 13, 9, 0x6a}, {14, 3, 10, 0xc6}, {8, 3, 14, 0x78}, {2, 13, 8, 0xa9}, {15, 17, 4, 0x87}, {9, 14, 5, 0x97}, {19, 17, 4, 0x93}, {3, 19, 2, 0x7a}, {1, 21, 8, 0x95}, {12, 3, 22, 0x5c}, {23, 1, 5, 0x1b}, {23, 2, 24, 0xe2}, {25, 4, 22, 0xb8}, {1, 20, 18, 0xac}, {26, 7, 0, 0xbe}, {22, 28, 16, 0x99}, {1, 13, 20, 0x97}, {29, 2, 30, 0xd2}}, {52, 28, 54, 62}},
  {25, {{3, 0, 4, 0x69}, {4, 1, 3, 0x39}, {2, 6, 7, 0xc6}, {7, 1, 8, 0x97}, {9, 2, 7, 0xb1}, {0, 9, 10, 0xac}, {5, 8, 11, 0xac}, {4, 0, 12, 0x47}, {11, 0, 5, 0xbd}, {3, 13, 14, 0x6c}, {2, 0, 3, 0x6d}, {14, 2, 8, 0xad}, {5, 16, 17, 0xbc}, {1, 15, 18, 0x6c}, {10, 0, 6, 0x65}, {5, 11, 20, 0xac}, {10, 3, 18, 0x69}, {8, 3, 4, 0x67}, {2, 22, 23, 0xc6}, {1, 21, 24, 0xca}, {3, 10, 21, 0xd6}, {14, 21, 25, 0x2e}, {2, 26, 27, 0xc6}, {10, 19, 25, 0x69}, {20, 28, 29, 0xc6}}, {50, 38, 60, 24}},
  {23, {{2, 0, 4, 0xf2}, {5, 6, 4, 0xb6}, {0, 5, 3, 0xd0}, {3, 4, 2, 0xa9}, {1, 3, 6, 0xc5}, {1, 0, 9, 0xd6}, {3, 8, 0, 0x6d}, {1, 11, 8, 0x2e}, {8, 12, 4, 0x32}, {14, 7, 13, 0x96}, {4, 5, 8, 0x2a}, {0, 11, 2, 0x9c}, {10, 17, 4, 0x6c}, {9, 8, 15, 0x96}, {4, 18, 10, 0xac}, {3, 20, 19, 0x6a}, {18, 5, 21, 0xb8}, {16, 6, 14, 0x36}, {12, 7, 17, 0xbf}, {23, 1, 24, 0x78}, {22, 4, 23, 0x95}, {21, 3, 26, 0x2e}, {18, 5, 27, 0x2e}}, {56, 30, 50, 44}},
};
