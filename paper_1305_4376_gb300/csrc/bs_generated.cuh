// Generated by gen/gen_bitslice.py from des_tables.h and gen/sbox_circuits.json.
// Do not edit by hand.  Straight-line bitsliced DES round code (see the
// generator's docstring for the plane layout and the key absorption).
#pragma once

#define DES3_BS_SBOX_GATES 235  // LOP3 gates of S1..S8 together
#define DES3_BS_S1_GATES 31
#define DES3_BS_S2_GATES 29
#define DES3_BS_S3_GATES 29
#define DES3_BS_S4_GATES 28
#define DES3_BS_S5_GATES 30
#define DES3_BS_S6_GATES 30
#define DES3_BS_S7_GATES 29
#define DES3_BS_S8_GATES 29
// ALU instructions per round for 32 blocks: 16 key corrections + gates + 32 state XORs
#define DES3_BS_OPS_PER_ROUND (16 + DES3_BS_SBOX_GATES + 32)
// mask words: 48 rounds x (16 corrections, 32 deltas), then remasks of the
// source half before rounds 0, 16 and 32 (32 words each), then the final unmask of
// L-planes and R-planes (32 words each)
#define DES3_BS_MASK_WORDS (48 * 48 + 5 * 32)
#define DES3_BS_PRE0 (48 * 48)
#define DES3_BS_PRE16 (48 * 48 + 32)
#define DES3_BS_PRE32 (48 * 48 + 64)
#define DES3_BS_POST_L (48 * 48 + 96)
#define DES3_BS_POST_R (48 * 48 + 128)

// E position (0..47) of the first use of R bit i (1..32); index 0 unused.
static constexpr int kBsFirstPos[33] = {-1, 1, 2, 3, 4, 5, 8, 9, 10, 11, 14, 15, 16, 17, 20, 21, 22, 23, 26, 27, 28, 29, 32, 33, 34, 35, 38, 39, 40, 41, 44, 45, 0};
// The 16 bits E uses twice: {bit, first position, second position}.
static constexpr int kBsDup[16][3] = {{4, 4, 6}, {5, 5, 7}, {8, 10, 12}, {9, 11, 13}, {12, 16, 18}, {13, 17, 19}, {16, 22, 24}, {17, 23, 25}, {20, 28, 30}, {21, 29, 31}, {24, 34, 36}, {25, 35, 37}, {28, 40, 42}, {29, 41, 43}, {32, 0, 46}, {1, 1, 47}};

// bs_round_A: L ^= f(R, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator).
__host__ __device__ __forceinline__ void bs_round_A(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  {  // S1
    const uint32_t n0 = w[1];
    const uint32_t n1 = w[63];
    const uint32_t n2 = w[55];
    const uint32_t n3 = w[47];
    const uint32_t n4 = w[39];
    const uint32_t n5 = w[31];
    const uint32_t n6 = lop3<0x1a>(n1, n3, n5);
    const uint32_t n7 = lop3<0x96>(n0, n1, n3);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x67>(n5, n1, n7);
    const uint32_t n10 = lop3<0xca>(n2, n8, n9);
    const uint32_t n11 = lop3<0x92>(n2, n3, n5);
    const uint32_t n12 = lop3<0xb1>(n8, n2, n5);
    const uint32_t n13 = lop3<0xac>(n1, n11, n12);
    const uint32_t n14 = lop3<0x63>(n5, n7, n13);
    const uint32_t n15 = lop3<0xca>(n0, n13, n14);
    const uint32_t n16 = lop3<0xac>(n4, n10, n15);
    const uint32_t n17 = lop3<0xc7>(n10, n1, n14);
    const uint32_t n18 = lop3<0xe3>(n5, n7, n10);
    const uint32_t n19 = lop3<0xac>(n0, n17, n18);
    const uint32_t n20 = lop3<0xe9>(n11, n2, n5);
    const uint32_t n21 = lop3<0xdb>(n9, n2, n12);
    const uint32_t n22 = lop3<0xac>(n0, n20, n21);
    const uint32_t n23 = lop3<0xc6>(n4, n19, n22);
    const uint32_t n24 = lop3<0x4e>(n7, n13, n18);
    const uint32_t n25 = lop3<0xac>(n2, n21, n24);
    const uint32_t n26 = lop3<0xb4>(n18, n2, n24);
    const uint32_t n27 = lop3<0xa6>(n6, n21, n24);
    const uint32_t n28 = lop3<0xac>(n1, n26, n27);
    const uint32_t n29 = lop3<0xca>(n4, n25, n28);
    const uint32_t n30 = lop3<0x68>(n11, n0, n4);
    const uint32_t n31 = lop3<0x69>(n29, n16, n23);
    const uint32_t n32 = lop3<0xac>(n3, n30, n31);
    const uint32_t n33 = lop3<0xd5>(n25, n16, n31);
    const uint32_t n34 = lop3<0x1d>(n30, n4, n31);
    const uint32_t n35 = lop3<0xac>(n5, n33, n34);
    const uint32_t n36 = lop3<0xac>(n1, n32, n35);
    w[60] = lop3<0x96>(w[60], n23, m[24]);
    w[58] = lop3<0x96>(w[58], n16, m[32]);
    w[10] = lop3<0x96>(w[10], n29, m[38]);
    w[8] = lop3<0x96>(w[8], n36, m[46]);
  }
  {  // S2
    const uint32_t n0 = w[39] ^ m[0];
    const uint32_t n1 = w[31] ^ m[1];
    const uint32_t n2 = w[23];
    const uint32_t n3 = w[15];
    const uint32_t n4 = w[7];
    const uint32_t n5 = w[61];
    const uint32_t n6 = lop3<0x93>(n2, n4, n5);
    const uint32_t n7 = lop3<0x16>(n5, n2, n4);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x5a>(n3, n8, n8);
    const uint32_t n10 = lop3<0x39>(n4, n7, n9);
    const uint32_t n11 = lop3<0xec>(n5, n3, n4);
    const uint32_t n12 = lop3<0xac>(n0, n10, n11);
    const uint32_t n13 = lop3<0xc6>(n1, n9, n12);
    const uint32_t n14 = lop3<0x96>(n0, n5, n6);
    const uint32_t n15 = lop3<0x35>(n4, n0, n14);
    const uint32_t n16 = lop3<0xac>(n3, n14, n15);
    const uint32_t n17 = lop3<0x4b>(n2, n3, n5);
    const uint32_t n18 = lop3<0xba>(n4, n5, n17);
    const uint32_t n19 = lop3<0xe8>(n0, n17, n18);
    const uint32_t n20 = lop3<0x6c>(n1, n16, n19);
    const uint32_t n21 = lop3<0x5c>(n0, n9, n10);
    const uint32_t n22 = lop3<0x71>(n6, n19, n21);
    const uint32_t n23 = lop3<0xac>(n2, n21, n22);
    const uint32_t n24 = lop3<0x35>(n20, n6, n22);
    const uint32_t n25 = lop3<0xd2>(n14, n3, n24);
    const uint32_t n26 = lop3<0xca>(n2, n24, n25);
    const uint32_t n27 = lop3<0xac>(n1, n23, n26);
    const uint32_t n28 = lop3<0x96>(n15, n3, n6);
    const uint32_t n29 = lop3<0xb8>(n10, n5, n6);
    const uint32_t n30 = lop3<0xac>(n1, n28, n29);
    const uint32_t n31 = lop3<0xbd>(n1, n5, n13);
    const uint32_t n32 = lop3<0x58>(n1, n3, n5);
    const uint32_t n33 = lop3<0x8c>(n4, n31, n32);
    const uint32_t n34 = lop3<0xc6>(n0, n30, n33);
    w[28] = lop3<0x96>(w[28], n13, m[28]);
    w[32] = lop3<0x96>(w[32], n20, m[43]);
    w[54] = lop3<0x96>(w[54], n27, m[17]);
    w[50] = lop3<0x96>(w[50], n34, m[33]);
  }
  {  // S3
    const uint32_t n0 = w[7] ^ m[2];
    const uint32_t n1 = w[61] ^ m[3];
    const uint32_t n2 = w[53];
    const uint32_t n3 = w[45];
    const uint32_t n4 = w[37];
    const uint32_t n5 = w[29];
    const uint32_t n6 = lop3<0x6a>(n2, n4, n5);
    const uint32_t n7 = lop3<0x99>(n6, n2, n4);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x76>(n1, n6, n8);
    const uint32_t n10 = lop3<0xbc>(n1, n8, n9);
    const uint32_t n11 = lop3<0x96>(n0, n1, n6);
    const uint32_t n12 = lop3<0x15>(n11, n5, n9);
    const uint32_t n13 = lop3<0xca>(n4, n11, n12);
    const uint32_t n14 = lop3<0xac>(n3, n10, n13);
    const uint32_t n15 = lop3<0xa9>(n11, n5, n8);
    const uint32_t n16 = lop3<0xa3>(n3, n11, n15);
    const uint32_t n17 = lop3<0xef>(n14, n4, n8);
    const uint32_t n18 = lop3<0x75>(n10, n0, n17);
    const uint32_t n19 = lop3<0xbc>(n3, n17, n18);
    const uint32_t n20 = lop3<0xc6>(n2, n16, n19);
    const uint32_t n21 = lop3<0x96>(n3, n5, n7);
    const uint32_t n22 = lop3<0x69>(n4, n15, n21);
    const uint32_t n23 = lop3<0xca>(n1, n21, n22);
    const uint32_t n24 = lop3<0x52>(n1, n13, n15);
    const uint32_t n25 = lop3<0xed>(n18, n1, n7);
    const uint32_t n26 = lop3<0xac>(n3, n24, n25);
    const uint32_t n27 = lop3<0xc6>(n0, n23, n26);
    const uint32_t n28 = lop3<0x9c>(n27, n2, n14);
    const uint32_t n29 = lop3<0xa6>(n8, n11, n21);
    const uint32_t n30 = lop3<0xac>(n4, n28, n29);
    const uint32_t n31 = lop3<0x89>(n20, n0, n21);
    const uint32_t n32 = lop3<0x96>(n2, n8, n13);
    const uint32_t n33 = lop3<0xac>(n3, n31, n32);
    const uint32_t n34 = lop3<0xac>(n1, n30, n33);
    w[2] = lop3<0x96>(w[2], n27, m[39]);
    w[4] = lop3<0x96>(w[4], n20, m[31]);
    w[16] = lop3<0x96>(w[16], n34, m[45]);
    w[22] = lop3<0x96>(w[22], n14, m[21]);
  }
  {  // S4
    const uint32_t n0 = w[37] ^ m[4];
    const uint32_t n1 = w[29] ^ m[5];
    const uint32_t n2 = w[21];
    const uint32_t n3 = w[13];
    const uint32_t n4 = w[5];
    const uint32_t n5 = w[59];
    const uint32_t n6 = lop3<0xc6>(n2, n3, n4);
    const uint32_t n7 = lop3<0xb4>(n2, n3, n4);
    const uint32_t n8 = lop3<0xac>(n1, n6, n7);
    const uint32_t n9 = lop3<0x39>(n8, n1, n3);
    const uint32_t n10 = lop3<0xe2>(n1, n3, n4);
    const uint32_t n11 = lop3<0xac>(n2, n9, n10);
    const uint32_t n12 = lop3<0xac>(n5, n8, n11);
    const uint32_t n13 = lop3<0xa7>(n4, n7, n11);
    const uint32_t n14 = lop3<0x83>(n3, n6, n9);
    const uint32_t n15 = lop3<0xac>(n5, n13, n14);
    const uint32_t n16 = lop3<0x6c>(n0, n12, n15);
    const uint32_t n17 = lop3<0x78>(n11, n0, n14);
    const uint32_t n18 = lop3<0x87>(n8, n0, n13);
    const uint32_t n19 = lop3<0xac>(n5, n17, n18);
    const uint32_t n20 = lop3<0x79>(n17, n0, n4);
    const uint32_t n21 = lop3<0x66>(n13, n0, n4);
    const uint32_t n22 = lop3<0xac>(n3, n20, n21);
    const uint32_t n23 = lop3<0x7c>(n21, n9, n22);
    const uint32_t n24 = lop3<0xac>(n5, n22, n23);
    const uint32_t n25 = lop3<0xda>(n24, n5, n8);
    const uint32_t n26 = lop3<0x56>(n18, n1, n3);
    const uint32_t n27 = lop3<0xac>(n4, n25, n26);
    const uint32_t n28 = lop3<0x6c>(n2, n24, n27);
    const uint32_t n29 = lop3<0x2e>(n22, n5, n23);
    const uint32_t n30 = lop3<0x69>(n27, n4, n29);
    const uint32_t n31 = lop3<0xac>(n2, n29, n30);
    const uint32_t n32 = lop3<0x21>(n7, n11, n18);
    const uint32_t n33 = lop3<0xc6>(n1, n31, n32);
    w[48] = lop3<0x96>(w[48], n16, m[41]);
    w[34] = lop3<0x96>(w[34], n19, m[35]);
    w[52] = lop3<0x96>(w[52], n33, m[25]);
    w[62] = lop3<0x96>(w[62], n28, m[16]);
  }
  {  // S5
    const uint32_t n0 = w[5] ^ m[6];
    const uint32_t n1 = w[59] ^ m[7];
    const uint32_t n2 = w[51];
    const uint32_t n3 = w[43];
    const uint32_t n4 = w[35];
    const uint32_t n5 = w[27];
    const uint32_t n6 = lop3<0xc5>(n4, n0, n2);
    const uint32_t n7 = lop3<0x49>(n0, n2, n4);
    const uint32_t n8 = lop3<0xac>(n3, n6, n7);
    const uint32_t n9 = lop3<0x17>(n4, n7, n8);
    const uint32_t n10 = lop3<0xca>(n5, n8, n9);
    const uint32_t n11 = lop3<0x68>(n2, n0, n5);
    const uint32_t n12 = lop3<0xd6>(n3, n11, n1);
    const uint32_t n13 = lop3<0xc6>(n1, n10, n12);
    const uint32_t n14 = lop3<0x9e>(n4, n1, n11);
    const uint32_t n15 = lop3<0x86>(n1, n2, n4);
    const uint32_t n16 = lop3<0xac>(n3, n14, n15);
    const uint32_t n17 = lop3<0x2b>(n12, n4, n5);
    const uint32_t n18 = lop3<0xac>(n1, n17, n3);
    const uint32_t n19 = lop3<0xe1>(n10, n15, n18);
    const uint32_t n20 = lop3<0xac>(n2, n18, n19);
    const uint32_t n21 = lop3<0xca>(n0, n16, n20);
    const uint32_t n22 = lop3<0xb5>(n13, n9, n12);
    const uint32_t n23 = lop3<0x76>(n6, n20, n22);
    const uint32_t n24 = lop3<0xac>(n4, n22, n23);
    const uint32_t n25 = lop3<0x58>(n2, n5, n14);
    const uint32_t n26 = lop3<0x3d>(n7, n19, n25);
    const uint32_t n27 = lop3<0xac>(n3, n25, n26);
    const uint32_t n28 = lop3<0xca>(n1, n24, n27);
    const uint32_t n29 = lop3<0xd2>(n16, n4, n5);
    const uint32_t n30 = lop3<0x86>(n7, n18, n25);
    const uint32_t n31 = lop3<0xa4>(n3, n29, n30);
    const uint32_t n32 = lop3<0x9a>(n27, n4, n12);
    const uint32_t n33 = lop3<0x68>(n24, n14, n19);
    const uint32_t n34 = lop3<0xac>(n5, n32, n33);
    const uint32_t n35 = lop3<0xac>(n0, n31, n34);
    w[6] = lop3<0x96>(w[6], n35, m[23]);
    w[20] = lop3<0x96>(w[20], n13, m[29]);
    w[56] = lop3<0x96>(w[56], n21, m[40]);
    w[46] = lop3<0x96>(w[46], n28, m[18]);
  }
  {  // S6
    const uint32_t n0 = w[35] ^ m[8];
    const uint32_t n1 = w[27] ^ m[9];
    const uint32_t n2 = w[19];
    const uint32_t n3 = w[11];
    const uint32_t n4 = w[3];
    const uint32_t n5 = w[57];
    const uint32_t n6 = lop3<0x69>(n3, n0, n4);
    const uint32_t n7 = lop3<0x8f>(n6, n0, n3);
    const uint32_t n8 = lop3<0xe2>(n3, n0, n4);
    const uint32_t n9 = lop3<0xac>(n1, n7, n8);
    const uint32_t n10 = lop3<0xac>(n5, n6, n9);
    const uint32_t n11 = lop3<0x97>(n7, n4, n5);
    const uint32_t n12 = lop3<0x94>(n4, n5, n6);
    const uint32_t n13 = lop3<0xac>(n1, n11, n12);
    const uint32_t n14 = lop3<0xca>(n2, n10, n13);
    const uint32_t n15 = lop3<0x06>(n6, n0, n1);
    const uint32_t n16 = lop3<0x8e>(n5, n9, n15);
    const uint32_t n17 = lop3<0x69>(n6, n1, n5);
    const uint32_t n18 = lop3<0xca>(n4, n16, n17);
    const uint32_t n19 = lop3<0x1e>(n18, n1, n4);
    const uint32_t n20 = lop3<0xb5>(n5, n7, n17);
    const uint32_t n21 = lop3<0xac>(n0, n19, n20);
    const uint32_t n22 = lop3<0xca>(n2, n18, n21);
    const uint32_t n23 = lop3<0x52>(n8, n9, n17);
    const uint32_t n24 = lop3<0xa3>(n2, n17, n23);
    const uint32_t n25 = lop3<0x69>(n20, n2, n13);
    const uint32_t n26 = lop3<0xa6>(n2, n18, n20);
    const uint32_t n27 = lop3<0xac>(n0, n25, n26);
    const uint32_t n28 = lop3<0xac>(n3, n24, n27);
    const uint32_t n29 = lop3<0xbd>(n27, n14, n16);
    const uint32_t n30 = lop3<0x98>(n2, n25, n26);
    const uint32_t n31 = lop3<0xbc>(n3, n29, n30);
    const uint32_t n32 = lop3<0x4d>(n20, n5, n14);
    const uint32_t n33 = lop3<0xea>(n22, n23, n32);
    const uint32_t n34 = lop3<0xca>(n0, n32, n33);
    const uint32_t n35 = lop3<0x6c>(n1, n31, n34);
    w[38] = lop3<0x96>(w[38], n14, m[19]);
    w[24] = lop3<0x96>(w[24], n28, m[44]);
    w[44] = lop3<0x96>(w[44], n22, m[26]);
    w[42] = lop3<0x96>(w[42], n35, m[34]);
  }
  {  // S7
    const uint32_t n0 = w[3] ^ m[10];
    const uint32_t n1 = w[57] ^ m[11];
    const uint32_t n2 = w[49];
    const uint32_t n3 = w[41];
    const uint32_t n4 = w[33];
    const uint32_t n5 = w[25];
    const uint32_t n6 = lop3<0x96>(n0, n3, n4);
    const uint32_t n7 = lop3<0x42>(n0, n3, n4);
    const uint32_t n8 = lop3<0xac>(n1, n6, n7);
    const uint32_t n9 = lop3<0xc5>(n5, n8, n6);
    const uint32_t n10 = lop3<0x4b>(n1, n3, n4);
    const uint32_t n11 = lop3<0xee>(n7, n0, n10);
    const uint32_t n12 = lop3<0xac>(n5, n10, n11);
    const uint32_t n13 = lop3<0xc6>(n2, n9, n12);
    const uint32_t n14 = lop3<0xc6>(n2, n7, n11);
    const uint32_t n15 = lop3<0xe1>(n6, n0, n2);
    const uint32_t n16 = lop3<0xac>(n5, n14, n15);
    const uint32_t n17 = lop3<0xd9>(n2, n3, n5);
    const uint32_t n18 = lop3<0xdb>(n8, n2, n3);
    const uint32_t n19 = lop3<0xac>(n0, n17, n18);
    const uint32_t n20 = lop3<0xc6>(n1, n16, n19);
    const uint32_t n21 = lop3<0x96>(n13, n2, n20);
    const uint32_t n22 = lop3<0x69>(n10, n16, n21);
    const uint32_t n23 = lop3<0xca>(n3, n21, n22);
    const uint32_t n24 = lop3<0xe5>(n18, n1, n2);
    const uint32_t n25 = lop3<0xe1>(n24, n4, n23);
    const uint32_t n26 = lop3<0xac>(n5, n24, n25);
    const uint32_t n27 = lop3<0x6c>(n0, n23, n26);
    const uint32_t n28 = lop3<0x64>(n5, n13, n15);
    const uint32_t n29 = lop3<0x39>(n28, n12, n18);
    const uint32_t n30 = lop3<0xac>(n3, n28, n29);
    const uint32_t n31 = lop3<0x6a>(n10, n13, n26);
    const uint32_t n32 = lop3<0x71>(n9, n22, n28);
    const uint32_t n33 = lop3<0xac>(n4, n31, n32);
    const uint32_t n34 = lop3<0xac>(n1, n30, n33);
    w[0] = lop3<0x96>(w[0], n20, m[47]);
    w[36] = lop3<0x96>(w[36], n27, m[27]);
    w[18] = lop3<0x96>(w[18], n34, m[37]);
    w[14] = lop3<0x96>(w[14], n13, m[22]);
  }
  {  // S8
    const uint32_t n0 = w[33] ^ m[12];
    const uint32_t n1 = w[25] ^ m[13];
    const uint32_t n2 = w[17];
    const uint32_t n3 = w[9];
    const uint32_t n4 = w[1] ^ m[14];
    const uint32_t n5 = w[63] ^ m[15];
    const uint32_t n6 = lop3<0x49>(n4, n1, n3);
    const uint32_t n7 = lop3<0x3e>(n2, n6, n6);
    const uint32_t n8 = lop3<0x2b>(n2, n1, n4);
    const uint32_t n9 = lop3<0x1d>(n7, n1, n4);
    const uint32_t n10 = lop3<0xac>(n3, n8, n9);
    const uint32_t n11 = lop3<0xac>(n5, n7, n10);
    const uint32_t n12 = lop3<0xeb>(n9, n2, n4);
    const uint32_t n13 = lop3<0xfe>(n7, n1, n3);
    const uint32_t n14 = lop3<0xac>(n5, n12, n13);
    const uint32_t n15 = lop3<0x6c>(n0, n11, n14);
    const uint32_t n16 = lop3<0xe1>(n7, n0, n3);
    const uint32_t n17 = lop3<0xc7>(n1, n0, n2);
    const uint32_t n18 = lop3<0x18>(n3, n17, n17);
    const uint32_t n19 = lop3<0xac>(n4, n16, n18);
    const uint32_t n20 = lop3<0x4c>(n10, n0, n4);
    const uint32_t n21 = lop3<0x61>(n14, n16, n20);
    const uint32_t n22 = lop3<0xca>(n3, n20, n21);
    const uint32_t n23 = lop3<0x6c>(n5, n19, n22);
    const uint32_t n24 = lop3<0x93>(n0, n7, n12);
    const uint32_t n25 = lop3<0x76>(n20, n3, n4);
    const uint32_t n26 = lop3<0x5c>(n1, n25, n21);
    const uint32_t n27 = lop3<0xd2>(n9, n21, n25);
    const uint32_t n28 = lop3<0xca>(n2, n26, n27);
    const uint32_t n29 = lop3<0xca>(n5, n24, n28);
    const uint32_t n30 = lop3<0x4d>(n16, n18, n25);
    const uint32_t n31 = lop3<0xa9>(n22, n9, n10);
    const uint32_t n32 = lop3<0xac>(n0, n30, n31);
    const uint32_t n33 = lop3<0xbf>(n17, n22, n30);
    const uint32_t n34 = lop3<0x6c>(n5, n32, n33);
    w[30] = lop3<0x96>(w[30], n29, m[20]);
    w[40] = lop3<0x96>(w[40], n34, m[42]);
    w[12] = lop3<0x96>(w[12], n23, m[30]);
    w[26] = lop3<0x96>(w[26], n15, m[36]);
  }
}

// bs_round_B: R ^= f(L, K).  m[0..15]: corrections of the duplicated E inputs,
// m[16 + i - 1]: mask change of destination plane i (see the generator).
__host__ __device__ __forceinline__ void bs_round_B(uint32_t (&w)[64], const uint32_t* __restrict__ m) {
  {  // S1
    const uint32_t n0 = w[0];
    const uint32_t n1 = w[62];
    const uint32_t n2 = w[54];
    const uint32_t n3 = w[46];
    const uint32_t n4 = w[38];
    const uint32_t n5 = w[30];
    const uint32_t n6 = lop3<0x1a>(n1, n3, n5);
    const uint32_t n7 = lop3<0x96>(n0, n1, n3);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x67>(n5, n1, n7);
    const uint32_t n10 = lop3<0xca>(n2, n8, n9);
    const uint32_t n11 = lop3<0x92>(n2, n3, n5);
    const uint32_t n12 = lop3<0xb1>(n8, n2, n5);
    const uint32_t n13 = lop3<0xac>(n1, n11, n12);
    const uint32_t n14 = lop3<0x63>(n5, n7, n13);
    const uint32_t n15 = lop3<0xca>(n0, n13, n14);
    const uint32_t n16 = lop3<0xac>(n4, n10, n15);
    const uint32_t n17 = lop3<0xc7>(n10, n1, n14);
    const uint32_t n18 = lop3<0xe3>(n5, n7, n10);
    const uint32_t n19 = lop3<0xac>(n0, n17, n18);
    const uint32_t n20 = lop3<0xe9>(n11, n2, n5);
    const uint32_t n21 = lop3<0xdb>(n9, n2, n12);
    const uint32_t n22 = lop3<0xac>(n0, n20, n21);
    const uint32_t n23 = lop3<0xc6>(n4, n19, n22);
    const uint32_t n24 = lop3<0x4e>(n7, n13, n18);
    const uint32_t n25 = lop3<0xac>(n2, n21, n24);
    const uint32_t n26 = lop3<0xb4>(n18, n2, n24);
    const uint32_t n27 = lop3<0xa6>(n6, n21, n24);
    const uint32_t n28 = lop3<0xac>(n1, n26, n27);
    const uint32_t n29 = lop3<0xca>(n4, n25, n28);
    const uint32_t n30 = lop3<0x68>(n11, n0, n4);
    const uint32_t n31 = lop3<0x69>(n29, n16, n23);
    const uint32_t n32 = lop3<0xac>(n3, n30, n31);
    const uint32_t n33 = lop3<0xd5>(n25, n16, n31);
    const uint32_t n34 = lop3<0x1d>(n30, n4, n31);
    const uint32_t n35 = lop3<0xac>(n5, n33, n34);
    const uint32_t n36 = lop3<0xac>(n1, n32, n35);
    w[61] = lop3<0x96>(w[61], n23, m[24]);
    w[59] = lop3<0x96>(w[59], n16, m[32]);
    w[11] = lop3<0x96>(w[11], n29, m[38]);
    w[9] = lop3<0x96>(w[9], n36, m[46]);
  }
  {  // S2
    const uint32_t n0 = w[38] ^ m[0];
    const uint32_t n1 = w[30] ^ m[1];
    const uint32_t n2 = w[22];
    const uint32_t n3 = w[14];
    const uint32_t n4 = w[6];
    const uint32_t n5 = w[60];
    const uint32_t n6 = lop3<0x93>(n2, n4, n5);
    const uint32_t n7 = lop3<0x16>(n5, n2, n4);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x5a>(n3, n8, n8);
    const uint32_t n10 = lop3<0x39>(n4, n7, n9);
    const uint32_t n11 = lop3<0xec>(n5, n3, n4);
    const uint32_t n12 = lop3<0xac>(n0, n10, n11);
    const uint32_t n13 = lop3<0xc6>(n1, n9, n12);
    const uint32_t n14 = lop3<0x96>(n0, n5, n6);
    const uint32_t n15 = lop3<0x35>(n4, n0, n14);
    const uint32_t n16 = lop3<0xac>(n3, n14, n15);
    const uint32_t n17 = lop3<0x4b>(n2, n3, n5);
    const uint32_t n18 = lop3<0xba>(n4, n5, n17);
    const uint32_t n19 = lop3<0xe8>(n0, n17, n18);
    const uint32_t n20 = lop3<0x6c>(n1, n16, n19);
    const uint32_t n21 = lop3<0x5c>(n0, n9, n10);
    const uint32_t n22 = lop3<0x71>(n6, n19, n21);
    const uint32_t n23 = lop3<0xac>(n2, n21, n22);
    const uint32_t n24 = lop3<0x35>(n20, n6, n22);
    const uint32_t n25 = lop3<0xd2>(n14, n3, n24);
    const uint32_t n26 = lop3<0xca>(n2, n24, n25);
    const uint32_t n27 = lop3<0xac>(n1, n23, n26);
    const uint32_t n28 = lop3<0x96>(n15, n3, n6);
    const uint32_t n29 = lop3<0xb8>(n10, n5, n6);
    const uint32_t n30 = lop3<0xac>(n1, n28, n29);
    const uint32_t n31 = lop3<0xbd>(n1, n5, n13);
    const uint32_t n32 = lop3<0x58>(n1, n3, n5);
    const uint32_t n33 = lop3<0x8c>(n4, n31, n32);
    const uint32_t n34 = lop3<0xc6>(n0, n30, n33);
    w[29] = lop3<0x96>(w[29], n13, m[28]);
    w[33] = lop3<0x96>(w[33], n20, m[43]);
    w[55] = lop3<0x96>(w[55], n27, m[17]);
    w[51] = lop3<0x96>(w[51], n34, m[33]);
  }
  {  // S3
    const uint32_t n0 = w[6] ^ m[2];
    const uint32_t n1 = w[60] ^ m[3];
    const uint32_t n2 = w[52];
    const uint32_t n3 = w[44];
    const uint32_t n4 = w[36];
    const uint32_t n5 = w[28];
    const uint32_t n6 = lop3<0x6a>(n2, n4, n5);
    const uint32_t n7 = lop3<0x99>(n6, n2, n4);
    const uint32_t n8 = lop3<0xac>(n0, n6, n7);
    const uint32_t n9 = lop3<0x76>(n1, n6, n8);
    const uint32_t n10 = lop3<0xbc>(n1, n8, n9);
    const uint32_t n11 = lop3<0x96>(n0, n1, n6);
    const uint32_t n12 = lop3<0x15>(n11, n5, n9);
    const uint32_t n13 = lop3<0xca>(n4, n11, n12);
    const uint32_t n14 = lop3<0xac>(n3, n10, n13);
    const uint32_t n15 = lop3<0xa9>(n11, n5, n8);
    const uint32_t n16 = lop3<0xa3>(n3, n11, n15);
    const uint32_t n17 = lop3<0xef>(n14, n4, n8);
    const uint32_t n18 = lop3<0x75>(n10, n0, n17);
    const uint32_t n19 = lop3<0xbc>(n3, n17, n18);
    const uint32_t n20 = lop3<0xc6>(n2, n16, n19);
    const uint32_t n21 = lop3<0x96>(n3, n5, n7);
    const uint32_t n22 = lop3<0x69>(n4, n15, n21);
    const uint32_t n23 = lop3<0xca>(n1, n21, n22);
    const uint32_t n24 = lop3<0x52>(n1, n13, n15);
    const uint32_t n25 = lop3<0xed>(n18, n1, n7);
    const uint32_t n26 = lop3<0xac>(n3, n24, n25);
    const uint32_t n27 = lop3<0xc6>(n0, n23, n26);
    const uint32_t n28 = lop3<0x9c>(n27, n2, n14);
    const uint32_t n29 = lop3<0xa6>(n8, n11, n21);
    const uint32_t n30 = lop3<0xac>(n4, n28, n29);
    const uint32_t n31 = lop3<0x89>(n20, n0, n21);
    const uint32_t n32 = lop3<0x96>(n2, n8, n13);
    const uint32_t n33 = lop3<0xac>(n3, n31, n32);
    const uint32_t n34 = lop3<0xac>(n1, n30, n33);
    w[3] = lop3<0x96>(w[3], n27, m[39]);
    w[5] = lop3<0x96>(w[5], n20, m[31]);
    w[17] = lop3<0x96>(w[17], n34, m[45]);
    w[23] = lop3<0x96>(w[23], n14, m[21]);
  }
  {  // S4
    const uint32_t n0 = w[36] ^ m[4];
    const uint32_t n1 = w[28] ^ m[5];
    const uint32_t n2 = w[20];
    const uint32_t n3 = w[12];
    const uint32_t n4 = w[4];
    const uint32_t n5 = w[58];
    const uint32_t n6 = lop3<0xc6>(n2, n3, n4);
    const uint32_t n7 = lop3<0xb4>(n2, n3, n4);
    const uint32_t n8 = lop3<0xac>(n1, n6, n7);
    const uint32_t n9 = lop3<0x39>(n8, n1, n3);
    const uint32_t n10 = lop3<0xe2>(n1, n3, n4);
    const uint32_t n11 = lop3<0xac>(n2, n9, n10);
    const uint32_t n12 = lop3<0xac>(n5, n8, n11);
    const uint32_t n13 = lop3<0xa7>(n4, n7, n11);
    const uint32_t n14 = lop3<0x83>(n3, n6, n9);
    const uint32_t n15 = lop3<0xac>(n5, n13, n14);
    const uint32_t n16 = lop3<0x6c>(n0, n12, n15);
    const uint32_t n17 = lop3<0x78>(n11, n0, n14);
    const uint32_t n18 = lop3<0x87>(n8, n0, n13);
    const uint32_t n19 = lop3<0xac>(n5, n17, n18);
    const uint32_t n20 = lop3<0x79>(n17, n0, n4);
    const uint32_t n21 = lop3<0x66>(n13, n0, n4);
    const uint32_t n22 = lop3<0xac>(n3, n20, n21);
    const uint32_t n23 = lop3<0x7c>(n21, n9, n22);
    const uint32_t n24 = lop3<0xac>(n5, n22, n23);
    const uint32_t n25 = lop3<0xda>(n24, n5, n8);
    const uint32_t n26 = lop3<0x56>(n18, n1, n3);
    const uint32_t n27 = lop3<0xac>(n4, n25, n26);
    const uint32_t n28 = lop3<0x6c>(n2, n24, n27);
    const uint32_t n29 = lop3<0x2e>(n22, n5, n23);
    const uint32_t n30 = lop3<0x69>(n27, n4, n29);
    const uint32_t n31 = lop3<0xac>(n2, n29, n30);
    const uint32_t n32 = lop3<0x21>(n7, n11, n18);
    const uint32_t n33 = lop3<0xc6>(n1, n31, n32);
    w[49] = lop3<0x96>(w[49], n16, m[41]);
    w[35] = lop3<0x96>(w[35], n19, m[35]);
    w[53] = lop3<0x96>(w[53], n33, m[25]);
    w[63] = lop3<0x96>(w[63], n28, m[16]);
  }
  {  // S5
    const uint32_t n0 = w[4] ^ m[6];
    const uint32_t n1 = w[58] ^ m[7];
    const uint32_t n2 = w[50];
    const uint32_t n3 = w[42];
    const uint32_t n4 = w[34];
    const uint32_t n5 = w[26];
    const uint32_t n6 = lop3<0xc5>(n4, n0, n2);
    const uint32_t n7 = lop3<0x49>(n0, n2, n4);
    const uint32_t n8 = lop3<0xac>(n3, n6, n7);
    const uint32_t n9 = lop3<0x17>(n4, n7, n8);
    const uint32_t n10 = lop3<0xca>(n5, n8, n9);
    const uint32_t n11 = lop3<0x68>(n2, n0, n5);
    const uint32_t n12 = lop3<0xd6>(n3, n11, n1);
    const uint32_t n13 = lop3<0xc6>(n1, n10, n12);
    const uint32_t n14 = lop3<0x9e>(n4, n1, n11);
    const uint32_t n15 = lop3<0x86>(n1, n2, n4);
    const uint32_t n16 = lop3<0xac>(n3, n14, n15);
    const uint32_t n17 = lop3<0x2b>(n12, n4, n5);
    const uint32_t n18 = lop3<0xac>(n1, n17, n3);
    const uint32_t n19 = lop3<0xe1>(n10, n15, n18);
    const uint32_t n20 = lop3<0xac>(n2, n18, n19);
    const uint32_t n21 = lop3<0xca>(n0, n16, n20);
    const uint32_t n22 = lop3<0xb5>(n13, n9, n12);
    const uint32_t n23 = lop3<0x76>(n6, n20, n22);
    const uint32_t n24 = lop3<0xac>(n4, n22, n23);
    const uint32_t n25 = lop3<0x58>(n2, n5, n14);
    const uint32_t n26 = lop3<0x3d>(n7, n19, n25);
    const uint32_t n27 = lop3<0xac>(n3, n25, n26);
    const uint32_t n28 = lop3<0xca>(n1, n24, n27);
    const uint32_t n29 = lop3<0xd2>(n16, n4, n5);
    const uint32_t n30 = lop3<0x86>(n7, n18, n25);
    const uint32_t n31 = lop3<0xa4>(n3, n29, n30);
    const uint32_t n32 = lop3<0x9a>(n27, n4, n12);
    const uint32_t n33 = lop3<0x68>(n24, n14, n19);
    const uint32_t n34 = lop3<0xac>(n5, n32, n33);
    const uint32_t n35 = lop3<0xac>(n0, n31, n34);
    w[7] = lop3<0x96>(w[7], n35, m[23]);
    w[21] = lop3<0x96>(w[21], n13, m[29]);
    w[57] = lop3<0x96>(w[57], n21, m[40]);
    w[47] = lop3<0x96>(w[47], n28, m[18]);
  }
  {  // S6
    const uint32_t n0 = w[34] ^ m[8];
    const uint32_t n1 = w[26] ^ m[9];
    const uint32_t n2 = w[18];
    const uint32_t n3 = w[10];
    const uint32_t n4 = w[2];
    const uint32_t n5 = w[56];
    const uint32_t n6 = lop3<0x69>(n3, n0, n4);
    const uint32_t n7 = lop3<0x8f>(n6, n0, n3);
    const uint32_t n8 = lop3<0xe2>(n3, n0, n4);
    const uint32_t n9 = lop3<0xac>(n1, n7, n8);
    const uint32_t n10 = lop3<0xac>(n5, n6, n9);
    const uint32_t n11 = lop3<0x97>(n7, n4, n5);
    const uint32_t n12 = lop3<0x94>(n4, n5, n6);
    const uint32_t n13 = lop3<0xac>(n1, n11, n12);
    const uint32_t n14 = lop3<0xca>(n2, n10, n13);
    const uint32_t n15 = lop3<0x06>(n6, n0, n1);
    const uint32_t n16 = lop3<0x8e>(n5, n9, n15);
    const uint32_t n17 = lop3<0x69>(n6, n1, n5);
    const uint32_t n18 = lop3<0xca>(n4, n16, n17);
    const uint32_t n19 = lop3<0x1e>(n18, n1, n4);
    const uint32_t n20 = lop3<0xb5>(n5, n7, n17);
    const uint32_t n21 = lop3<0xac>(n0, n19, n20);
    const uint32_t n22 = lop3<0xca>(n2, n18, n21);
    const uint32_t n23 = lop3<0x52>(n8, n9, n17);
    const uint32_t n24 = lop3<0xa3>(n2, n17, n23);
    const uint32_t n25 = lop3<0x69>(n20, n2, n13);
    const uint32_t n26 = lop3<0xa6>(n2, n18, n20);
    const uint32_t n27 = lop3<0xac>(n0, n25, n26);
    const uint32_t n28 = lop3<0xac>(n3, n24, n27);
    const uint32_t n29 = lop3<0xbd>(n27, n14, n16);
    const uint32_t n30 = lop3<0x98>(n2, n25, n26);
    const uint32_t n31 = lop3<0xbc>(n3, n29, n30);
    const uint32_t n32 = lop3<0x4d>(n20, n5, n14);
    const uint32_t n33 = lop3<0xea>(n22, n23, n32);
    const uint32_t n34 = lop3<0xca>(n0, n32, n33);
    const uint32_t n35 = lop3<0x6c>(n1, n31, n34);
    w[39] = lop3<0x96>(w[39], n14, m[19]);
    w[25] = lop3<0x96>(w[25], n28, m[44]);
    w[45] = lop3<0x96>(w[45], n22, m[26]);
    w[43] = lop3<0x96>(w[43], n35, m[34]);
  }
  {  // S7
    const uint32_t n0 = w[2] ^ m[10];
    const uint32_t n1 = w[56] ^ m[11];
    const uint32_t n2 = w[48];
    const uint32_t n3 = w[40];
    const uint32_t n4 = w[32];
    const uint32_t n5 = w[24];
    const uint32_t n6 = lop3<0x96>(n0, n3, n4);
    const uint32_t n7 = lop3<0x42>(n0, n3, n4);
    const uint32_t n8 = lop3<0xac>(n1, n6, n7);
    const uint32_t n9 = lop3<0xc5>(n5, n8, n6);
    const uint32_t n10 = lop3<0x4b>(n1, n3, n4);
    const uint32_t n11 = lop3<0xee>(n7, n0, n10);
    const uint32_t n12 = lop3<0xac>(n5, n10, n11);
    const uint32_t n13 = lop3<0xc6>(n2, n9, n12);
    const uint32_t n14 = lop3<0xc6>(n2, n7, n11);
    const uint32_t n15 = lop3<0xe1>(n6, n0, n2);
    const uint32_t n16 = lop3<0xac>(n5, n14, n15);
    const uint32_t n17 = lop3<0xd9>(n2, n3, n5);
    const uint32_t n18 = lop3<0xdb>(n8, n2, n3);
    const uint32_t n19 = lop3<0xac>(n0, n17, n18);
    const uint32_t n20 = lop3<0xc6>(n1, n16, n19);
    const uint32_t n21 = lop3<0x96>(n13, n2, n20);
    const uint32_t n22 = lop3<0x69>(n10, n16, n21);
    const uint32_t n23 = lop3<0xca>(n3, n21, n22);
    const uint32_t n24 = lop3<0xe5>(n18, n1, n2);
    const uint32_t n25 = lop3<0xe1>(n24, n4, n23);
    const uint32_t n26 = lop3<0xac>(n5, n24, n25);
    const uint32_t n27 = lop3<0x6c>(n0, n23, n26);
    const uint32_t n28 = lop3<0x64>(n5, n13, n15);
    const uint32_t n29 = lop3<0x39>(n28, n12, n18);
    const uint32_t n30 = lop3<0xac>(n3, n28, n29);
    const uint32_t n31 = lop3<0x6a>(n10, n13, n26);
    const uint32_t n32 = lop3<0x71>(n9, n22, n28);
    const uint32_t n33 = lop3<0xac>(n4, n31, n32);
    const uint32_t n34 = lop3<0xac>(n1, n30, n33);
    w[1] = lop3<0x96>(w[1], n20, m[47]);
    w[37] = lop3<0x96>(w[37], n27, m[27]);
    w[19] = lop3<0x96>(w[19], n34, m[37]);
    w[15] = lop3<0x96>(w[15], n13, m[22]);
  }
  {  // S8
    const uint32_t n0 = w[32] ^ m[12];
    const uint32_t n1 = w[24] ^ m[13];
    const uint32_t n2 = w[16];
    const uint32_t n3 = w[8];
    const uint32_t n4 = w[0] ^ m[14];
    const uint32_t n5 = w[62] ^ m[15];
    const uint32_t n6 = lop3<0x49>(n4, n1, n3);
    const uint32_t n7 = lop3<0x3e>(n2, n6, n6);
    const uint32_t n8 = lop3<0x2b>(n2, n1, n4);
    const uint32_t n9 = lop3<0x1d>(n7, n1, n4);
    const uint32_t n10 = lop3<0xac>(n3, n8, n9);
    const uint32_t n11 = lop3<0xac>(n5, n7, n10);
    const uint32_t n12 = lop3<0xeb>(n9, n2, n4);
    const uint32_t n13 = lop3<0xfe>(n7, n1, n3);
    const uint32_t n14 = lop3<0xac>(n5, n12, n13);
    const uint32_t n15 = lop3<0x6c>(n0, n11, n14);
    const uint32_t n16 = lop3<0xe1>(n7, n0, n3);
    const uint32_t n17 = lop3<0xc7>(n1, n0, n2);
    const uint32_t n18 = lop3<0x18>(n3, n17, n17);
    const uint32_t n19 = lop3<0xac>(n4, n16, n18);
    const uint32_t n20 = lop3<0x4c>(n10, n0, n4);
    const uint32_t n21 = lop3<0x61>(n14, n16, n20);
    const uint32_t n22 = lop3<0xca>(n3, n20, n21);
    const uint32_t n23 = lop3<0x6c>(n5, n19, n22);
    const uint32_t n24 = lop3<0x93>(n0, n7, n12);
    const uint32_t n25 = lop3<0x76>(n20, n3, n4);
    const uint32_t n26 = lop3<0x5c>(n1, n25, n21);
    const uint32_t n27 = lop3<0xd2>(n9, n21, n25);
    const uint32_t n28 = lop3<0xca>(n2, n26, n27);
    const uint32_t n29 = lop3<0xca>(n5, n24, n28);
    const uint32_t n30 = lop3<0x4d>(n16, n18, n25);
    const uint32_t n31 = lop3<0xa9>(n22, n9, n10);
    const uint32_t n32 = lop3<0xac>(n0, n30, n31);
    const uint32_t n33 = lop3<0xbf>(n17, n22, n30);
    const uint32_t n34 = lop3<0x6c>(n5, n32, n33);
    w[31] = lop3<0x96>(w[31], n29, m[20]);
    w[41] = lop3<0x96>(w[41], n34, m[42]);
    w[13] = lop3<0x96>(w[13], n23, m[30]);
    w[27] = lop3<0x96>(w[27], n15, m[36]);
  }
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
  {31, {{1, 3, 5, 0x1a}, {0, 1, 3, 0x96}, {0, 6, 7, 0xac}, {5, 1, 7, 0x67}, {2, 8, 9, 0xca}, {2, 3, 5, 0x92}, {8, 2, 5, 0xb1}, {1, 11, 12, 0xac}, {5, 7, 13, 0x63}, {0, 13, 14, 0xca}, {4, 10, 15, 0xac}, {10, 1, 14, 0xc7}, {5, 7, 10, 0xe3}, {0, 17, 18, 0xac}, {11, 2, 5, 0xe9}, {9, 2, 12, 0xdb}, {0, 20, 21, 0xac}, {4, 19, 22, 0xc6}, {7, 13, 18, 0x4e}, {2, 21, 24, 0xac}, {18, 2, 24, 0xb4}, {6, 21, 24, 0xa6}, {1, 26, 27, 0xac}, {4, 25, 28, 0xca}, {11, 0, 4, 0x68}, {29, 16, 23, 0x69}, {3, 30, 31, 0xac}, {25, 16, 31, 0xd5}, {30, 4, 31, 0x1d}, {5, 33, 34, 0xac}, {1, 32, 35, 0xac}}, {46, 32, 58, 72}},
  {29, {{2, 4, 5, 0x93}, {5, 2, 4, 0x16}, {0, 6, 7, 0xac}, {3, 8, 8, 0x5a}, {4, 7, 9, 0x39}, {5, 3, 4, 0xec}, {0, 10, 11, 0xac}, {1, 9, 12, 0xc6}, {0, 5, 6, 0x96}, {4, 0, 14, 0x35}, {3, 14, 15, 0xac}, {2, 3, 5, 0x4b}, {4, 5, 17, 0xba}, {0, 17, 18, 0xe8}, {1, 16, 19, 0x6c}, {0, 9, 10, 0x5c}, {6, 19, 21, 0x71}, {2, 21, 22, 0xac}, {20, 6, 22, 0x35}, {14, 3, 24, 0xd2}, {2, 24, 25, 0xca}, {1, 23, 26, 0xac}, {15, 3, 6, 0x96}, {10, 5, 6, 0xb8}, {1, 28, 29, 0xac}, {1, 5, 13, 0xbd}, {1, 3, 5, 0x58}, {4, 31, 32, 0x8c}, {0, 30, 33, 0xc6}}, {26, 40, 54, 68}},
  {29, {{2, 4, 5, 0x6a}, {6, 2, 4, 0x99}, {0, 6, 7, 0xac}, {1, 6, 8, 0x76}, {1, 8, 9, 0xbc}, {0, 1, 6, 0x96}, {11, 5, 9, 0x15}, {4, 11, 12, 0xca}, {3, 10, 13, 0xac}, {11, 5, 8, 0xa9}, {3, 11, 15, 0xa3}, {14, 4, 8, 0xef}, {10, 0, 17, 0x75}, {3, 17, 18, 0xbc}, {2, 16, 19, 0xc6}, {3, 5, 7, 0x96}, {4, 15, 21, 0x69}, {1, 21, 22, 0xca}, {1, 13, 15, 0x52}, {18, 1, 7, 0xed}, {3, 24, 25, 0xac}, {0, 23, 26, 0xc6}, {27, 2, 14, 0x9c}, {8, 11, 21, 0xa6}, {4, 28, 29, 0xac}, {20, 0, 21, 0x89}, {2, 8, 13, 0x96}, {3, 31, 32, 0xac}, {1, 30, 33, 0xac}}, {54, 40, 68, 28}},
  {28, {{2, 3, 4, 0xc6}, {2, 3, 4, 0xb4}, {1, 6, 7, 0xac}, {8, 1, 3, 0x39}, {1, 3, 4, 0xe2}, {2, 9, 10, 0xac}, {5, 8, 11, 0xac}, {4, 7, 11, 0xa7}, {3, 6, 9, 0x83}, {5, 13, 14, 0xac}, {0, 12, 15, 0x6c}, {11, 0, 14, 0x78}, {8, 0, 13, 0x87}, {5, 17, 18, 0xac}, {17, 0, 4, 0x79}, {13, 0, 4, 0x66}, {3, 20, 21, 0xac}, {21, 9, 22, 0x7c}, {5, 22, 23, 0xac}, {24, 5, 8, 0xda}, {18, 1, 3, 0x56}, {4, 25, 26, 0xac}, {2, 24, 27, 0x6c}, {22, 5, 23, 0x2e}, {27, 4, 29, 0x69}, {2, 29, 30, 0xac}, {7, 11, 18, 0x21}, {1, 31, 32, 0xc6}}, {32, 38, 66, 56}},
  {30, {{4, 0, 2, 0xc5}, {0, 2, 4, 0x49}, {3, 6, 7, 0xac}, {4, 7, 8, 0x17}, {5, 8, 9, 0xca}, {2, 0, 5, 0x68}, {3, 11, 1, 0xd6}, {1, 10, 12, 0xc6}, {4, 1, 11, 0x9e}, {1, 2, 4, 0x86}, {3, 14, 15, 0xac}, {12, 4, 5, 0x2b}, {1, 17, 3, 0xac}, {10, 15, 18, 0xe1}, {2, 18, 19, 0xac}, {0, 16, 20, 0xca}, {13, 9, 12, 0xb5}, {6, 20, 22, 0x76}, {4, 22, 23, 0xac}, {2, 5, 14, 0x58}, {7, 19, 25, 0x3d}, {3, 25, 26, 0xac}, {1, 24, 27, 0xca}, {16, 4, 5, 0xd2}, {7, 18, 25, 0x86}, {3, 29, 30, 0xa4}, {27, 4, 12, 0x9a}, {24, 14, 19, 0x68}, {5, 32, 33, 0xac}, {0, 31, 34, 0xac}}, {70, 26, 42, 56}},
  {30, {{3, 0, 4, 0x69}, {6, 0, 3, 0x8f}, {3, 0, 4, 0xe2}, {1, 7, 8, 0xac}, {5, 6, 9, 0xac}, {7, 4, 5, 0x97}, {4, 5, 6, 0x94}, {1, 11, 12, 0xac}, {2, 10, 13, 0xca}, {6, 0, 1, 0x06}, {5, 9, 15, 0x8e}, {6, 1, 5, 0x69}, {4, 16, 17, 0xca}, {18, 1, 4, 0x1e}, {5, 7, 17, 0xb5}, {0, 19, 20, 0xac}, {2, 18, 21, 0xca}, {8, 9, 17, 0x52}, {2, 17, 23, 0xa3}, {20, 2, 13, 0x69}, {2, 18, 20, 0xa6}, {0, 25, 26, 0xac}, {3, 24, 27, 0xac}, {27, 14, 16, 0xbd}, {2, 25, 26, 0x98}, {3, 29, 30, 0xbc}, {20, 5, 14, 0x4d}, {22, 23, 32, 0xea}, {0, 32, 33, 0xca}, {1, 31, 34, 0x6c}}, {28, 56, 44, 70}},
  {29, {{0, 3, 4, 0x96}, {0, 3, 4, 0x42}, {1, 6, 7, 0xac}, {5, 8, 6, 0xc5}, {1, 3, 4, 0x4b}, {7, 0, 10, 0xee}, {5, 10, 11, 0xac}, {2, 9, 12, 0xc6}, {2, 7, 11, 0xc6}, {6, 0, 2, 0xe1}, {5, 14, 15, 0xac}, {2, 3, 5, 0xd9}, {8, 2, 3, 0xdb}, {0, 17, 18, 0xac}, {1, 16, 19, 0xc6}, {13, 2, 20, 0x96}, {10, 16, 21, 0x69}, {3, 21, 22, 0xca}, {18, 1, 2, 0xe5}, {24, 4, 23, 0xe1}, {5, 24, 25, 0xac}, {0, 23, 26, 0x6c}, {5, 13, 15, 0x64}, {28, 12, 18, 0x39}, {3, 28, 29, 0xac}, {10, 13, 26, 0x6a}, {9, 22, 28, 0x71}, {4, 31, 32, 0xac}, {1, 30, 33, 0xac}}, {40, 54, 68, 26}},
  {29, {{4, 1, 3, 0x49}, {2, 6, 6, 0x3e}, {2, 1, 4, 0x2b}, {7, 1, 4, 0x1d}, {3, 8, 9, 0xac}, {5, 7, 10, 0xac}, {9, 2, 4, 0xeb}, {7, 1, 3, 0xfe}, {5, 12, 13, 0xac}, {0, 11, 14, 0x6c}, {7, 0, 3, 0xe1}, {1, 0, 2, 0xc7}, {3, 17, 17, 0x18}, {4, 16, 18, 0xac}, {10, 0, 4, 0x4c}, {14, 16, 20, 0x61}, {3, 20, 21, 0xca}, {5, 19, 22, 0x6c}, {0, 7, 12, 0x93}, {20, 3, 4, 0x76}, {1, 25, 21, 0x5c}, {9, 21, 25, 0xd2}, {2, 26, 27, 0xca}, {5, 24, 28, 0xca}, {16, 18, 25, 0x4d}, {22, 9, 10, 0xa9}, {0, 30, 31, 0xac}, {17, 22, 30, 0xbf}, {5, 32, 33, 0x6c}}, {58, 68, 46, 30}},
};
