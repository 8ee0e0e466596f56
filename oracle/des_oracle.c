/*
 * Plain CPU oracle for DES and 3DES-EDE in ECB mode.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU library must compute.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may build, load or call
 * it.  It shares no code, table or header with the CUDA library.
 *
 * What it follows:
 *   - The paper (3DES ECB on CUDA, Sec. II.A) defines 3DES encryption as
 *     "encrypt with the first key, decrypt with the second, encrypt with the
 *     third", and decryption as the same steps in reverse.
 *   - The block cipher itself is the DES standard the paper relies on without
 *     printing it (FIPS PUB 46-3): initial permutation IP, sixteen Feistel
 *     rounds R_i = L_{i-1} xor P(S(E(R_{i-1}) xor K_i)), L_i = R_{i-1}, and
 *     the final permutation IP^-1 applied to R16 || L16.  The key schedule is
 *     PC-1, sixteen left rotations of the 28-bit halves C and D, then PC-2.
 *   - ECB mode (paper, abstract and Fig. 2): every 64-bit block is processed
 *     on its own, with no chaining and no padding.
 *
 * Conventions (the paper is silent on them; these are the readings taken):
 *   - Bits are numbered 1..64 from the most significant bit of byte 0 of a
 *     block, as in the standard; a block is eight bytes in memory order.
 *   - A key is eight bytes; the low bit of each byte is a parity bit that
 *     PC-1 never selects, so parity is ignored.
 *   - A 3DES key is 24 bytes K1 || K2 || K3.  Two-key 3DES is K1 || K2 || K1.
 *
 * Every permutation is evaluated bit by bit from its table; every S-box is a
 * direct row/column lookup.  There is no combined table, no bit slicing and
 * no word-level trick anywhere in this file.
 */
#include <stddef.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- FIPS 46-3 tables (1-based bit positions) ------------------------- */

/* Initial permutation IP: output bit i is input bit IP_TAB[i-1]. */
static const int IP_TAB[64] = {
    58, 50, 42, 34, 26, 18, 10, 2,  60, 52, 44, 36, 28, 20, 12, 4,
    62, 54, 46, 38, 30, 22, 14, 6,  64, 56, 48, 40, 32, 24, 16, 8,
    57, 49, 41, 33, 25, 17, 9,  1,  59, 51, 43, 35, 27, 19, 11, 3,
    61, 53, 45, 37, 29, 21, 13, 5,  63, 55, 47, 39, 31, 23, 15, 7};

/* Final permutation IP^-1. */
static const int FP_TAB[64] = {
    40, 8, 48, 16, 56, 24, 64, 32, 39, 7, 47, 15, 55, 23, 63, 31,
    38, 6, 46, 14, 54, 22, 62, 30, 37, 5, 45, 13, 53, 21, 61, 29,
    36, 4, 44, 12, 52, 20, 60, 28, 35, 3, 43, 11, 51, 19, 59, 27,
    34, 2, 42, 10, 50, 18, 58, 26, 33, 1, 41, 9,  49, 17, 57, 25};

/* Expansion E: 32 -> 48 bits. */
static const int E_TAB[48] = {
    32, 1,  2,  3,  4,  5,  4,  5,  6,  7,  8,  9,  8,  9,  10, 11,
    12, 13, 12, 13, 14, 15, 16, 17, 16, 17, 18, 19, 20, 21, 20, 21,
    22, 23, 24, 25, 24, 25, 26, 27, 28, 29, 28, 29, 30, 31, 32, 1};

/* Permutation P applied to the 32 S-box output bits. */
static const int P_TAB[32] = {
    16, 7, 20, 21, 29, 12, 28, 17, 1,  15, 23, 26, 5,  18, 31, 10,
    2,  8, 24, 14, 32, 27, 3,  9,  19, 13, 30, 6,  22, 11, 4,  25};

/* Permuted choice 1: 64 -> 56 key bits (C0 = first 28, D0 = last 28). */
static const int PC1_TAB[56] = {
    57, 49, 41, 33, 25, 17, 9,  1,  58, 50, 42, 34, 26, 18,
    10, 2,  59, 51, 43, 35, 27, 19, 11, 3,  60, 52, 44, 36,
    63, 55, 47, 39, 31, 23, 15, 7,  62, 54, 46, 38, 30, 22,
    14, 6,  61, 53, 45, 37, 29, 21, 13, 5,  28, 20, 12, 4};

/* Permuted choice 2: 56 -> 48 bits of round key K_i. */
static const int PC2_TAB[48] = {
    14, 17, 11, 24, 1,  5,  3,  28, 15, 6,  21, 10,
    23, 19, 12, 4,  26, 8,  16, 7,  27, 20, 13, 2,
    41, 52, 31, 37, 47, 55, 30, 40, 51, 45, 33, 48,
    44, 49, 39, 56, 34, 53, 46, 42, 50, 36, 29, 32};

/* Left-rotation amounts of C and D before rounds 1..16. */
static const int SHIFT_TAB[16] = {1, 1, 2, 2, 2, 2, 2, 2, 1, 2, 2, 2, 2, 2, 2, 1};

/* S-boxes S1..S8, each 4 rows x 16 columns. */
static const int SBOX_TAB[8][4][16] = {
    {{14, 4, 13, 1, 2, 15, 11, 8, 3, 10, 6, 12, 5, 9, 0, 7},
     {0, 15, 7, 4, 14, 2, 13, 1, 10, 6, 12, 11, 9, 5, 3, 8},
     {4, 1, 14, 8, 13, 6, 2, 11, 15, 12, 9, 7, 3, 10, 5, 0},
     {15, 12, 8, 2, 4, 9, 1, 7, 5, 11, 3, 14, 10, 0, 6, 13}},
    {{15, 1, 8, 14, 6, 11, 3, 4, 9, 7, 2, 13, 12, 0, 5, 10},
     {3, 13, 4, 7, 15, 2, 8, 14, 12, 0, 1, 10, 6, 9, 11, 5},
     {0, 14, 7, 11, 10, 4, 13, 1, 5, 8, 12, 6, 9, 3, 2, 15},
     {13, 8, 10, 1, 3, 15, 4, 2, 11, 6, 7, 12, 0, 5, 14, 9}},
    {{10, 0, 9, 14, 6, 3, 15, 5, 1, 13, 12, 7, 11, 4, 2, 8},
     {13, 7, 0, 9, 3, 4, 6, 10, 2, 8, 5, 14, 12, 11, 15, 1},
     {13, 6, 4, 9, 8, 15, 3, 0, 11, 1, 2, 12, 5, 10, 14, 7},
     {1, 10, 13, 0, 6, 9, 8, 7, 4, 15, 14, 3, 11, 5, 2, 12}},
    {{7, 13, 14, 3, 0, 6, 9, 10, 1, 2, 8, 5, 11, 12, 4, 15},
     {13, 8, 11, 5, 6, 15, 0, 3, 4, 7, 2, 12, 1, 10, 14, 9},
     {10, 6, 9, 0, 12, 11, 7, 13, 15, 1, 3, 14, 5, 2, 8, 4},
     {3, 15, 0, 6, 10, 1, 13, 8, 9, 4, 5, 11, 12, 7, 2, 14}},
    {{2, 12, 4, 1, 7, 10, 11, 6, 8, 5, 3, 15, 13, 0, 14, 9},
     {14, 11, 2, 12, 4, 7, 13, 1, 5, 0, 15, 10, 3, 9, 8, 6},
     {4, 2, 1, 11, 10, 13, 7, 8, 15, 9, 12, 5, 6, 3, 0, 14},
     {11, 8, 12, 7, 1, 14, 2, 13, 6, 15, 0, 9, 10, 4, 5, 3}},
    {{12, 1, 10, 15, 9, 2, 6, 8, 0, 13, 3, 4, 14, 7, 5, 11},
     {10, 15, 4, 2, 7, 12, 9, 5, 6, 1, 13, 14, 0, 11, 3, 8},
     {9, 14, 15, 5, 2, 8, 12, 3, 7, 0, 4, 10, 1, 13, 11, 6},
     {4, 3, 2, 12, 9, 5, 15, 10, 11, 14, 1, 7, 6, 0, 8, 13}},
    {{4, 11, 2, 14, 15, 0, 8, 13, 3, 12, 9, 7, 5, 10, 6, 1},
     {13, 0, 11, 7, 4, 9, 1, 10, 14, 3, 5, 12, 2, 15, 8, 6},
     {1, 4, 11, 13, 12, 3, 7, 14, 10, 15, 6, 8, 0, 5, 9, 2},
     {6, 11, 13, 8, 1, 4, 10, 7, 9, 5, 0, 15, 14, 2, 3, 12}},
    {{13, 2, 8, 4, 6, 15, 11, 1, 10, 9, 3, 14, 5, 0, 12, 7},
     {1, 15, 13, 8, 10, 3, 7, 4, 12, 5, 6, 11, 0, 14, 9, 2},
     {7, 11, 4, 1, 9, 12, 14, 2, 0, 6, 10, 13, 15, 3, 5, 8},
     {2, 1, 14, 7, 4, 10, 8, 13, 15, 12, 9, 0, 3, 5, 6, 11}}};

/* ---- bit-level helpers ------------------------------------------------ */

/* Bit n (1-based, 1 = most significant) of a value `width` bits wide. */
static unsigned bit_of(uint64_t x, int width, int n) {
    return (unsigned)((x >> (width - n)) & 1u);
}

/* Generic table permutation: output bit i (1-based, MSB first) of an
 * `out_width`-bit result is input bit table[i-1] of the `in_width`-bit input. */
static uint64_t permute(uint64_t in, int in_width, const int* table, int out_width) {
    uint64_t out = 0;
    for (int i = 0; i < out_width; i++) out = (out << 1) | bit_of(in, in_width, table[i]);
    return out;
}

static uint64_t load_be64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v = (v << 8) | p[i];
    return v;
}

static void store_be64(uint8_t* p, uint64_t v) {
    for (int i = 7; i >= 0; i--) {
        p[i] = (uint8_t)(v & 0xFF);
        v >>= 8;
    }
}

static uint32_t rotl28(uint32_t v, int s) {
    return ((v << s) | (v >> (28 - s))) & 0x0FFFFFFFu;
}

/* ---- DES (FIPS 46-3) -------------------------------------------------- */

/* Key schedule: 16 round keys K_1..K_16, each a 48-bit value (bit 1 = MSB). */
void oracle_des_key_schedule(const uint8_t key[8], uint64_t subkeys[16]) {
    uint64_t k = load_be64(key);
    uint64_t cd = permute(k, 64, PC1_TAB, 56);
    uint32_t c = (uint32_t)(cd >> 28) & 0x0FFFFFFFu;
    uint32_t d = (uint32_t)cd & 0x0FFFFFFFu;
    for (int i = 0; i < 16; i++) {
        c = rotl28(c, SHIFT_TAB[i]);
        d = rotl28(d, SHIFT_TAB[i]);
        subkeys[i] = permute(((uint64_t)c << 28) | d, 56, PC2_TAB, 48);
    }
}

/* The cipher function f(R, K) = P(S(E(R) xor K)). */
static uint32_t cipher_f(uint32_t r, uint64_t k) {
    uint64_t x = permute(r, 32, E_TAB, 48) ^ k;
    uint64_t s = 0;
    for (int j = 0; j < 8; j++) {
        unsigned six = (unsigned)(x >> (42 - 6 * j)) & 63u; /* bits b1..b6 of group j */
        unsigned row = ((six >> 5) & 1u) * 2u + (six & 1u); /* b1 b6 */
        unsigned col = (six >> 1) & 15u;                    /* b2 b3 b4 b5 */
        s = (s << 4) | (uint64_t)SBOX_TAB[j][row][col];
    }
    return (uint32_t)permute(s, 32, P_TAB, 32);
}

/* One DES block with a prepared schedule; decrypt uses K_16..K_1. */
uint64_t oracle_des_block(const uint64_t subkeys[16], uint64_t block, int decrypt) {
    uint64_t t = permute(block, 64, IP_TAB, 64);
    uint32_t l = (uint32_t)(t >> 32), r = (uint32_t)t;
    for (int i = 0; i < 16; i++) {
        uint64_t k = subkeys[decrypt ? 15 - i : i];
        uint32_t next_r = l ^ cipher_f(r, k);
        l = r;
        r = next_r;
    }
    return permute(((uint64_t)r << 32) | l, 64, FP_TAB, 64);
}

/* ---- 3DES-EDE (paper Sec. II.A) --------------------------------------- */

/* Encrypt: E_K3(D_K2(E_K1(x))).  Decrypt, the same steps in reverse:
 * D_K1(E_K2(D_K3(x))). */
static uint64_t tdes_block(const uint64_t ks[3][16], uint64_t x, int decrypt) {
    if (!decrypt) {
        x = oracle_des_block(ks[0], x, 0);
        x = oracle_des_block(ks[1], x, 1);
        x = oracle_des_block(ks[2], x, 0);
    } else {
        x = oracle_des_block(ks[2], x, 1);
        x = oracle_des_block(ks[1], x, 0);
        x = oracle_des_block(ks[0], x, 1);
    }
    return x;
}

/* ECB over `nbytes` (a multiple of 8) with a 24-byte key K1||K2||K3.
 * in and out may be the same buffer.  nthreads <= 0 uses the OpenMP
 * default.  Returns 0, or -1 when nbytes is not a multiple of 8. */
int oracle_tdes_ecb(const uint8_t key24[24], const uint8_t* in, uint8_t* out,
                    uint64_t nbytes, int decrypt, int nthreads) {
    if (nbytes % 8 != 0) return -1;
    uint64_t ks[3][16];
    for (int k = 0; k < 3; k++) oracle_des_key_schedule(key24 + 8 * k, ks[k]);
    int64_t nblocks = (int64_t)(nbytes / 8);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t b = 0; b < nblocks; b++) {
        uint64_t x = load_be64(in + 8 * b);
        store_be64(out + 8 * b, tdes_block((const uint64_t(*)[16])ks, x, decrypt));
    }
    (void)nthreads;
    return 0;
}

/* ---- CBC and CTR modes (NIST SP 800-38A), built on the same block function.
 * They are not in the paper, which uses ECB only; they are the library's
 * extension to the two other modes whose work is parallel over blocks. ---- */

/* CBC: C_i = E(P_i xor C_{i-1}), C_0 = IV; decryption P_i = D(C_i) xor C_{i-1}.
 * in and out may be the same buffer. */
int oracle_tdes_cbc(const uint8_t key24[24], const uint8_t iv[8], const uint8_t* in, uint8_t* out,
                    uint64_t nbytes, int decrypt) {
    if (nbytes % 8 != 0) return -1;
    uint64_t ks[3][16];
    for (int k = 0; k < 3; k++) oracle_des_key_schedule(key24 + 8 * k, ks[k]);
    uint64_t prev = load_be64(iv);
    for (uint64_t b = 0; b < nbytes / 8; b++) {
        const uint64_t x = load_be64(in + 8 * b);
        if (!decrypt) {
            prev = tdes_block((const uint64_t(*)[16])ks, x ^ prev, 0);
            store_be64(out + 8 * b, prev);
        } else {
            store_be64(out + 8 * b, tdes_block((const uint64_t(*)[16])ks, x, 1) ^ prev);
            prev = x;
        }
    }
    return 0;
}

/* CTR: the i-th counter block is T_0 + i modulo 2^64, the whole 64-bit block
 * read as a big-endian integer (the standard incrementing function);
 * out_i = in_i xor E(T_i).  The same call decrypts.  OpenMP over blocks. */
int oracle_tdes_ctr(const uint8_t key24[24], const uint8_t ctr0[8], const uint8_t* in, uint8_t* out,
                    uint64_t nbytes, int nthreads) {
    if (nbytes % 8 != 0) return -1;
    uint64_t ks[3][16];
    for (int k = 0; k < 3; k++) oracle_des_key_schedule(key24 + 8 * k, ks[k]);
    const uint64_t t0 = load_be64(ctr0);
    int64_t nblocks = (int64_t)(nbytes / 8);
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nthreads)
#endif
    for (int64_t b = 0; b < nblocks; b++) {
        const uint64_t o = tdes_block((const uint64_t(*)[16])ks, t0 + (uint64_t)b, 0);
        store_be64(out + 8 * b, load_be64(in + 8 * b) ^ o);
    }
    (void)nthreads;
    return 0;
}

/* Single DES in ECB with an 8-byte key (used by the pins only). */
int oracle_des_ecb(const uint8_t key8[8], const uint8_t* in, uint8_t* out,
                   uint64_t nbytes, int decrypt) {
    if (nbytes % 8 != 0) return -1;
    uint64_t ks[16];
    oracle_des_key_schedule(key8, ks);
    for (uint64_t b = 0; b < nbytes / 8; b++)
        store_be64(out + 8 * b, oracle_des_block(ks, load_be64(in + 8 * b), decrypt));
    return 0;
}

/* Number of threads an OpenMP region would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Read-only access to the tables, for the structural pins.  Returns the
 * number of entries (0 for an unknown name) and stores a pointer. */
int oracle_table(const char* name, const int** out) {
    struct { const char* n; const int* t; int len; } tabs[] = {
        {"IP", IP_TAB, 64},   {"FP", FP_TAB, 64},   {"E", E_TAB, 48},
        {"P", P_TAB, 32},     {"PC1", PC1_TAB, 56}, {"PC2", PC2_TAB, 48},
        {"SHIFT", SHIFT_TAB, 16}, {"SBOX", &SBOX_TAB[0][0][0], 512},
    };
    for (size_t i = 0; i < sizeof(tabs) / sizeof(tabs[0]); i++)
        if (strcmp(tabs[i].n, name) == 0) {
            *out = tabs[i].t;
            return tabs[i].len;
        }
    *out = NULL;
    return 0;
}
