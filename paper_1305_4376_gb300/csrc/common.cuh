// common.cuh -- bit-level building blocks shared by the library's kernels.
//
// Everything here is __host__ __device__ so that the host self test can run
// exactly the code the GPU runs (the device versions use PTX lop3/prmt; the
// host versions emulate those two instructions bit for bit).
#pragma once

#include <cstdint>

#include "des_tables.h"

#ifndef DES3_HD
#define DES3_HD __host__ __device__ __forceinline__
#endif

namespace des3 {

// One lop3.b32: any boolean function of three words; IMM is its truth table
// indexed by 4a + 2b + c.
template <uint32_t IMM>
DES3_HD uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(IMM));
    return d;
#else
    uint32_t r = 0;
    for (int k = 0; k < 8; k++)
        if ((IMM >> k) & 1u) r |= ((k & 4) ? a : ~a) & ((k & 2) ? b : ~b) & ((k & 1) ? c : ~c);
    return r;
#endif
}

// prmt.b32 (default mode): result byte i is byte sel_i of the 8-byte value y:x.
DES3_HD uint32_t prmt(uint32_t x, uint32_t y, uint32_t sel) {
#ifdef __CUDA_ARCH__
    return __byte_perm(x, y, sel);
#else
    uint64_t v = ((uint64_t)y << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; i++) r |= (uint32_t)((v >> (8 * ((sel >> (4 * i)) & 7u))) & 0xFFu) << (8 * i);
    return r;
#endif
}

DES3_HD uint32_t bswap32(uint32_t x) { return prmt(x, 0, 0x0123); }

DES3_HD uint32_t rotr32(uint32_t x, int s) {
#ifdef __CUDA_ARCH__
    return __funnelshift_r(x, x, s);
#else
    s &= 31;
    return s ? (x >> s) | (x << (32 - s)) : x;
#endif
}

DES3_HD uint32_t rotl32(uint32_t x, int s) {
#ifdef __CUDA_ARCH__
    return __funnelshift_l(x, x, s);
#else
    s &= 31;
    return s ? (x << s) | (x >> (32 - s)) : x;
#endif
}

// Swap the bits of b selected by m with the bits of a selected by m << n.
DES3_HD void swap_move(uint32_t& a, uint32_t& b, int n, uint32_t m) {
    uint32_t t = ((a >> n) ^ b) & m;
    b ^= t;
    a ^= t << n;
}

// IP on a block held as two big-endian words (hi = DES bits 1..32, lo =
// bits 33..64).  Afterwards hi = L0 and lo = R0.  Five swap-moves; the
// sequence was derived by search against the standard's IP table and is
// re-checked by des3_self_test().
DES3_HD void initial_perm(uint32_t& hi, uint32_t& lo) {
    swap_move(hi, lo, 4, 0x0f0f0f0fu);
    swap_move(hi, lo, 16, 0x0000ffffu);
    swap_move(lo, hi, 2, 0x33333333u);
    swap_move(lo, hi, 8, 0x00ff00ffu);
    swap_move(hi, lo, 1, 0x55555555u);
}

// FP = IP^-1: the same swap-moves in reverse order.  Input hi||lo is the
// pre-output R16||L16; output hi||lo is the ciphertext block (big-endian).
DES3_HD void final_perm(uint32_t& hi, uint32_t& lo) {
    swap_move(hi, lo, 1, 0x55555555u);
    swap_move(lo, hi, 8, 0x00ff00ffu);
    swap_move(lo, hi, 2, 0x33333333u);
    swap_move(hi, lo, 16, 0x0000ffffu);
    swap_move(hi, lo, 4, 0x0f0f0f0fu);
}

// ---- bitsliced kernel: 32 x 32 bit-matrix transpose --------------------
//
// a[m] bit b  ->  a[b] bit m, in place.  Stages of 16 and 8 move whole bytes
// (prmt); stages of 4, 2 and 1 are masked bit selects (lop3).
DES3_HD uint32_t bsel(uint32_t m, uint32_t a, uint32_t b) { return lop3<0xCA>(m, a, b); }  // m ? a : b

template <int J, uint32_t M>
DES3_HD void transpose_stage(uint32_t* a) {
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & J) continue;
        uint32_t x = a[k], y = a[k + J];
        a[k + J] = bsel(M, x >> J, y);
        a[k] = bsel(M << J, y << J, x);
    }
}

DES3_HD void transpose32(uint32_t* a) {
#pragma unroll
    for (int k = 0; k < 16; k++) {
        uint32_t x = a[k], y = a[k + 16];
        a[k] = prmt(x, y, 0x5410);
        a[k + 16] = prmt(x, y, 0x7632);
    }
#pragma unroll
    for (int k = 0; k < 32; k++) {
        if (k & 8) continue;
        uint32_t x = a[k], y = a[k + 8];
        a[k] = prmt(x, y, 0x6240);
        a[k + 8] = prmt(x, y, 0x7351);
    }
    transpose_stage<4, 0x0F0F0F0Fu>(a);
    transpose_stage<2, 0x33333333u>(a);
    transpose_stage<1, 0x55555555u>(a);
}

// Key correction of a duplicated E input: x ^ c with c = 0 or ~0.  With
// DES3_BS_IMAD_CORR the same value is computed as x * s + c (s = c | 1),
// a multiply-add that issues to the FMA pipe instead of the ALU pipe.
DES3_HD uint32_t bs_correct(uint32_t x, uint32_t c, uint32_t s);

#include "bs_generated.cuh"

DES3_HD uint32_t bs_correct(uint32_t x, uint32_t c, uint32_t s) {
#if DES3_BS_IMAD_CORR
#ifdef __CUDA_ARCH__
    uint32_t d;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(s), "r"(c));
    return d;
#else
    return x * s + c;
#endif
#else
    (void)s;
    return x ^ c;
#endif
}

// ---- key masks of the bitsliced kernel -----------------------------------
//
// Every key bit is the same for all 32 blocks of a thread, so it enters the
// bitsliced rounds as a word of all ones or all zeros.  bs_mask_words()
// derives, from the 48 round keys, the DES3_BS_KEY_WORDS masks the host packs
// one bit each (layout in bs_generated.cuh; the rounds read them expanded by
// bs_mask_from_bits into DES3_BS_MASK_WORDS words): each plane is kept XORed with
// the key bit of its next use as an S-box input, so that only the 16
// duplicated E inputs need a key XOR per round.  The schedule of which half
// is the source in round r follows the three-DES pipeline of bs_tdes32().
constexpr int kBsKeyWords = DES3_BS_KEY_WORDS;    // as the host builds them, one bit each

// The expanded layouts: FOLD = false for the unfolded rounds (bs_round_A/B),
// true for the folded ones (bs_round_A_f/B_f), whose rounds carry the folds'
// multipliers after their 64 words.
template <bool FOLD>
struct BsLayout {
    static constexpr int kRound = FOLD ? DES3_BS_ROUND_WORDS_F : DES3_BS_ROUND_WORDS;
    static constexpr int kWords = 48 * kRound + 5 * 32;
    static constexpr int kPre0 = 48 * kRound, kPre16 = kPre0 + 32, kPre32 = kPre0 + 64;
    static constexpr int kPostL = kPre0 + 96, kPostR = kPre0 + 128;
};
constexpr int kBsMaskWords = BsLayout<false>::kWords;   // unfolded rounds (batched kernel)
constexpr int kBsMaskWordsF = BsLayout<true>::kWords;   // folded rounds (single-buffer kernel)
static_assert(kBsMaskWords == DES3_BS_MASK_WORDS && kBsMaskWordsF == DES3_BS_MASK_WORDS_F, "mask layouts");
constexpr int kBsMaskBitWords = (DES3_BS_KEY_WORDS + 31) / 32;  // packed

// true when round r (0..47) reads the R-planes (R0's half) as its source
constexpr bool bs_source_is_r(int r) {
    return ((r / 16) == 1) ? ((r % 16) % 2 == 1) : ((r % 16) % 2 == 0);
}

// The host's layout (DES3_BS_KEY_*), one word per mask; out holds kBsKeyWords.
inline void bs_mask_words(const uint64_t* rk, uint32_t* out, int nrounds = 48) {
    auto kb = [&](int r, int q) -> uint32_t { return (uint32_t)((rk[r] >> (47 - q)) & 1u); };
    for (int i = 0; i < kBsKeyWords; i++) out[i] = 0;
    uint32_t mu[2][33] = {};  // [0] = L-planes, [1] = R-planes: key bit each plane is stored XORed with
    for (int r = 0; r < nrounds; r++) {
        const int S = bs_source_is_r(r) ? 1 : 0, D = 1 - S;
        if (r == 0 || r == 16 || r == 32) {  // the source half is used twice in a row here
            uint32_t* pre = out + (r == 0 ? DES3_BS_KEY_PRE0 : r == 16 ? DES3_BS_KEY_PRE16 : DES3_BS_KEY_PRE32);
            for (int i = 1; i <= 32; i++) {
                const uint32_t nw = kb(r, kBsFirstPos[i]);
                pre[i - 1] = mu[S][i] ^ nw;
                mu[S][i] = nw;
            }
        }
        uint32_t* m = out + r * DES3_BS_KEY_ROUND_WORDS;
        for (int d = 0; d < 16; d++) m[d] = m[48 + d] = kb(r, kBsDup[d][1]) ^ kb(r, kBsDup[d][2]);
        int next = -1;  // next round that reads the destination half
        for (int r2 = r + 1; r2 < nrounds && next < 0; r2++)
            if ((bs_source_is_r(r2) ? 1 : 0) == D) next = r2;
        for (int i = 1; i <= 32; i++) {
            const uint32_t nw = next >= 0 ? kb(next, kBsFirstPos[i]) : 0u;
            m[16 + i - 1] = mu[D][i] ^ nw;
            mu[D][i] = nw;
        }
    }
    for (int i = 1; i <= 32; i++) {
        out[DES3_BS_KEY_POST_L + i - 1] = mu[0][i];
        out[DES3_BS_KEY_POST_R + i - 1] = mu[1][i];
    }
}

// The masks packed one bit each (what kernels receive and expand).
// nrounds: 48 for 3DES, 16 for single DES (the first DES of the pipeline).
//
// The same recurrence as bs_mask_words, on whole words: a round's 64 masks
// are two packed words (16 duplicated-input masks, then the 32 plane masks,
// then the 16 again), and the 32 planes' key bits of a round are one word.
// Expanding word by word and packing afterwards took 9 us per key and
// direction on the host, paid by every bitsliced launch and by every key of
// a batch; this form takes 0.3 us.  The library self-test checks it against
// bs_mask_words.
inline uint32_t bs_plane_key_bits(uint64_t k) {  // bit i-1 = key bit of plane i's first use
    uint32_t g = 0;
    for (int i = 1; i <= 32; i++) g |= (uint32_t)((k >> (47 - kBsFirstPos[i])) & 1u) << (i - 1);
    return g;
}
inline uint32_t bs_dup_key_bits(uint64_t k) {  // bit d = correction of duplicated input d
    uint32_t c = 0;
    for (int d = 0; d < 16; d++)
        c |= (uint32_t)(((k >> (47 - kBsDup[d][1])) ^ (k >> (47 - kBsDup[d][2]))) & 1u) << d;
    return c;
}
// Both functions above select or XOR key bits, so they are linear over
// GF(2): each is the XOR of its values on the six bytes of the round key
// taken alone.  One table per byte (plane bits low, duplicate bits high),
// built once, turns a round key into both with six lookups.
inline const uint64_t (&bs_key_bit_tables())[6][256] {
    static const struct T {
        uint64_t v[6][256];
        T() {
            for (int j = 0; j < 6; j++)
                for (int x = 0; x < 256; x++) {
                    const uint64_t k = (uint64_t)x << (8 * j);
                    v[j][x] = bs_plane_key_bits(k) | ((uint64_t)bs_dup_key_bits(k) << 32);
                }
        }
    } t;
    return t.v;
}
inline void bs_mask_bits(const uint64_t* rk, uint32_t bits[kBsMaskBitWords], int nrounds = 48) {
    static_assert(DES3_BS_KEY_ROUND_WORDS == 64 && kBsKeyWords == 48 * 64 + 5 * 32, "packed mask layout");
    static_assert(DES3_BS_KEY_PRE0 % 32 == 0 && DES3_BS_KEY_PRE16 % 32 == 0 && DES3_BS_KEY_PRE32 % 32 == 0 &&
                      DES3_BS_KEY_POST_L % 32 == 0 && DES3_BS_KEY_POST_R % 32 == 0,
                  "pre- and post-masks start whole words");
    const uint64_t(&tab)[6][256] = bs_key_bit_tables();
    uint32_t g[48], dups[48];
    for (int r = 0; r < nrounds; r++) {
        uint64_t v = 0;
        for (int j = 0; j < 6; j++) v ^= tab[j][(rk[r] >> (8 * j)) & 0xFF];
        g[r] = (uint32_t)v;
        dups[r] = (uint32_t)(v >> 32);
    }
    for (int i = 0; i < kBsMaskBitWords; i++) bits[i] = 0;
    uint32_t mu[2] = {0u, 0u};  // key bits the L- and R-planes are stored XORed with
    for (int r = 0; r < nrounds; r++) {
        const int S = bs_source_is_r(r) ? 1 : 0, D = 1 - S;
        if (r == 0 || r == 16 || r == 32) {
            bits[(r == 0 ? DES3_BS_KEY_PRE0 : r == 16 ? DES3_BS_KEY_PRE16 : DES3_BS_KEY_PRE32) / 32] = mu[S] ^ g[r];
            mu[S] = g[r];
        }
        int next = -1;
        for (int r2 = r + 1; r2 < nrounds && next < 0; r2++)
            if ((bs_source_is_r(r2) ? 1 : 0) == D) next = r2;
        const uint32_t nw = next >= 0 ? g[next] : 0u;
        const uint32_t planes = mu[D] ^ nw;
        mu[D] = nw;
        const uint32_t dup = dups[r];
        bits[2 * r] = dup | (planes << 16);
        bits[2 * r + 1] = (planes >> 16) | (dup << 16);
    }
    bits[DES3_BS_KEY_POST_L / 32] = mu[0];
    bits[DES3_BS_KEY_POST_R / 32] = mu[1];
}

// Expanded mask word w of layout BsLayout<FOLD> from the packed bits (the
// host's layout, DES3_BS_KEY_ROUND_WORDS per round).  A round's words 0..63
// are its packed bits in order, 48..63 being the corrections' multipliers
// s = c | 1; folded rounds' words 64.. are the multipliers of the folded
// outputs' deltas, from those deltas' bits.  The remasks after the rounds are
// the packed bits in order.
template <bool FOLD>
DES3_HD uint32_t bs_mask_from_bits(const uint32_t* bits, int w) {
    using L = BsLayout<FOLD>;
    int b = w;
    bool mul = false;
    if (w < 48 * L::kRound) {
        const int r = w / L::kRound, k = w % L::kRound;
        b = r * DES3_BS_KEY_ROUND_WORDS + (k < 64 ? k : bs_fold_delta(k - 64));
        mul = k >= 48;
    } else {
        b = DES3_BS_KEY_PRE0 + (w - L::kPre0);
    }
    const uint32_t m = 0u - ((bits[b >> 5] >> (b & 31)) & 1u);
    return mul ? (m | 1u) : m;
}

// All BsLayout<FOLD>::kWords expanded words, thread t of n writing every n-th of
// each round's words: the same words as bs_mask_from_bits.  A round's masks
// all come from its two packed words (the folds' deltas are among them), so
// each round loads those two once, the same for every thread, and rounds are
// unrolled to keep several loads in flight: a batched warp re-expands on
// every change of key or direction, and one dependent load per word made
// that a chain of a hundred load latencies.
template <bool FOLD>
DES3_HD void bs_expand_masks(const uint32_t* bits, uint32_t* masks, int t, int n) {
    using L = BsLayout<FOLD>;
    static_assert(DES3_BS_KEY_ROUND_WORDS == 64, "two packed words per round");
#pragma unroll 4
    for (int r = 0; r < 48; r++) {
        const uint32_t w0 = bits[2 * r], w1 = bits[2 * r + 1];
        uint32_t* m = masks + r * L::kRound;
        for (int k = t; k < L::kRound; k += n) {
            const int kk = k < 64 ? k : bs_fold_delta(k - 64);
            const uint32_t v = 0u - (((kk < 32 ? w0 : w1) >> (kk & 31)) & 1u);
            m[k] = k >= 48 ? (v | 1u) : v;
        }
    }
    for (int i = t; i < 5 * 32; i += n) {
        const int b = DES3_BS_KEY_PRE0 + i;
        masks[L::kPre0 + i] = 0u - ((bits[b >> 5] >> (b & 31)) & 1u);
    }
}

// The same words again, each thread loading the packed word of each of its
// words itself, the threads in groups of one round's words, group g taking
// rounds g, g + groups, ...  The single-buffer kernel expands once per CTA
// with this form.  Measured on one GB300 (each variant twice): against the
// round-by-round loads above its round loop was scheduled better (4 GiB
// 412.6 against 409.1 GB/s with a flat loop over all words), and against
// every thread walking all 48 rounds its prologue is short (a 1 MiB call
// 18.4 against 22.5 us, 16 MiB 303.5 against 292.4 GB/s).
template <bool FOLD>
DES3_HD void bs_expand_masks_per_word(const uint32_t* bits, uint32_t* masks, int t, int n) {
    using L = BsLayout<FOLD>;
    // threads in groups of one round's words; group g takes rounds g, g + groups, ...
    const int groups = n >= L::kRound ? n / L::kRound : 1;
    const int g = n >= L::kRound ? t / L::kRound : 0;
    const int t0 = n >= L::kRound ? t % L::kRound : t;
    const int step = n >= L::kRound ? L::kRound : n;
    for (int r = g; r < 48 && g < groups; r += groups) {
        uint32_t* m = masks + r * L::kRound;
        for (int k = t0; k < L::kRound; k += step) {
            const int b = r * DES3_BS_KEY_ROUND_WORDS + (k < 64 ? k : bs_fold_delta(k - 64));
            const uint32_t v = 0u - ((bits[b >> 5] >> (b & 31)) & 1u);
            m[k] = k >= 48 ? (v | 1u) : v;
        }
    }
    for (int i = t; i < 5 * 32; i += n) {
        const int b = DES3_BS_KEY_PRE0 + i;
        masks[L::kPre0 + i] = 0u - ((bits[b >> 5] >> (b & 31)) & 1u);
    }
}

// The whole bitsliced pipeline on 32 blocks held as w[m] = low word, w[32+m]
// = high word of block m (little-endian words of the bytes in memory order).
// NR = 48: 3DES-EDE (three DES); NR = 16: single DES (the first of them
// alone).  masks: the expanded masks of bs_mask_words for the same NR.
// Result in the same layout.
//
// One copy of the round pair (round_A, round_B) serves all three DES: before
// the second DES the L- and R-planes are exchanged, which turns its (B, A)
// round order into (A, B), and before the third they are exchanged back.
// The two switches cost 96 register moves each; the loop body a third the
// size of three unrolled DES measured 2 % faster on a single buffer and 7 %
// faster in the batched kernel, whose warps run out of step.  Within a DES
// the round-pair loop is unrolled twice (four rounds per iteration): +0.9 %
// over no unrolling, while four round pairs per iteration overflow the
// instruction cache (-4 %).
//
// bs_tdes32_planes() is the same pipeline entered with the 64 bit planes
// already formed (w[p] = plane p), for callers that can build planes more
// cheaply than by transposing.
// FOLD selects the folded rounds (and their mask layout); the single-buffer
// kernel runs them, the batched kernel the unfolded ones (with the folds its
// larger register set scheduled worse and lost 2 % on a batch of 4096 jobs).
template <int NR = 48, bool FOLD = false>
DES3_HD void bs_tdes32_planes(uint32_t (&w)[64], const uint32_t* masks) {
    static_assert(NR == 16 || NR == 48, "DES or 3DES");
    using L = BsLayout<FOLD>;
    const uint32_t* k = masks;
#pragma unroll 1
    for (int st = 0; st < NR / 16; st++) {
        if (st) bs_swap_halves(w);
        // the first source of every DES lies in the R-planes after the swaps
        bs_remask_R(w, masks + (st == 0 ? L::kPre0 : st == 1 ? L::kPre16 : L::kPre32));
#pragma unroll 2
        for (int i = 0; i < 8; i++, k += 2 * L::kRound) {
            if constexpr (FOLD) {
                bs_round_A_f(w, k);
                bs_round_B_f(w, k + L::kRound);
            } else {
                bs_round_A(w, k);
                bs_round_B(w, k + L::kRound);
            }
        }
    }
    // After two switches the planes are back in their original roles.  The
    // last round writes the R-planes, which no later round reads, so their
    // stored mask is already zero (bs_mask_words gives them the key bit of no
    // next use) and only the L-planes are unmasked.
    bs_remask_L(w, masks + L::kPostL);
    uint32_t o[64];
    bs_final_perm(w, o);
    transpose32(o);
    transpose32(o + 32);
#pragma unroll
    for (int i = 0; i < 64; i++) w[i] = o[i];
}

template <int NR = 48, bool FOLD = false>
DES3_HD void bs_tdes32(uint32_t (&w)[64], const uint32_t* masks) {
    transpose32(w);
    transpose32(w + 32);
    bs_tdes32_planes<NR, FOLD>(w, masks);
}

}  // namespace des3
