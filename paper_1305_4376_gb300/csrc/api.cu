// api.cu -- the C ABI (include/des3.h): argument checking, the host key
// schedule, kernel choice, error reporting and the host self test.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "sptable.cuh"
#include "tuning.h"

namespace des3 {

namespace {
thread_local int t_last_cuda_error = 0;

std::mutex g_dev_mu;
DeviceInfo g_dev[64];
bool g_dev_valid[64];
}  // namespace

int cuda_fail(cudaError_t e) {
    t_last_cuda_error = (int)e;
    return DES3_ECUDA;
}

int launch_single(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks, int kernel,
                  cudaStream_t s, int nrounds) {
    const LaunchShape sh = tuned_single(nblocks * 8, kernel);
    return sh.kernel == DES3_KERNEL_SPTABLE
               ? launch_sptable(rk, in, out, nblocks, s, sh.threads, sh.ctas_per_sm, nrounds)
               : launch_bitslice(rk, in, out, nblocks, s, sh.threads, sh.ctas_per_sm, nrounds);
}

void rk48(const des3_ks_t* ks, int dir, uint64_t out[48]) {
    if (!(ks->flags & DES3_KS_SINGLE_DES)) {
        for (int r = 0; r < 48; r++) out[r] = ks->rk[dir][r];
        return;
    }
    uint64_t enc[48];
    for (int r = 0; r < 16; r++) {
        enc[r] = ks->rk[0][r];            // E_K
        enc[16 + r] = ks->rk[0][15 - r];  // D_K
        enc[32 + r] = ks->rk[0][r];       // E_K
    }
    for (int r = 0; r < 48; r++) out[r] = dir ? enc[47 - r] : enc[r];
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DES3_OK : cuda_fail(e);
}

int current_device_info(DeviceInfo* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e == cudaErrorNoDevice ? (t_last_cuda_error = (int)e, DES3_ENODEV) : cuda_fail(e);
    if (dev < 0 || dev >= 64) return DES3_ENODEV;
    std::lock_guard<std::mutex> g(g_dev_mu);
    if (!g_dev_valid[dev]) {
        DeviceInfo d;
        d.device = dev;
        int major = 0, minor = 0;
        if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev)) != cudaSuccess) return cuda_fail(e);
        if ((e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev)) != cudaSuccess) return cuda_fail(e);
        if (major != 10 || minor != 3) return DES3_ENODEV;  // the binary holds sm_103a code only
        g_dev[dev] = d;
        g_dev_valid[dev] = true;
    }
    *out = g_dev[dev];
    return DES3_OK;
}

// ---- host key schedule (FIPS 46-3: PC-1, rotations, PC-2) ---------------

static uint64_t load_be64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; i++) v = (v << 8) | p[i];
    return v;
}

static void des_subkeys(const uint8_t key[8], uint64_t sub[16]) {
    const uint64_t k = load_be64(key);
    uint64_t cd = 0;
    for (int i = 0; i < 56; i++) cd = (cd << 1) | ((k >> (64 - fips::kPC1[i])) & 1u);
    uint32_t c = (uint32_t)(cd >> 28), d = (uint32_t)(cd & 0x0FFFFFFFu);
    for (int r = 0; r < 16; r++) {
        const int s = fips::kShift[r];
        c = ((c << s) | (c >> (28 - s))) & 0x0FFFFFFFu;
        d = ((d << s) | (d >> (28 - s))) & 0x0FFFFFFFu;
        const uint64_t x = ((uint64_t)c << 28) | d;
        uint64_t kr = 0;
        for (int i = 0; i < 48; i++) kr = (kr << 1) | ((x >> (56 - fips::kPC2[i])) & 1u);
        sub[r] = kr;
    }
}

static bool overlaps_partially(const void* a, const void* b, size_t n) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    if (x == y) return false;
    return x < y + n && y < x + n;
}

// ---- host self test -------------------------------------------------------

// The rotated table kernel's lookup on the host: with a lane base of 0 the
// address is x * 1024 for entry x; any other bit set means the address
// arithmetic is wrong, which the self test then reports.
struct HostRotLookup {
    const SpTable* t;
    template <int J>
    DES3_HD uint32_t at(uint32_t addr) const {
        return (addr & ~(63u << 10)) ? 0xDEADBEEFu : t->v[J][addr >> 10];
    }
};

// (ke, ko) pairs of n round keys, two rounds per uint4.
static void rot_keys(const uint64_t* rk, int n, uint4* k4) {
    for (int r = 0; r < n; r += 2) {
        uint32_t a, b, c, d;
        sp_rot_key(rk[r], &a, &b);
        sp_rot_key(rk[r + 1], &c, &d);
        k4[r / 2] = make_uint4(a, b, c, d);
    }
}

// The packed masks (word-parallel, table-driven) against the masks expanded
// one word each by the plain recurrence.
static bool packed_masks_match(const uint64_t* rk, const uint32_t* bits, int nrounds) {
    static uint32_t words[kBsKeyWords];
    bs_mask_words(rk, words, nrounds);
    for (int i = 0; i < kBsKeyWords; i++)
        if (((bits[i >> 5] >> (i & 31)) & 1u) != (words[i] & 1u)) return false;
    return true;
}

// The bitsliced pipeline of layout FOLD on the 32 blocks `in` against the
// table path's results, with its masks expanded all three ways (word by word,
// round by round by three threads, per word by five threads).
template <int NR, bool FOLD>
static bool bs_pipeline_matches(const uint32_t* bits, const uint32_t* in, const uint32_t* ref_lo,
                                const uint32_t* ref_hi) {
    using L = BsLayout<FOLD>;
    static uint32_t masks[L::kWords], again[L::kWords];
    for (int i = 0; i < L::kWords; i++) masks[i] = bs_mask_from_bits<FOLD>(bits, i);
    for (int t = 0; t < 3; t++) bs_expand_masks<FOLD>(bits, again, t, 3);
    for (int i = 0; i < L::kWords; i++)
        if (again[i] != masks[i]) return false;
    for (int t = 0; t < 5; t++) bs_expand_masks_per_word<FOLD>(bits, again, t, 5);
    for (int i = 0; i < L::kWords; i++)
        if (again[i] != masks[i]) return false;
    // the pipeline leaves the R-planes unmasked by construction
    for (int i = 0; i < 32; i++)
        if (masks[L::kPostR + i]) return false;
    uint32_t w[64];
    for (int i = 0; i < 64; i++) w[i] = in[i];
    bs_tdes32<NR, FOLD>(w, masks);
    for (int m = 0; m < 32; m++)
        if (w[m] != ref_lo[m] || w[32 + m] != ref_hi[m]) return false;
    return true;
}

static int self_test_impl() {
    // IP/FP networks against the tables.
    for (int bit = 1; bit <= 64; bit++) {
        uint32_t hi = bit <= 32 ? 1u << (32 - bit) : 0u, lo = bit > 32 ? 1u << (64 - bit) : 0u;
        initial_perm(hi, lo);
        const uint64_t out = ((uint64_t)hi << 32) | lo;
        // output bit i (1-based MSB) is input bit kIP[i-1]: the single set bit moves to the i with kIP[i-1] == bit
        for (int i = 1; i <= 64; i++) {
            const bool set = (out >> (64 - i)) & 1u;
            if (set != (fips::kIP[i - 1] == bit)) return DES3_EINVAL;
        }
    }
    for (int bit = 1; bit <= 64; bit++) {
        uint32_t hi = bit <= 32 ? 1u << (32 - bit) : 0u, lo = bit > 32 ? 1u << (64 - bit) : 0u;
        final_perm(hi, lo);
        const uint64_t out = ((uint64_t)hi << 32) | lo;
        for (int i = 1; i <= 64; i++) {
            const bool set = (out >> (64 - i)) & 1u;
            if (set != (fips::kFP[i - 1] == bit)) return DES3_EINVAL;
        }
    }
    // Combined S+P tables: P applied to S, bit by bit.
    constexpr SpTable sp = make_sp_table();
    for (int j = 0; j < 8; j++)
        for (uint32_t x = 0; x < 64; x++) {
            const uint32_t s = fips::sbox(j, x);
            for (int t = 0; t < 4; t++) {
                const int q = 4 * j + t + 1;  // S output bit
                int i = 0;
                while (fips::kP[i] != q) i++;
                const uint32_t got = (sp.v[j][x] >> (31 - i)) & 1u;
                if (got != ((s >> (3 - t)) & 1u)) return DES3_EINVAL;
            }
        }
    // Rotated table round (the kernel's) against f(R, K) above, on seeded
    // halves and round keys: sp_round_rot(0, rotr(R, 1)) = rotr(f(R, K), 1).
    constexpr SpTable sp_rot = make_sp_rot_table();
    const HostRotLookup rlk{&sp_rot};
    {
        uint64_t z = 0x243F6A8885A308D3ull;
        auto next = [&]() {  // SplitMix64 steps
            z += 0x9E3779B97F4A7C15ull;
            uint64_t x = z;
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            return x ^ (x >> 31);
        };
        auto lk0 = [&](int jj, uint32_t off) { return sp.v[jj][off >> 7]; };
        for (int it = 0; it < 4096; it++) {
            const uint32_t r = (uint32_t)next();
            const uint64_t rk = next() & 0xFFFFFFFFFFFFull;
            uint32_t k8[8], ke, ko;
            for (int jj = 0; jj < 8; jj++) k8[jj] = sp_key_word(rk, jj);
            sp_rot_key(rk, &ke, &ko);
            const uint32_t want = rotr32(sp_f(r, k8, lk0), 1);
            if (sp_round_rot(0u, rotr32(r, 1), ke, ko, 0u, rlk) != want) return DES3_EINVAL;
        }
    }
    // LOP3 circuits against the S-boxes, all 64 inputs.
    for (int j = 0; j < 8; j++) {
        const BsCircuit& c = kBsCircuits[j];
        for (uint32_t x = 0; x < 64; x++) {
            int val[6 + 64];
            for (int m = 0; m < 6; m++) val[m] = (x >> (5 - m)) & 1u;
            for (int g = 0; g < c.ngates; g++) {
                const int k = val[c.g[g][0]] * 4 + val[c.g[g][1]] * 2 + val[c.g[g][2]];
                val[6 + g] = (c.g[g][3] >> k) & 1;
            }
            const uint32_t s = fips::sbox(j, x);
            for (int t = 0; t < 4; t++)
                if ((uint32_t)(val[c.out[t] >> 1] ^ (c.out[t] & 1)) != ((s >> (3 - t)) & 1u)) return DES3_EINVAL;
        }
    }
    // Whole pipelines on the host: the table path and the bitsliced path
    // (the exact device code, compiled for the host) must agree on 32 blocks.
    uint8_t key[24];
    for (int i = 0; i < 24; i++) key[i] = (uint8_t)(0x9D * i + 0x31);
    des3_ks_t ks;
    des3_key_schedule(key, &ks);
    uint32_t w[64];
    uint32_t ref_hi[32], ref_lo[32];
    for (int dir = 0; dir < 2; dir++) {
        for (int m = 0; m < 32; m++) {
            const uint32_t a = 0x01234567u * (m + 1) + 0x89ABCDEFu * dir, b = 0xFEDCBA98u ^ (m * 0x2545F491u);
            w[m] = a;
            w[32 + m] = b;
            // table path, one block: big-endian words of the little-endian pair
            uint32_t hi = bswap32(a), lo = bswap32(b);
            initial_perm(hi, lo);
            uint32_t L = hi, R = lo;
            uint32_t k8[8];
            auto lk = [&](int jj, uint32_t off) { return sp.v[jj][off >> 7]; };
            for (int r = 0; r < 48; r++) {
                for (int jj = 0; jj < 8; jj++) k8[jj] = sp_key_word(ks.rk[dir][r], jj);
                const bool update_L = ((r / 16) == 1) ? (r % 2 == 1) : (r % 2 == 0);
                if (update_L) L ^= sp_f(R, k8, lk);
                else R ^= sp_f(L, k8, lk);
            }
            hi = R;
            lo = L;
            final_perm(hi, lo);
            ref_lo[m] = bswap32(hi);
            ref_hi[m] = bswap32(lo);
            // the kernel's rotated table pipeline on the same block
            uint32_t rh[1] = {bswap32(a)}, rl[1] = {bswap32(b)};
            uint4 k4[24];
            rot_keys(ks.rk[dir], 48, k4);
            sp_tdes_rot<1, 3>(rh, rl, k4, 0u, rlk);
            if (bswap32(rh[0]) != ref_lo[m] || bswap32(rl[0]) != ref_hi[m]) return DES3_EINVAL;
        }
        static uint32_t bits[kBsMaskBitWords];
        bs_mask_bits(ks.rk[dir], bits);
        if (!packed_masks_match(ks.rk[dir], bits, 48)) return DES3_EINVAL;
        if (!bs_pipeline_matches<48, false>(bits, w, ref_lo, ref_hi)) return DES3_EINVAL;
        if (!bs_pipeline_matches<48, true>(bits, w, ref_lo, ref_hi)) return DES3_EINVAL;
    }
    // single DES (16 rounds): bitsliced against the table path
    des3_ks_t ks1;
    des3_key_schedule_des(key, &ks1);
    for (int dir = 0; dir < 2; dir++) {
        uint32_t v[64];
        for (int m = 0; m < 32; m++) {
            const uint32_t a = 0x9E3779B9u * (m + 7) ^ (uint32_t)dir, b = 0x85EBCA6Bu * (m + 3);
            v[m] = a;
            v[32 + m] = b;
            uint32_t hi = bswap32(a), lo = bswap32(b);
            initial_perm(hi, lo);
            uint32_t L = hi, R = lo, k8[8];
            auto lk = [&](int jj, uint32_t off) { return sp.v[jj][off >> 7]; };
            for (int r = 0; r < 16; r++) {
                for (int jj = 0; jj < 8; jj++) k8[jj] = sp_key_word(ks1.rk[dir][r], jj);
                if (r % 2 == 0) L ^= sp_f(R, k8, lk);
                else R ^= sp_f(L, k8, lk);
            }
            hi = R;
            lo = L;
            final_perm(hi, lo);
            ref_lo[m] = bswap32(hi);
            ref_hi[m] = bswap32(lo);
            uint32_t rh[1] = {bswap32(a)}, rl[1] = {bswap32(b)};
            uint4 k4[8];
            rot_keys(ks1.rk[dir], 16, k4);
            sp_tdes_rot<1, 1>(rh, rl, k4, 0u, rlk);
            if (bswap32(rh[0]) != ref_lo[m] || bswap32(rl[0]) != ref_hi[m]) return DES3_EINVAL;
        }
        static uint32_t bits1[kBsMaskBitWords];
        bs_mask_bits(ks1.rk[dir], bits1, 16);
        if (!packed_masks_match(ks1.rk[dir], bits1, 16)) return DES3_EINVAL;
        if (!bs_pipeline_matches<16, false>(bits1, v, ref_lo, ref_hi)) return DES3_EINVAL;
        if (!bs_pipeline_matches<16, true>(bits1, v, ref_lo, ref_hi)) return DES3_EINVAL;
    }
    return DES3_OK;
}

}  // namespace des3

using namespace des3;

extern "C" {

int des3_key_schedule(const uint8_t key[24], des3_ks_t* ks) {
    if (!key || !ks) return DES3_EINVAL;
    uint64_t sub[3][16];
    for (int i = 0; i < 3; i++) des_subkeys(key + 8 * i, sub[i]);
    std::memset(ks, 0, sizeof(*ks));
    ks->magic = DES3_KS_MAGIC;
    for (int r = 0; r < 16; r++) {
        ks->rk[0][r] = sub[0][r];        // E_K1: K1 forward
        ks->rk[0][16 + r] = sub[1][15 - r];  // D_K2: K2 backward
        ks->rk[0][32 + r] = sub[2][r];   // E_K3: K3 forward
    }
    for (int r = 0; r < 48; r++) ks->rk[1][r] = ks->rk[0][47 - r];
    return DES3_OK;
}

int des3_key_schedule_des(const uint8_t key[8], des3_ks_t* ks) {
    if (!key || !ks) return DES3_EINVAL;
    uint64_t sub[16];
    des_subkeys(key, sub);
    std::memset(ks, 0, sizeof(*ks));
    ks->magic = DES3_KS_MAGIC;
    ks->flags = DES3_KS_SINGLE_DES;
    for (int r = 0; r < 16; r++) {
        ks->rk[0][r] = sub[r];
        ks->rk[1][r] = sub[15 - r];
    }
    return DES3_OK;
}

int des3_ecb_crypt_ex(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes, int decrypt,
                      int kernel, des3_stream_t stream) {
    if (!ks || ((!d_in || !d_out) && nbytes)) return DES3_EINVAL;
    if (ks->magic != DES3_KS_MAGIC) return DES3_EKEY;
    if (nbytes % 8) return DES3_EINVAL;
    if (decrypt != 0 && decrypt != 1) return DES3_EINVAL;
    if (kernel < DES3_KERNEL_AUTO || kernel > DES3_KERNEL_SPTABLE) return DES3_EINVAL;
    if (nbytes == 0) return DES3_OK;
    if (((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 7) != 0) return DES3_EINVAL;
    if (overlaps_partially(d_in, d_out, nbytes)) return DES3_EINVAL;
    return launch_single(ks->rk[decrypt], static_cast<const uint8_t*>(d_in), static_cast<uint8_t*>(d_out),
                         nbytes / 8, kernel, reinterpret_cast<cudaStream_t>(stream), ks_rounds(ks));
}

static int mode_call(const des3_ks_t* ks, const uint8_t iv[8], const void* d_in, void* d_out, size_t nbytes,
                     int mode, des3_stream_t stream) {
    if (!ks || !iv || ((!d_in || !d_out) && nbytes)) return DES3_EINVAL;
    if (ks->magic != DES3_KS_MAGIC) return DES3_EKEY;
    if (nbytes % 8) return DES3_EINVAL;
    if (nbytes == 0) return DES3_OK;
    if (((reinterpret_cast<uintptr_t>(d_in) | reinterpret_cast<uintptr_t>(d_out)) & 7) != 0) return DES3_EINVAL;
    if (overlaps_partially(d_in, d_out, nbytes)) return DES3_EINVAL;
    if (mode == 2 && d_in == d_out) return DES3_EINVAL;  // CBC decryption reads the previous input block
    const LaunchShape sh = tuned_single(nbytes, DES3_KERNEL_BITSLICE);
    // CTR always encrypts the counters; CBC decryption decrypts the input
    uint64_t rk[48];
    rk48(ks, mode == 2 ? 1 : 0, rk);
    return launch_bitslice_mode(rk, static_cast<const uint8_t*>(d_in),
                                static_cast<uint8_t*>(d_out), nbytes / 8, mode, iv,
                                reinterpret_cast<cudaStream_t>(stream), sh.threads, sh.ctas_per_sm);
}

int des3_ctr_crypt(const des3_ks_t* ks, const uint8_t counter[8], const void* d_in, void* d_out, size_t nbytes,
                   des3_stream_t stream) {
    return mode_call(ks, counter, d_in, d_out, nbytes, 1, stream);
}

int des3_cbc_decrypt(const des3_ks_t* ks, const uint8_t iv[8], const void* d_in, void* d_out, size_t nbytes,
                     des3_stream_t stream) {
    return mode_call(ks, iv, d_in, d_out, nbytes, 2, stream);
}

int des3_ecb_encrypt(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes, des3_stream_t stream) {
    return des3_ecb_crypt_ex(ks, d_in, d_out, nbytes, 0, DES3_KERNEL_AUTO, stream);
}

int des3_ecb_decrypt(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes, des3_stream_t stream) {
    return des3_ecb_crypt_ex(ks, d_in, d_out, nbytes, 1, DES3_KERNEL_AUTO, stream);
}

const char* des3_strerror(int code) {
    switch (code) {
        case DES3_OK: return "ok";
        case DES3_EINVAL: return "invalid argument";
        case DES3_EKEY: return "key schedule not initialised by des3_key_schedule";
        case DES3_ECUDA: return "CUDA runtime error (see des3_last_cuda_error)";
        case DES3_ETIMEOUT: return "bounded device wait timed out";
        case DES3_ENOMEM: return "out of memory or admission budget exceeded";
        case DES3_ENODEV: return "no usable sm_103 CUDA device";
        case DES3_EBUSY: return "queue full";
        default: return "unknown error";
    }
}

int des3_last_cuda_error(void) { return t_last_cuda_error; }

int des3_self_test(void) { return self_test_impl(); }

int des3_kernel_info(int kernel, des3_kernel_info_t* info) {
    if (!info) return DES3_EINVAL;
    if (kernel == DES3_KERNEL_AUTO) kernel = DES3_KERNEL_BITSLICE;
    if (kernel == DES3_KERNEL_BITSLICE) {
        // per 32 blocks: 48 rounds x (16 key corrections + gates + 32 state
        // updates), four 32-word remasks (one before each DES, one unmask at
        // the end), and four 32x32 transposes of 256 instructions; the
        // corrections and the folded outputs' updates are multiply-adds when
        // DES3_BS_IMAD_CORR is set
        const double corr = 48.0 * (16.0 + DES3_BS_FOLDS) / 32.0;
        info->alu_ops_per_block = (48.0 * DES3_BS_OPS_PER_ROUND_F + 4.0 * 32.0 + 4.0 * 256.0) / 32.0 -
                                  (DES3_BS_IMAD_CORR ? corr : 0.0);
        info->fma_ops_per_block = DES3_BS_IMAD_CORR ? corr : 0.0;
        info->smem_loads_per_block = (double)kBsMaskWordsF / 32.0;
        info->sbox_gates = DES3_BS_SBOX_GATES_F;
        info->blocks_per_thread = 32;
        return DES3_OK;
    }
    if (kernel == DES3_KERNEL_SPTABLE) {
        // per round: 8 and-xor LOP3s (one per S-box field), 8 address
        // computations (a shift and an add each, counted once: the compiler
        // fuses them), 8 table loads, and the lookups XORed into the other
        // half three to a LOP3 (4).  Per block once: IP and FP (5 swap-moves
        // of 5 ops each), the rotations into and out of the rotated form (4)
        // and 4 byte swaps.  A 16-byte key load per two rounds is shared by
        // the thread's blocks: four on large buffers, which these figures are
        // for (fewer on buffers too small to give every thread slot four).
        info->alu_ops_per_block = 48.0 * (8 + 8 + 4) + 2 * 5 * 5 + 4 + 4;
        info->fma_ops_per_block = 0.0;
        info->smem_loads_per_block = 48.0 * 8 + 48.0 / 2 / 4;
        info->sbox_gates = 0;
        info->blocks_per_thread = 4;
        return DES3_OK;
    }
    return DES3_EINVAL;
}

const char* des3_version(void) { return "0.3.0"; }

}  // extern "C"
