// kernels.cu -- the bitsliced single-buffer 3DES-EDE kernel for sm_103a (the
// table kernel is in sptable.cu).
//
// It computes, for every 64-bit block x of the buffer (paper Sec. II.A,
// ECB as in the abstract and Fig. 2):
//     encrypt: E_K3(D_K2(E_K1(x)))        decrypt: D_K1(E_K2(D_K3(x)))
// as IP, 48 Feistel rounds with the round keys in application order, FP.
// Between the three DES operations FP and the next IP cancel, so only the
// halves swap.
//
// * bitslice_kernel: each warp owns tiles of 1024 blocks; each lane holds
//   32 blocks as 64 bit planes, and the S-boxes are LOP3 circuits
//   (bs_generated.cuh).  E, P, IP and FP are renamings of registers.
// Global memory is read and written once, 16 bytes per lane per access,
// fully coalesced, with streaming cache hints.
#include "common.cuh"
#include "internal.h"
#include "tile_io.cuh"
#include "tuning.h"

namespace des3 {

// ------------------------------------------------------------------------
// Bitsliced kernel
// ------------------------------------------------------------------------

// Compiled for one CTA of kBsThreadsPerSm (384) threads per SM; smaller CTAs
// (more of them per SM) fit the same register budget.
constexpr int kBsThreads = kBsThreadsPerSm;
constexpr int kBsCtasPerSm = 1;

struct BsParams {
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    uint32_t vec;     // 1: in and out are 16-byte aligned
    uint32_t iv_w0;   // CBC: the IV's bytes 0..3 and 4..7 as little-endian words
    uint32_t iv_w1;
    uint32_t pad;
    uint64_t ctr0;    // CTR: the first counter block as a big-endian integer
    uint32_t mbits[kBsMaskBitWords];  // packed key masks (bs_mask_bits)
};

// ECB: out = E(in).  CTR: out = in ^ E(T0 + i), T0 + i the i-th counter
// block (SP 800-38A's standard increment of the whole big-endian block).
// CBC decryption: out_i = D(in_i) ^ in_{i-1}, in_{-1} = IV (out of place).
enum : int { kModeEcb = 0, kModeCtr = 1, kModeCbcDec = 2 };

// The lane's m-th block of a tile: 64 * (m / 2) + 2 * lane + (m % 2).
__device__ __forceinline__ uint32_t tile_block(int m, int lane) { return 64 * (m >> 1) + 2 * lane + (m & 1); }

template <int MODE, int NR>
__global__ void __launch_bounds__(kBsThreads, kBsCtasPerSm) bitslice_kernel(const __grid_constant__ BsParams p) {
    __shared__ __align__(16) uint32_t masks[kBsMaskWordsF];  // the folded rounds' layout
    bs_expand_masks_per_word<true>(p.mbits, masks, threadIdx.x, blockDim.x);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    // Warp numbers run across the CTAs first (warp w of CTA b is number
    // w * gridDim + b), so consecutive tiles go to different SMs: a buffer of
    // few tiles spreads over the whole GPU, and the last partial round of a
    // large one is shared by all SMs instead of piling onto the first CTAs.
    const uint64_t warp = (uint64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t ntiles = (p.nblocks + kTileBlocks - 1) / kTileBlocks;
    for (uint64_t t = warp; t < ntiles; t += nwarps) {
        const uint64_t first = t * kTileBlocks;
        const uint32_t valid = (uint32_t)min((uint64_t)kTileBlocks, p.nblocks - first);
        uint32_t w[64];
        if (MODE == kModeCtr) {
            // Counter blocks, big-endian: bytes 0..3 hold the high word.  The
            // lane's blocks lie 64 * (m / 2) + m % 2 <= 961 after its first
            // one, so unless the low word of some lane is about to wrap, the
            // high word is the same for all of them, its 32 bit planes are
            // constant words, and only the low words need a transpose.
            const uint64_t base = p.ctr0 + first + 2 * lane;
            const uint32_t lo0 = (uint32_t)base;
            if (__all_sync(0xFFFFFFFFu, lo0 <= 0xFFFFFFFFu - 1023u)) {
                const uint32_t hi = bswap32((uint32_t)(base >> 32));
#pragma unroll
                for (int q = 0; q < 32; q++) w[q] = 0u - ((hi >> q) & 1u);
#pragma unroll
                for (int m = 0; m < 32; m++) w[32 + m] = bswap32(lo0 + (uint32_t)(64 * (m >> 1) + (m & 1)));
                transpose32(w + 32);
            } else {
#pragma unroll
                for (int m = 0; m < 32; m++) {
                    const uint64_t c = base + (uint64_t)(64 * (m >> 1) + (m & 1));
                    w[m] = bswap32((uint32_t)(c >> 32));
                    w[32 + m] = bswap32((uint32_t)c);
                }
                transpose32(w);
                transpose32(w + 32);
            }
            bs_tdes32_planes<NR, true>(w, masks);
        } else {
            bs_load_tile(w, p.in + 8 * first, valid, p.vec, lane);
            bs_tdes32<NR, true>(w, masks);
        }
        if (MODE == kModeCtr) {
            // keystream XOR data, read and written with the tile's access pattern
            bs_xor_load_tile(w, p.in + 8 * first, valid, p.vec, lane);
        } else if (MODE == kModeCbcDec) {
            const uint2* src = reinterpret_cast<const uint2*>(p.in);
#pragma unroll
            for (int m = 0; m < 32; m++) {
                const uint64_t b = first + tile_block(m, lane);
                if (tile_block(m, lane) < valid) {
                    const uint2 prev = b == 0 ? make_uint2(p.iv_w0, p.iv_w1) : __ldcs(src + b - 1);
                    w[m] ^= prev.x;
                    w[32 + m] ^= prev.y;
                }
            }
        }
        bs_store_tile(w, p.out + 8 * first, valid, p.vec, lane);
    }
}

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------

int launch_bitslice_mode(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks, int mode,
                         const uint8_t iv[8], cudaStream_t s, int threads, int ctas_per_sm, int nrounds) {
    if (!shape_fits(DES3_TUNE_SINGLE, DES3_KERNEL_BITSLICE, threads, ctas_per_sm)) return DES3_EINVAL;
    if (nrounds != 48 && !(nrounds == 16 && mode == kModeEcb)) return DES3_EINVAL;
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    BsParams p;
    p.in = in;
    p.out = out;
    p.nblocks = nblocks;
    p.vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    p.iv_w0 = p.iv_w1 = p.pad = 0;
    p.ctr0 = 0;
    if (iv) {
        for (int i = 3; i >= 0; i--) p.iv_w0 = (p.iv_w0 << 8) | iv[i];
        for (int i = 7; i >= 4; i--) p.iv_w1 = (p.iv_w1 << 8) | iv[i];
        for (int i = 0; i < 8; i++) p.ctr0 = (p.ctr0 << 8) | iv[i];
    }
    bs_mask_bits(rk, p.mbits, nrounds);
    // one CTA per tile up to the persistent grid (SMs x CTAs per SM): a
    // small buffer gets one warp per SM rather than a few full CTAs
    const uint64_t ntiles = (nblocks + kTileBlocks - 1) / kTileBlocks;
    uint64_t grid = ntiles;
    const uint64_t maxgrid = (uint64_t)di.sms * ctas_per_sm;
    if (grid > maxgrid) grid = maxgrid;
    if (grid < 1) grid = 1;
    if (mode == kModeCtr) bitslice_kernel<kModeCtr, 48><<<(unsigned)grid, threads, 0, s>>>(p);
    else if (mode == kModeCbcDec) bitslice_kernel<kModeCbcDec, 48><<<(unsigned)grid, threads, 0, s>>>(p);
    else if (nrounds == 16) bitslice_kernel<kModeEcb, 16><<<(unsigned)grid, threads, 0, s>>>(p);
    else bitslice_kernel<kModeEcb, 48><<<(unsigned)grid, threads, 0, s>>>(p);
    return check_launch();
}

int launch_bitslice(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks,
                    cudaStream_t s, int threads, int ctas_per_sm, int nrounds) {
    return launch_bitslice_mode(rk, in, out, nblocks, kModeEcb, nullptr, s, threads, ctas_per_sm, nrounds);
}

}  // namespace des3
