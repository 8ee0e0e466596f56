// kernels.cu -- the two single-buffer 3DES-EDE ECB kernels for sm_103a.
//
// Both compute, for every 64-bit block x of the buffer (paper Sec. II.A,
// ECB as in the abstract and Fig. 2):
//     encrypt: E_K3(D_K2(E_K1(x)))        decrypt: D_K1(E_K2(D_K3(x)))
// as IP, 48 Feistel rounds with the round keys in application order, FP.
// Between the three DES operations FP and the next IP cancel, so only the
// halves swap (the three loops below alternate which half they update).
//
// * sptable_kernel: one block per thread (two per thread for ILP, as the
//   paper's kernel gives each thread its own block).  f(R,K) is eight
//   lookups in combined S+P tables that live in shared memory, replicated
//   once per lane (entry x of table j for lane l at word (64j + x) * 32 + l),
//   so that every lookup of a warp hits 32 distinct banks.
// * bitslice_kernel: each warp owns tiles of 1024 blocks; each lane holds
//   32 blocks as 64 bit planes, and the S-boxes are LOP3 circuits
//   (bs_generated.cuh).  E, P, IP and FP are renamings of registers.
// Global memory is read and written once, 16 bytes per lane per access,
// fully coalesced, with streaming cache hints.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tile_io.cuh"
#include "tuning.h"

namespace des3 {

// ------------------------------------------------------------------------
// SP-table kernel
// ------------------------------------------------------------------------

__constant__ SpTable c_sp = make_sp_table();

constexpr int kSpThreads = 256;
constexpr int kSpCtasPerSm = 3;
constexpr int kSpTableBytes = 8 * 64 * 32 * 4;  // 64 KiB
constexpr int kSpKeyWords = 48 * 8;
constexpr int kSpSmemBytes = kSpTableBytes + kSpKeyWords * 4;

struct SpParams {
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    uint32_t vec;   // 1: in and out are 16-byte aligned after `head` blocks
    uint32_t head;  // blocks processed one at a time before the pairs
    uint32_t k[kSpKeyWords];
};

struct SmemLookup {
    const char* tb;  // table base + 4 * lane
    __device__ __forceinline__ uint32_t operator()(int j, uint32_t off) const {
        return *reinterpret_cast<const uint32_t*>(tb + off + j * (64 * 128));
    }
};

// 3DES (NS = 3) or single DES (NS = 1) on NB blocks held as big-endian
// (hi, lo) word pairs.
template <int NB, int NS>
__device__ __forceinline__ void sp_tdes(uint32_t (&hi)[NB], uint32_t (&lo)[NB], const uint32_t* sk,
                                        const SmemLookup& lk) {
    uint32_t a[NB], b[NB];
#pragma unroll
    for (int i = 0; i < NB; i++) {
        initial_perm(hi[i], lo[i]);
        a[i] = hi[i];  // L0
        b[i] = lo[i];  // R0
    }
    const uint32_t* k = sk;
#pragma unroll 1
    for (int r = 0; r < 8; r++, k += 16) {
#pragma unroll
        for (int i = 0; i < NB; i++) a[i] ^= sp_f(b[i], k, lk);
#pragma unroll
        for (int i = 0; i < NB; i++) b[i] ^= sp_f(a[i], k + 8, lk);
    }
    if (NS == 3) {
#pragma unroll 1
        for (int r = 0; r < 8; r++, k += 16) {
#pragma unroll
            for (int i = 0; i < NB; i++) b[i] ^= sp_f(a[i], k, lk);
#pragma unroll
            for (int i = 0; i < NB; i++) a[i] ^= sp_f(b[i], k + 8, lk);
        }
#pragma unroll 1
        for (int r = 0; r < 8; r++, k += 16) {
#pragma unroll
            for (int i = 0; i < NB; i++) a[i] ^= sp_f(b[i], k, lk);
#pragma unroll
            for (int i = 0; i < NB; i++) b[i] ^= sp_f(a[i], k + 8, lk);
        }
    }
#pragma unroll
    for (int i = 0; i < NB; i++) {
        hi[i] = b[i];  // R16 of the last DES
        lo[i] = a[i];
        final_perm(hi[i], lo[i]);
    }
}

template <int NS>
__device__ __forceinline__ void sp_single(const SpParams& p, uint64_t blk, const uint32_t* sk,
                                          const SmemLookup& lk) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(p.in) + blk);
    uint32_t hi[1] = {bswap32(v.x)}, lo[1] = {bswap32(v.y)};
    sp_tdes<1, NS>(hi, lo, sk, lk);
    __stcs(reinterpret_cast<uint2*>(p.out) + blk, make_uint2(bswap32(hi[0]), bswap32(lo[0])));
}

template <int NS>
__global__ void __launch_bounds__(kSpThreads, kSpCtasPerSm) sptable_kernel(const __grid_constant__ SpParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t* tab = smem;
    uint32_t* sk = smem + kSpTableBytes / 4;
    for (int i = threadIdx.x; i < 8 * 64 * 32; i += blockDim.x) tab[i] = c_sp.v[0][i >> 5];
    for (int i = threadIdx.x; i < kSpKeyWords; i += blockDim.x) sk[i] = p.k[i];
    __syncthreads();
    const SmemLookup lk{reinterpret_cast<const char*>(tab) + 4 * (threadIdx.x & 31)};

    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gsize = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t body = p.nblocks - p.head;
    const uint64_t npairs = body / 2;
    const uint8_t* in = p.in + 8 * (uint64_t)p.head;
    uint8_t* out = p.out + 8 * (uint64_t)p.head;
    for (uint64_t u = gtid; u < npairs; u += gsize) {
        uint32_t hi[2], lo[2];
        if (p.vec) {
            uint4 v = __ldcs(reinterpret_cast<const uint4*>(in) + u);
            hi[0] = bswap32(v.x); lo[0] = bswap32(v.y);
            hi[1] = bswap32(v.z); lo[1] = bswap32(v.w);
        } else {
            uint2 v0 = __ldcs(reinterpret_cast<const uint2*>(in) + 2 * u);
            uint2 v1 = __ldcs(reinterpret_cast<const uint2*>(in) + 2 * u + 1);
            hi[0] = bswap32(v0.x); lo[0] = bswap32(v0.y);
            hi[1] = bswap32(v1.x); lo[1] = bswap32(v1.y);
        }
        sp_tdes<2, NS>(hi, lo, sk, lk);
        if (p.vec) {
            __stcs(reinterpret_cast<uint4*>(out) + u,
                   make_uint4(bswap32(hi[0]), bswap32(lo[0]), bswap32(hi[1]), bswap32(lo[1])));
        } else {
            __stcs(reinterpret_cast<uint2*>(out) + 2 * u, make_uint2(bswap32(hi[0]), bswap32(lo[0])));
            __stcs(reinterpret_cast<uint2*>(out) + 2 * u + 1, make_uint2(bswap32(hi[1]), bswap32(lo[1])));
        }
    }
    // at most two blocks left over: the unaligned head and an odd tail
    if (gtid == 0 && p.head) sp_single<NS>(p, 0, sk, lk);
    if (gtid == (gsize > 1 ? 1 : 0) && (body & 1)) sp_single<NS>(p, p.nblocks - 1, sk, lk);
}

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
    __shared__ __align__(16) uint32_t masks[kBsMaskWords];
    for (int i = threadIdx.x; i < kBsMaskWords; i += blockDim.x) masks[i] = bs_mask_from_bits(p.mbits, i);
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
            bs_tdes32_planes<NR>(w, masks);
        } else {
            bs_load_tile(w, p.in + 8 * first, valid, p.vec, lane);
            bs_tdes32<NR>(w, masks);
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

namespace {
std::mutex g_attr_mu;
bool g_sp_attr_done[64];
}  // namespace

int launch_sptable(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks,
                   cudaStream_t s, int threads, int ctas_per_sm, int nrounds) {
    if (nrounds != 16 && nrounds != 48) return DES3_EINVAL;
    if (!shape_fits(DES3_TUNE_SINGLE, DES3_KERNEL_SPTABLE, threads, ctas_per_sm)) return DES3_EINVAL;
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    {
        std::lock_guard<std::mutex> g(g_attr_mu);
        if (di.device < 64 && !g_sp_attr_done[di.device]) {
            cudaError_t e = cudaFuncSetAttribute(sptable_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kSpSmemBytes);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(sptable_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpSmemBytes);
            if (e != cudaSuccess) return cuda_fail(e);
            g_sp_attr_done[di.device] = true;
        }
    }
    SpParams p;
    p.in = in;
    p.out = out;
    p.nblocks = nblocks;
    const uintptr_t ai = reinterpret_cast<uintptr_t>(in), ao = reinterpret_cast<uintptr_t>(out);
    p.head = 0;
    p.vec = 0;
    if ((ai & 15) == (ao & 15)) {
        p.vec = 1;
        p.head = (ai & 15) ? 1 : 0;
        if (p.head > nblocks) p.head = 0, p.vec = 0;
    }
    for (int r = 0; r < 48; r++)
        for (int j = 0; j < 8; j++) p.k[r * 8 + j] = r < nrounds ? sp_key_word(rk[r], j) : 0u;
    const uint64_t units = (nblocks - p.head) / 2 + 1;
    uint64_t grid = (units + threads - 1) / threads;
    const uint64_t maxgrid = (uint64_t)di.sms * ctas_per_sm;
    if (grid > maxgrid) grid = maxgrid;
    if (grid < 1) grid = 1;
    if (nrounds == 16) sptable_kernel<1><<<(unsigned)grid, threads, kSpSmemBytes, s>>>(p);
    else sptable_kernel<3><<<(unsigned)grid, threads, kSpSmemBytes, s>>>(p);
    return check_launch();
}

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
