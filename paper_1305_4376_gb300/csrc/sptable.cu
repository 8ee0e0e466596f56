// sptable.cu -- the table kernel: 3DES-EDE ECB with combined S+P tables in
// shared memory, for sm_103a.
//
// For every 64-bit block x of the buffer (paper Sec. II.A, ECB as in the
// abstract and Fig. 2): encrypt E_K3(D_K2(E_K1(x))), decrypt D_K1(E_K2(D_K3(x)))
// as IP, 48 Feistel rounds with the round keys in application order, FP.
// Each thread carries whole blocks (one to four, as the paper's kernel gives
// each thread its own block).  f(R,K) is eight lookups in combined S+P tables
// that live in shared memory, replicated once per lane so that every lookup
// of a warp hits 32 distinct banks; the halves are kept rotated by one bit so
// that each lookup's address is one LOP3, a shift and an add (sp_round_rot in
// sptable.cuh).  Global memory is read and written once, 16 bytes per access
// where the buffers allow it, with streaming cache hints.
#include <mutex>

#include "internal.h"
#include "sptable.cuh"
#include "tuning.h"

namespace des3 {

// ------------------------------------------------------------------------
// SP-table kernel
// ------------------------------------------------------------------------

// The rotated S+P tables in [entry][S-box] order (512 words), in global
// memory: word 8 x + j is entry x of S-box j.  The kernel reads them through
// L1 to fill its replicated copy; a warp's loads then fall on 4 consecutive
// words, and all of a thread's loads are in flight at once.  (Read from the
// constant bank, whose cache serialises distinct addresses, the fill took
// about 6 us per launch and dominated calls of 1 MiB and less.)
struct SpTableXJ {
    uint32_t v[64][8];
};
constexpr SpTableXJ make_sp_rot_xj() {
    SpTableXJ t{};
    const SpTable r = make_sp_rot_table();
    for (int x = 0; x < 64; x++)
        for (int j = 0; j < 8; j++) t.v[x][j] = r.v[j][x];
    return t;
}
__device__ const SpTableXJ g_sp_rot_xj = make_sp_rot_xj();

constexpr int kSpThreadsMax = 384;
constexpr int kSpCtasPerSm = 3;
constexpr int kSpTableBytes = 8 * 64 * 32 * 4;  // 64 KiB
constexpr int kSpKeyWords = 48 * 2;             // (ke, ko) per round
constexpr int kSpSmemBytes = kSpTableBytes + kSpKeyWords * 4;

struct SpParams {
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    uint32_t vec;   // 1: in and out are 16-byte aligned after `head` blocks
    uint32_t head;  // 1: block 0 is processed on its own (in and out 8 mod 16)
    uint32_t k[kSpKeyWords];
};

// Table word at shared-memory address addr + 128 J (addr: a 32-bit
// shared-window address that already holds the lane's base).
struct SmemLookup {
    template <int J>
    __device__ __forceinline__ uint32_t at(uint32_t addr) const {
        uint32_t v;
        asm("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(J * 128));
        return v;
    }
};

template <int NS>
__device__ __forceinline__ void sp_single(const SpParams& p, uint64_t blk, const uint4* k4, uint32_t tb) {
    uint2 v = __ldcs(reinterpret_cast<const uint2*>(p.in) + blk);
    uint32_t hi[1] = {bswap32(v.x)}, lo[1] = {bswap32(v.y)};
    sp_tdes_rot<1, NS>(hi, lo, k4, tb, SmemLookup{});
    __stcs(reinterpret_cast<uint2*>(p.out) + blk, make_uint2(bswap32(hi[0]), bswap32(lo[0])));
}

// NB consecutive blocks starting at block `b` of `base` (16-byte loads when
// vec and NB is even: b is then even and the address 16-byte aligned).
template <int NB>
__device__ __forceinline__ void sp_load(const uint8_t* base, uint64_t b, bool vec, uint32_t (&hi)[NB],
                                        uint32_t (&lo)[NB]) {
    if (NB % 2 == 0 && vec) {
#pragma unroll
        for (int i = 0; i < NB; i += 2) {
            const uint4 v = __ldcs(reinterpret_cast<const uint4*>(base) + b / 2 + i / 2);
            hi[i] = bswap32(v.x); lo[i] = bswap32(v.y);
            hi[i + 1] = bswap32(v.z); lo[i + 1] = bswap32(v.w);
        }
    } else {
#pragma unroll
        for (int i = 0; i < NB; i++) {
            const uint2 v = __ldcs(reinterpret_cast<const uint2*>(base) + b + i);
            hi[i] = bswap32(v.x); lo[i] = bswap32(v.y);
        }
    }
}

template <int NB>
__device__ __forceinline__ void sp_store(uint8_t* base, uint64_t b, bool vec, const uint32_t (&hi)[NB],
                                         const uint32_t (&lo)[NB]) {
    if (NB % 2 == 0 && vec) {
#pragma unroll
        for (int i = 0; i < NB; i += 2)
            __stcs(reinterpret_cast<uint4*>(base) + b / 2 + i / 2,
                   make_uint4(bswap32(hi[i]), bswap32(lo[i]), bswap32(hi[i + 1]), bswap32(lo[i + 1])));
    } else {
#pragma unroll
        for (int i = 0; i < NB; i++)
            __stcs(reinterpret_cast<uint2*>(base) + b + i, make_uint2(bswap32(hi[i]), bswap32(lo[i])));
    }
}

// NS: 3 (3DES) or 1 (single DES).  NB: blocks per thread and iteration (1,
// 2 or 4), more for independent work to hide latency with, fewer for more
// threads on small buffers; the launcher picks it from the buffer size.
template <int NS, int NB>
__global__ void __launch_bounds__(kSpThreadsMax, kSpCtasPerSm) sptable_kernel(const __grid_constant__ SpParams p) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint4* tab4 = reinterpret_cast<uint4*>(smem);
    uint32_t* sk = smem + kSpTableBytes / 4;
    // 16-byte stores of four lanes' copies: store i holds entry i >> 6 of
    // S-box (i >> 3) & 7 for lanes 4 (i & 7) .. 4 (i & 7) + 3, i.e. word
    // i >> 3 of the [entry][S-box] table
    constexpr int kStores = kSpTableBytes / 16;
    constexpr int kChunk = 16;  // loads in flight per thread
    const uint32_t* src = &g_sp_rot_xj.v[0][0];
    for (int base = threadIdx.x; base < kStores; base += kChunk * blockDim.x) {
        uint32_t v[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; k++) {
            const int i = base + k * blockDim.x;
            v[k] = i < kStores ? __ldg(src + (i >> 3)) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kChunk; k++) {
            const int i = base + k * blockDim.x;
            if (i < kStores) tab4[i] = make_uint4(v[k], v[k], v[k], v[k]);
        }
    }
    for (int i = threadIdx.x; i < kSpKeyWords; i += blockDim.x) sk[i] = p.k[i];
    __syncthreads();
    const uint32_t tb = (uint32_t)__cvta_generic_to_shared(smem) + 4 * (threadIdx.x & 31);
    const uint4* k4 = reinterpret_cast<const uint4*>(sk);

    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t body = p.nblocks - p.head;
    const uint64_t nunits = body / NB;
    const uint8_t* in = p.in + 8 * (uint64_t)p.head;
    uint8_t* out = p.out + 8 * (uint64_t)p.head;
    // CTA b takes the contiguous units [b n / grid, (b + 1) n / grid): every
    // CTA gets the same work to within one unit, and with the grid a multiple
    // of the SM count, so does every SM
    const uint64_t u0 = nunits * blockIdx.x / gridDim.x, u1 = nunits * (blockIdx.x + 1) / gridDim.x;
    for (uint64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        uint32_t hi[NB], lo[NB];
        sp_load<NB>(in, u * NB, p.vec, hi, lo);
        sp_tdes_rot<NB, NS>(hi, lo, k4, tb, SmemLookup{});
        sp_store<NB>(out, u * NB, p.vec, hi, lo);
    }
    // at most NB blocks left over, one per thread: the body's last
    // body % NB blocks and the unaligned head block
    const uint64_t rem = body % NB;
    if (gtid < rem) sp_single<NS>(p, p.head + nunits * NB + gtid, k4, tb);
    if (p.head && gtid == rem) sp_single<NS>(p, 0, k4, tb);
}

// ------------------------------------------------------------------------
// Batched table kernel: many buffers with a key and direction each.
//
// The jobs are cut into segments of kSegBlocks (64) blocks, a warp's worth
// at two blocks per lane; a job of n blocks owns ceil(n / 64) consecutive
// segments (its tile_begin counts segments).  Every warp takes a contiguous
// range of the global segment sequence, finds its first job by a warp-wide
// search (warp_find_job) and walks on, and keeps the current job's 96
// round-key words in its own slot of shared memory, reloaded only when the
// key or direction changes.  A segment's data loads are issued before that
// reload, so that with one small job after another the two trips to memory
// overlap.
// The per-block arithmetic is the single-buffer table kernel's.  Against the
// bitsliced batch, whose grain is a 1024-block tile, a job far below one tile
// costs a 64-block segment instead of a whole tile.
// ------------------------------------------------------------------------

__global__ void __launch_bounds__(kSpThreadsMax, kSpCtasPerSm)
    batch_sptable_kernel(const BatchTileJob* __restrict__ jobs, uint32_t njobs, const uint32_t* __restrict__ spkeys,
                         uint64_t nsegs) {
    extern __shared__ __align__(16) uint32_t smem[];
    uint4* tab4 = reinterpret_cast<uint4*>(smem);
    constexpr int kStores = kSpTableBytes / 16;
    constexpr int kChunk = 16;
    const uint32_t* src = &g_sp_rot_xj.v[0][0];
    for (int base = threadIdx.x; base < kStores; base += kChunk * blockDim.x) {
        uint32_t v[kChunk];
#pragma unroll
        for (int k = 0; k < kChunk; k++) {
            const int i = base + k * blockDim.x;
            v[k] = i < kStores ? __ldg(src + (i >> 3)) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kChunk; k++) {
            const int i = base + k * blockDim.x;
            if (i < kStores) tab4[i] = make_uint4(v[k], v[k], v[k], v[k]);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint32_t* wkeys = smem + kSpTableBytes / 4 + (threadIdx.x >> 5) * kSpKeyStride;  // this warp's round keys
    const uint32_t tb = (uint32_t)__cvta_generic_to_shared(smem) + 4 * lane;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t s0 = nsegs * warp / nwarps, s1 = nsegs * (warp + 1) / nwarps;
    uint32_t cur_key = 0xFFFFFFFFu, cur_dir = 0xFFFFFFFFu;
    uint32_t j = s0 < s1 ? warp_find_job(jobs, njobs, s0) : 0;
    for (uint64_t sg = s0; sg < s1; sg++) {
        while (j + 1 < njobs && jobs[j + 1].tile_begin <= sg) j++;
        const BatchTileJob job = jobs[j];
        const uint64_t first = (sg - job.tile_begin) * kSegBlocks;
        const uint64_t left = job.nblocks - first;
        const uint32_t valid = left < kSegBlocks ? (uint32_t)left : (uint32_t)kSegBlocks;
        const uint32_t b = 2 * lane;  // the lane's blocks: b and b + 1 of the segment
        const uint2* in = reinterpret_cast<const uint2*>(job.in) + first;
        uint2* out = reinterpret_cast<uint2*>(job.out) + first;
        uint2 v[2];
#pragma unroll
        for (int i = 0; i < 2; i++) v[i] = b + i < valid ? __ldcs(in + b + i) : make_uint2(0u, 0u);
        if (job.key_index != cur_key || job.decrypt != cur_dir) {
            __syncwarp();
            const uint32_t* kw = spkeys + ((uint64_t)job.key_index * 2 + job.decrypt) * kSpKeyStride;
            for (int i = lane; i < kSpKeyStride; i += 32) wkeys[i] = kw[i];
            __syncwarp();
            cur_key = job.key_index;
            cur_dir = job.decrypt;
        }
        uint32_t hi[2], lo[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            hi[i] = bswap32(v[i].x);
            lo[i] = bswap32(v[i].y);
        }
        sp_tdes_rot<2, 3>(hi, lo, reinterpret_cast<const uint4*>(wkeys), tb, SmemLookup{});
#pragma unroll
        for (int i = 0; i < 2; i++)
            if (b + i < valid) __stcs(out + b + i, make_uint2(bswap32(hi[i]), bswap32(lo[i])));
    }
}

namespace {
std::mutex g_attr_mu;
bool g_sp_attr_done[64];
bool g_bsp_attr_done[64];

int batch_sptable_smem(int threads) { return kSpTableBytes + (threads / 32) * kSpKeyStride * 4; }
}  // namespace

void batch_fill_spkeys(const des3_ks_t* keys, uint32_t nkeys, uint32_t* out) {
    for (uint32_t k = 0; k < nkeys; k++)
        for (int dir = 0; dir < 2; dir++) {
            uint32_t* o = out + ((uint64_t)k * 2 + dir) * kSpKeyStride;
            uint64_t rk[48];
            rk48(&keys[k], dir, rk);
            for (int r = 0; r < 48; r++) sp_rot_key(rk[r], &o[2 * r], &o[2 * r + 1]);
        }
}

int batch_prepare_sptable() {
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    std::lock_guard<std::mutex> g(g_attr_mu);
    if (di.device < 64 && !g_bsp_attr_done[di.device]) {
        const cudaError_t e = cudaFuncSetAttribute(batch_sptable_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   batch_sptable_smem(kSpThreadsMax));
        if (e != cudaSuccess) return cuda_fail(e);
        g_bsp_attr_done[di.device] = true;
    }
    return DES3_OK;
}

int launch_batch_sptable(const BatchTileJob* d_jobs, uint32_t njobs, const uint32_t* d_spkeys, uint64_t nsegs,
                         int ctas_per_sm, int threads, cudaStream_t s) {
    if (nsegs == 0 || njobs == 0) return DES3_OK;
    if (!shape_fits(DES3_TUNE_BATCH, DES3_KERNEL_SPTABLE, threads, ctas_per_sm)) return DES3_EINVAL;
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    const uint64_t warps_per_cta = (uint64_t)threads / 32;
    uint64_t grid = (nsegs + warps_per_cta - 1) / warps_per_cta;
    const uint64_t maxgrid = (uint64_t)di.sms * (uint64_t)ctas_per_sm;
    if (grid > maxgrid) grid = maxgrid;
    batch_sptable_kernel<<<(unsigned)grid, threads, batch_sptable_smem(threads), s>>>(d_jobs, njobs, d_spkeys, nsegs);
    return check_launch();
}

template <int NS, int NB>
int set_sp_attr() {
    const cudaError_t e = cudaFuncSetAttribute(sptable_kernel<NS, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               kSpSmemBytes);
    return e == cudaSuccess ? DES3_OK : cuda_fail(e);
}

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
            int r = set_sp_attr<3, 1>();
            if (r == DES3_OK) r = set_sp_attr<3, 2>();
            if (r == DES3_OK) r = set_sp_attr<3, 4>();
            if (r == DES3_OK) r = set_sp_attr<1, 1>();
            if (r == DES3_OK) r = set_sp_attr<1, 2>();
            if (r == DES3_OK) r = set_sp_attr<1, 4>();
            if (r != DES3_OK) return r;
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
    for (int r = 0; r < 48; r++) {
        uint32_t ke = 0, ko = 0;
        if (r < nrounds) sp_rot_key(rk[r], &ke, &ko);
        p.k[2 * r] = ke;
        p.k[2 * r + 1] = ko;
    }
    // Blocks per thread: four once every thread slot of the grid gets four,
    // two once every slot gets one, else one (more threads for small buffers).
    const uint64_t body = nblocks - p.head;
    const uint64_t slots = (uint64_t)di.sms * ctas_per_sm * threads;
    const int nb = body >= 4 * slots ? 4 : body >= slots ? 2 : 1;
    // Grid: whole CTAs per SM, as many as the units need (at most
    // ctas_per_sm), so that the per-CTA ranges of the kernel are the same on
    // every SM; buffers too small to give each SM a full CTA use fewer CTAs.
    const uint64_t units = body / nb + 1;
    const uint64_t per_sm = (units + (uint64_t)di.sms * threads - 1) / ((uint64_t)di.sms * threads);
    uint64_t grid = (uint64_t)di.sms * (per_sm < (uint64_t)ctas_per_sm ? per_sm : (uint64_t)ctas_per_sm);
    const uint64_t need = (units + threads - 1) / threads;
    if (need < (uint64_t)di.sms) grid = need;
    if (grid < 1) grid = 1;
    const unsigned g = (unsigned)grid;
    if (nrounds == 16) {
        if (nb == 4) sptable_kernel<1, 4><<<g, threads, kSpSmemBytes, s>>>(p);
        else if (nb == 2) sptable_kernel<1, 2><<<g, threads, kSpSmemBytes, s>>>(p);
        else sptable_kernel<1, 1><<<g, threads, kSpSmemBytes, s>>>(p);
    } else {
        if (nb == 4) sptable_kernel<3, 4><<<g, threads, kSpSmemBytes, s>>>(p);
        else if (nb == 2) sptable_kernel<3, 2><<<g, threads, kSpSmemBytes, s>>>(p);
        else sptable_kernel<3, 1><<<g, threads, kSpSmemBytes, s>>>(p);
    }
    return check_launch();
}

}  // namespace des3
