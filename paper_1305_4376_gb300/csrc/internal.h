// internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "des3.h"

namespace des3 {

// Records the CUDA error for des3_last_cuda_error() and returns DES3_ECUDA.
int cuda_fail(cudaError_t e);
// Returns DES3_OK, or records and maps the launch error of the last launch.
int check_launch();

struct DeviceInfo {
    int device;
    int sms;
    int max_smem_optin;
};
// Cached properties of the current device; DES3_OK or an error code.
int current_device_info(DeviceInfo* out);

// One single-buffer launch.  rk: the round keys in application order (48 for
// 3DES, 16 for single DES: nrounds).  in/out: device pointers (8-byte
// aligned, may be equal); nblocks 64-bit blocks.
// threads / ctas_per_sm: the launch shape (see tuning.h); DES3_EINVAL if it
// does not fit the kernel's resources.
int launch_sptable(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks,
                   cudaStream_t s, int threads, int ctas_per_sm, int nrounds = 48);
int launch_bitslice(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks,
                    cudaStream_t s, int threads, int ctas_per_sm, int nrounds = 48);
// The bitsliced kernel in one of its modes (0 ECB, 1 CTR, 2 CBC decryption);
// iv: the 8-byte IV or first counter block (CTR, CBC), else null.
int launch_bitslice_mode(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks, int mode,
                         const uint8_t iv[8], cudaStream_t s, int threads, int ctas_per_sm, int nrounds = 48);
// Launches the single-buffer kernel and shape the tuning table picks.
int launch_single(const uint64_t* rk, const uint8_t* in, uint8_t* out, uint64_t nblocks,
                  int kernel, cudaStream_t s, int nrounds = 48);
// The 48 round keys of direction `dir` in 3DES application order; a single-
// DES schedule becomes 3DES with K1 = K2 = K3 (E_K D_K E_K = E_K), for the
// paths that only run 48 rounds.
void rk48(const des3_ks_t* ks, int dir, uint64_t out[48]);
inline int ks_rounds(const des3_ks_t* ks) { return (ks->flags & DES3_KS_SINGLE_DES) ? 16 : 48; }

// Blocks of work one bitsliced warp handles per tile (32 lanes x 32 blocks).
constexpr uint64_t kTileBlocks = 1024;

// The bitsliced kernels (single-buffer and batched) are compiled for this
// many threads per SM (__launch_bounds__(kBsThreadsPerSm, 1)), which holds
// them to 168 registers a thread: twelve warps per SM.  With the round code
// interleaved by depth they need 151 (single) and 162 (batched) registers
// without spilling, and measured 1.9 % faster than eight warps per SM; sixteen
// warps (127 registers) gained only 0.3 %.  Launch shapes with threads x
// CTAs per SM above this are rejected.
constexpr int kBsThreadsPerSm = 384;

// ---- batched launch (batch.cu) -----------------------------------------
struct BatchTileJob {     // one job as the device sees it
    const uint8_t* in;
    uint8_t* out;
    uint64_t nblocks;
    uint64_t tile_begin;  // index of the job's first tile in the global tile range
    uint32_t key_index;
    uint32_t decrypt;
};

#ifdef __CUDACC__
// The last job whose first unit (tile_begin) is <= u, for jobs in order of
// first unit starting at 0.  The whole warp searches: each step tests 32
// evenly spaced jobs of the remaining range at once (their tests come out
// true for a prefix of the lanes) and keeps the part after the last true one,
// so 4096 jobs take 3 rounds of loads instead of 12 one after another.  All
// 32 lanes must call it with the same u; each returns the same job.
__device__ __forceinline__ uint32_t warp_find_job(const BatchTileJob* jobs, uint32_t njobs, uint64_t u) {
    const uint64_t lane = threadIdx.x & 31;
    uint64_t lo = 0, n = njobs;  // the job is in [lo, lo + n)
    while (n > 1) {
        const uint64_t step = (n + 31) / 32;
        const uint64_t idx = lo + lane * step;
        const bool ok = lane == 0 || (idx < lo + n && jobs[idx].tile_begin <= u);
        const uint32_t last = 31 - __clz(__ballot_sync(0xFFFFFFFFu, ok));
        lo += last * step;
        n = min(step, n - last * step);
    }
    return (uint32_t)lo;
}
#endif

// Words of packed key masks per key and direction in a batch's device table
// (>= the bitsliced kernel's packed mask words, a multiple of 4).
constexpr int kKeyBitsStride = 104;

// Validates jobs against nkeys and returns the total tile count.
int batch_validate(const des3_job_t* jobs, uint32_t njobs, uint32_t nkeys, uint64_t* tiles,
                   uint64_t* total_bytes);
// Packed masks of every key, both directions (nkeys x 2 x kKeyBitsStride words).
void batch_fill_keys(const des3_ks_t* keys, uint32_t nkeys, uint32_t* out);
// Fills the device-side job table (host memory) from validated jobs; a job's
// tile_begin counts units of `grain` blocks (kTileBlocks for the bitsliced
// kernel, kSegBlocks for the table kernel).
void batch_fill_jobs(const des3_job_t* jobs, uint32_t njobs, BatchTileJob* out, uint64_t grain = kTileBlocks);
// Units of `grain` blocks over all jobs.
uint64_t batch_units(const des3_job_t* jobs, uint32_t njobs, uint64_t grain);

// ---- batched table kernel (sptable.cu) -----------------------------------
// A warp of the batched table kernel takes segments of kSegBlocks blocks (32
// lanes x 2 blocks); its job's round keys come from a device table of
// kSpKeyStride words per key and direction ((ke, ko) of the 48 rounds).
constexpr uint64_t kSegBlocks = 64;
constexpr int kSpKeyStride = 96;
// (ke, ko) round-key words of every key, both directions (nkeys x 2 x kSpKeyStride words).
void batch_fill_spkeys(const des3_ks_t* keys, uint32_t nkeys, uint32_t* out);
// Sets the batched table kernel's shared-memory limit (outside any stream capture).
int batch_prepare_sptable();
// Launches the batched table kernel over device-resident tables (tile_begin
// of the jobs in segments, nsegs segments in all).
int launch_batch_sptable(const BatchTileJob* d_jobs, uint32_t njobs, const uint32_t* d_spkeys, uint64_t nsegs,
                         int ctas_per_sm, int threads, cudaStream_t s);
// Sets the batched kernel's shared-memory limit (outside any stream capture).
int batch_prepare();
// Launches the persistent batched kernel over device-resident tables.
int launch_batch(const BatchTileJob* d_jobs, uint32_t njobs, const uint32_t* d_keybits,
                 uint64_t ntiles, int ctas_per_sm, int threads, cudaStream_t s);

}  // namespace des3
