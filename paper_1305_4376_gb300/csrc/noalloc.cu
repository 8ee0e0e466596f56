// noalloc.cu -- des3_ecb_batch_noalloc: the batched call for callers that
// cannot allocate device memory (see include/des3.h for who and why).
//
// The batched kernel reads two tables besides the caller's buffers: the job
// table (BatchTileJob, 40 bytes per job) and the packed key masks
// (kKeyBitsStride words per key and direction).  des3_ecb_batch allocates
// them per call; here they live in one fixed device array compiled into the
// library, sized for DES3_NOALLOC_MAX_JOBS jobs and DES3_NOALLOC_MAX_KEYS
// keys.  Host code cannot use the array's name as a device address, so the
// address is fetched once per device with cudaGetSymbolAddress.
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "tuning.h"

namespace des3 {
namespace {

constexpr size_t kJobsBytes = sizeof(BatchTileJob) * DES3_NOALLOC_MAX_JOBS;
constexpr size_t kKeysWords = (size_t)DES3_NOALLOC_MAX_KEYS * 2 * kKeyBitsStride;
static_assert(sizeof(BatchTileJob) == 40, "job record size is part of the stated scratch size");
static_assert(kKeyBitsStride * 2 * 4 == 832, "key record size is part of the stated scratch size");
static_assert(kJobsBytes % 256 == 0, "key table must stay 256-byte aligned");
static_assert(kJobsBytes + kKeysWords * 4 == DES3_NOALLOC_SCRATCH_BYTES, "scratch size as documented");

// The scratch array: job table, then packed key masks.
static __device__ __align__(256) unsigned char g_scratch[DES3_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;                 // guards the staging arrays and the per-device addresses
void* g_scratch_dev[64];         // device address of g_scratch, per device
BatchTileJob g_stage_jobs[DES3_NOALLOC_MAX_JOBS];
uint32_t g_stage_keys[kKeysWords];

// Device address of the scratch array on the current device (looked up once).
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= 64) return DES3_ENODEV;
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return DES3_OK;
}

}  // namespace
}  // namespace des3

using namespace des3;

extern "C" int des3_ecb_batch_noalloc(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs,
                                      uint32_t njobs, des3_stream_t stream) {
    if (njobs > DES3_NOALLOC_MAX_JOBS || nkeys > DES3_NOALLOC_MAX_KEYS) return DES3_EINVAL;
    if (nkeys && !keys) return DES3_EINVAL;
    for (uint32_t i = 0; i < nkeys; i++)
        if (keys[i].magic != DES3_KS_MAGIC) return DES3_EKEY;
    uint64_t ntiles = 0, total = 0;
    int rc = batch_validate(jobs, njobs, nkeys, &ntiles, &total);
    if (rc != DES3_OK || ntiles == 0) return rc;
    DeviceInfo di;
    if ((rc = current_device_info(&di)) != DES3_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    std::lock_guard<std::mutex> g(g_mu);
    void* base = nullptr;
    if ((rc = scratch_address(di.device, &base)) != DES3_OK) return rc;
    BatchTileJob* d_jobs = static_cast<BatchTileJob*>(base);
    uint32_t* d_keys = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + kJobsBytes);
    batch_fill_jobs(jobs, njobs, g_stage_jobs);
    batch_fill_keys(keys, nkeys, g_stage_keys);
    // Copies from pageable host memory are staged before cudaMemcpyAsync
    // returns, so the static staging arrays may be refilled by the next call.
    cudaError_t e = cudaMemcpyAsync(d_jobs, g_stage_jobs, sizeof(BatchTileJob) * njobs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemcpyAsync(d_keys, g_stage_keys, sizeof(uint32_t) * 2 * kKeyBitsStride * nkeys, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((rc = batch_prepare()) != DES3_OK) return rc;
    const BatchShape shape = tuned_batch_shape(total, njobs);
    return launch_batch(d_jobs, njobs, d_keys, ntiles, shape.ctas_per_sm, shape.threads, s);
}
