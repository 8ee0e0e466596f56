// noalloc.cu -- des3_ecb_batch_noalloc: the batched call for callers that
// cannot allocate device memory (see include/des3.h for who and why).
//
// The batched kernel reads two tables besides the caller's buffers: the job
// table (BatchTileJob, 40 bytes per job) and the packed key masks
// (kKeyBitsStride words per key and direction).  des3_ecb_batch allocates
// them per call; here they live in one fixed device array compiled into the
// library, sized for DES3_NOALLOC_MAX_JOBS jobs and DES3_NOALLOC_MAX_KEYS
// keys.  Host code cannot use the array's name as a device address, so the
// address is fetched once per device with cudaGetSymbolAddress, and fetched
// again when the device's context has been replaced (cudaDeviceReset
// destroys the primary context; the array then lives at a new address in
// the next one).
#include <cuda.h>  // driver types only: the two driver calls are looked up at run time

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

std::mutex g_mu;                      // guards the staging arrays and the per-device addresses
void* g_scratch_dev[64];              // device address of g_scratch, per device ...
unsigned long long g_scratch_ctx[64];  // ... in the context with this id (0: none yet)
BatchTileJob g_stage_jobs[DES3_NOALLOC_MAX_JOBS];
uint32_t g_stage_keys[kKeysWords];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
std::once_flag g_driver_once;

// Id of the calling thread's current context, or 0 if it cannot be read
// (then the address is looked up on every call, which is always right).
unsigned long long current_context_id() {
    std::call_once(g_driver_once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!g_ctx_get_current || !g_ctx_get_id || g_ctx_get_current(&c) != CUDA_SUCCESS || !c ||
        g_ctx_get_id(c, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up the
// first time, and again whenever the device's context is a new one.  Called
// with g_mu held, after a runtime call has made the context current.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= 64) return DES3_ENODEV;
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_dev[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        g_scratch_dev[dev] = p;
        g_scratch_ctx[dev] = ctx;
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
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // The tables are copied from the static staging arrays below, which the
    // next call overwrites; a copy recorded into a graph would replay some
    // later call's tables.  So a stream under capture is refused.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e);
    if (cap != cudaStreamCaptureStatusNone) return DES3_EINVAL;
    DeviceInfo di;
    if ((rc = current_device_info(&di)) != DES3_OK) return rc;

    std::lock_guard<std::mutex> g(g_mu);
    void* base = nullptr;
    if ((rc = scratch_address(di.device, &base)) != DES3_OK) return rc;
    BatchTileJob* d_jobs = static_cast<BatchTileJob*>(base);
    uint32_t* d_keys = reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + kJobsBytes);
    batch_fill_jobs(jobs, njobs, g_stage_jobs);
    batch_fill_keys(keys, nkeys, g_stage_keys);
    // Copies from pageable host memory are staged before cudaMemcpyAsync
    // returns, so the static staging arrays may be refilled by the next call.
    e = cudaMemcpyAsync(d_jobs, g_stage_jobs, sizeof(BatchTileJob) * njobs, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemcpyAsync(d_keys, g_stage_keys, sizeof(uint32_t) * 2 * kKeyBitsStride * nkeys, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e);
    if ((rc = batch_prepare()) != DES3_OK) return rc;
    const BatchShape shape = tuned_batch_shape(total, njobs);
    return launch_batch(d_jobs, njobs, d_keys, ntiles, shape.ctas_per_sm, shape.threads, s);
}
