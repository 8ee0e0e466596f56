// batch.cu -- many buffers, each with its own key schedule and direction,
// in one persistent launch (optionally replayed from a CUDA graph).  The
// tuning table picks, per size class of the batch's total bytes, the
// bitsliced batched kernel below or the batched table kernel (sptable.cu).
//
// The arithmetic per block is exactly the single-buffer bitsliced kernel's
// (paper Sec. II.A, ECB): only the bookkeeping differs.  The work is cut into
// tiles of 1024 blocks (one warp, 32 blocks per lane); a job of n blocks owns
// ceil(n / 1024) consecutive tiles, the last one partial.  Every warp takes a
// contiguous range of the global tile sequence, so it rarely changes job, and
// finds its first tile's job by a warp-wide search over the jobs' first-tile
// indices (warp_find_job).
// When the job's key or direction changes, the warp rebuilds its 48 x 48 key
// masks in its own slice of shared memory.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tile_io.cuh"
#include "tuning.h"

namespace des3 {

constexpr int kMaskWords = kBsMaskWords;
static_assert(kKeyBitsStride >= kBsMaskBitWords && kKeyBitsStride % 4 == 0, "packed key masks must fit their slot");

__global__ void __launch_bounds__(kBsThreadsPerSm, 1) batch_bitslice_kernel(const BatchTileJob* __restrict__ jobs, uint32_t njobs,
                                                             const uint32_t* __restrict__ keybits, uint64_t ntiles) {
    extern __shared__ __align__(16) uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    uint32_t* masks = smem + wib * kMaskWords;
    const uint64_t warp = (uint64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    // contiguous share of the tile range
    const uint64_t t0 = ntiles * warp / nwarps, t1 = ntiles * (warp + 1) / nwarps;
    uint32_t cur_key = 0xFFFFFFFFu, cur_dir = 0xFFFFFFFFu;
    uint32_t j = t0 < t1 ? warp_find_job(jobs, njobs, t0) : 0;
    for (uint64_t t = t0; t < t1; t++) {
        while (j + 1 < njobs && jobs[j + 1].tile_begin <= t) j++;
        const BatchTileJob job = jobs[j];
        if (job.key_index != cur_key || job.decrypt != cur_dir) {
            __syncwarp();
            const uint32_t* kb = keybits + ((uint64_t)job.key_index * 2 + job.decrypt) * kKeyBitsStride;
            bs_expand_masks<false>(kb, masks, lane, 32);
            __syncwarp();
            cur_key = job.key_index;
            cur_dir = job.decrypt;
        }
        const uint64_t first = (t - job.tile_begin) * kTileBlocks;
        const uint32_t valid = (uint32_t)min((uint64_t)kTileBlocks, job.nblocks - first);
        const bool vec = ((reinterpret_cast<uintptr_t>(job.in) | reinterpret_cast<uintptr_t>(job.out)) & 15) == 0;
        uint32_t w[64];
        bs_load_tile(w, job.in + 8 * first, valid, vec, lane);
        bs_tdes32<48, false>(w, masks);
        bs_store_tile(w, job.out + 8 * first, valid, vec, lane);
    }
}

int batch_validate(const des3_job_t* jobs, uint32_t njobs, uint32_t nkeys, uint64_t* tiles, uint64_t* total_bytes) {
    if (njobs && !jobs) return DES3_EINVAL;
    uint64_t t = 0, b = 0;
    for (uint32_t i = 0; i < njobs; i++) {
        const des3_job_t& jb = jobs[i];
        if (jb.nbytes % 8) return DES3_EINVAL;
        if (jb.flags & ~DES3_JOB_DECRYPT) return DES3_EINVAL;
        if (jb.key_index >= nkeys) return DES3_EINVAL;
        if (jb.nbytes == 0) continue;
        if (!jb.d_in || !jb.d_out) return DES3_EINVAL;
        if (((reinterpret_cast<uintptr_t>(jb.d_in) | reinterpret_cast<uintptr_t>(jb.d_out)) & 7) != 0) return DES3_EINVAL;
        const uintptr_t x = reinterpret_cast<uintptr_t>(jb.d_in), y = reinterpret_cast<uintptr_t>(jb.d_out);
        if (x != y && x < y + jb.nbytes && y < x + jb.nbytes) return DES3_EINVAL;
        t += (jb.nbytes / 8 + kTileBlocks - 1) / kTileBlocks;
        b += jb.nbytes;
    }
    *tiles = t;
    *total_bytes = b;
    return DES3_OK;
}

void batch_fill_keys(const des3_ks_t* keys, uint32_t nkeys, uint32_t* out) {
    for (uint32_t k = 0; k < nkeys; k++)
        for (int dir = 0; dir < 2; dir++) {
            uint32_t* o = out + ((uint64_t)k * 2 + dir) * kKeyBitsStride;
            for (int i = 0; i < kKeyBitsStride; i++) o[i] = 0;
            uint64_t rk[48];
            rk48(&keys[k], dir, rk);
            bs_mask_bits(rk, o);
        }
}

// The grain is a power of two (kTileBlocks or kSegBlocks): units are counted
// with a shift, not a 64-bit division per job.
static int grain_shift(uint64_t grain) {
    int sh = 0;
    while ((1ull << sh) < grain) sh++;
    return sh;
}

void batch_fill_jobs(const des3_job_t* jobs, uint32_t njobs, BatchTileJob* out, uint64_t grain) {
    const int sh = grain_shift(grain);
    uint64_t t = 0;
    for (uint32_t i = 0; i < njobs; i++) {
        const des3_job_t& jb = jobs[i];
        BatchTileJob& o = out[i];
        o.in = static_cast<const uint8_t*>(jb.d_in);
        o.out = static_cast<uint8_t*>(jb.d_out);
        o.nblocks = jb.nbytes / 8;
        o.tile_begin = t;
        o.key_index = jb.key_index;
        o.decrypt = jb.flags & DES3_JOB_DECRYPT;
        t += (o.nblocks + grain - 1) >> sh;
    }
}

uint64_t batch_units(const des3_job_t* jobs, uint32_t njobs, uint64_t grain) {
    const int sh = grain_shift(grain);
    uint64_t t = 0;
    for (uint32_t i = 0; i < njobs; i++) t += (jobs[i].nbytes / 8 + grain - 1) >> sh;
    return t;
}

int batch_prepare() {
    // the largest CTA (12 warps x 12.6 KiB of masks) is allowed once; smaller
    // CTAs use less of it
    cudaError_t e = cudaFuncSetAttribute(batch_bitslice_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (kBsThreadsPerSm / 32) * kMaskWords * 4);
    return e == cudaSuccess ? DES3_OK : cuda_fail(e);
}

int launch_batch(const BatchTileJob* d_jobs, uint32_t njobs, const uint32_t* d_keybits, uint64_t ntiles,
                 int ctas_per_sm, int threads, cudaStream_t s) {
    if (ntiles == 0 || njobs == 0) return DES3_OK;
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    if (!shape_fits(DES3_TUNE_BATCH, DES3_KERNEL_BITSLICE, threads, ctas_per_sm)) return DES3_EINVAL;
    const int smem = (threads / 32) * kMaskWords * 4;
    // One CTA per SM: always the whole grid.  With fewer tiles than warps,
    // the warps' equal contiguous shares leave the busy warps evenly spaced
    // over the CTAs, so a small batch spreads over the SMs instead of
    // stacking its tiles on a few of them: a single job of 64 KiB to 1 MiB
    // took 33-45 us on the fewest CTAs that hold its tiles, 21 us on all.
    // Several CTAs per SM: the fewest CTAs, up to the grid (a 4 MiB job on
    // 64 x 4 took 22.6 us so and 34 us on the whole grid).
    const uint64_t warps_per_cta = threads / 32;
    const uint64_t maxgrid = (uint64_t)di.sms * (uint64_t)std::max(1, ctas_per_sm);
    uint64_t grid = ctas_per_sm <= 1 ? maxgrid : (ntiles + warps_per_cta - 1) / warps_per_cta;
    if (grid > maxgrid) grid = maxgrid;
    batch_bitslice_kernel<<<(unsigned)grid, threads, smem, s>>>(d_jobs, njobs, d_keybits, ntiles);
    return check_launch();
}

}  // namespace des3

using namespace des3;

namespace {

int check_keys(const des3_ks_t* keys, uint32_t nkeys) {
    if (nkeys && !keys) return DES3_EINVAL;
    for (uint32_t i = 0; i < nkeys; i++)
        if (keys[i].magic != DES3_KS_MAGIC) return DES3_EKEY;
    return DES3_OK;
}

// The kernel and shape for a batch: the tuning table's entry for its size
// class; where that names the bitsliced kernel but the jobs fill their tiles
// so sparsely that the wave model predicts the table kernel faster, the
// table kernel in its default shape.  An explicit kernel keeps the table's
// shape when the table names it, else takes that kernel's default shape.
BatchShape choose_batch_shape(const des3_job_t* jobs, uint32_t njobs, uint64_t ntiles, uint64_t total, int kernel,
                              int sms) {
    if (kernel == DES3_KERNEL_AUTO)
        return auto_batch_shape(total, njobs, ntiles, batch_units(jobs, njobs, kSegBlocks), sms);
    const BatchShape shape = tuned_batch_shape(total, njobs, true);
    if (kernel == shape.kernel) return shape;
    return kernel == DES3_KERNEL_SPTABLE ? kTableBatchDefault : kBitsliceBatchDefault;
}

}  // namespace

struct des3_batch_plan {
    int device = -1;
    uint32_t njobs = 0;
    uint64_t ntiles = 0;
    uint64_t total_bytes = 0;
    BatchShape shape{};     // the captured launch's kernel and shape
    void* d_mem = nullptr;  // jobs, then the key table
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

int des3_ecb_batch(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs, uint32_t njobs,
                   des3_stream_t stream) {
    int rc = check_keys(keys, nkeys);
    if (rc != DES3_OK) return rc;
    uint64_t ntiles = 0, total = 0;
    if ((rc = batch_validate(jobs, njobs, nkeys, &ntiles, &total)) != DES3_OK) return rc;
    if (ntiles == 0) return DES3_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DeviceInfo di;
    if ((rc = current_device_info(&di)) != DES3_OK) return rc;
    const BatchShape shape = choose_batch_shape(jobs, njobs, ntiles, total, DES3_KERNEL_AUTO, di.sms);
    const bool table = shape.kernel == DES3_KERNEL_SPTABLE;
    std::vector<BatchTileJob> hj(njobs);
    batch_fill_jobs(jobs, njobs, hj.data(), table ? kSegBlocks : kTileBlocks);
    // Only the keys that jobs name are expanded and uploaded, renumbered in
    // order of first use: a call over a large key table pays for the keys it
    // uses, not for the table.
    std::vector<uint32_t> slot(nkeys, UINT32_MAX);
    std::vector<des3_ks_t> used;
    for (uint32_t i = 0; i < njobs; i++) {
        uint32_t& sl = slot[jobs[i].key_index];
        if (sl == UINT32_MAX) {
            sl = (uint32_t)used.size();
            used.push_back(keys[jobs[i].key_index]);
        }
        hj[i].key_index = sl;
    }
    const uint32_t nused = (uint32_t)used.size();
    std::vector<uint32_t> hk((size_t)nused * 2 * (table ? kSpKeyStride : kKeyBitsStride));
    if (table) batch_fill_spkeys(used.data(), nused, hk.data());
    else batch_fill_keys(used.data(), nused, hk.data());
    const size_t jbytes = (sizeof(BatchTileJob) * njobs + 255) / 256 * 256;
    const size_t kbytes = hk.size() * sizeof(uint32_t);
    void* d = nullptr;
    cudaError_t e = cudaMallocAsync(&d, jbytes + kbytes, s);
    if (e == cudaErrorMemoryAllocation) return DES3_ENOMEM;
    if (e != cudaSuccess) return cuda_fail(e);
    BatchTileJob* dj = static_cast<BatchTileJob*>(d);
    uint32_t* dk = reinterpret_cast<uint32_t*>(static_cast<char*>(d) + jbytes);
    if ((e = cudaMemcpyAsync(dj, hj.data(), sizeof(BatchTileJob) * njobs, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dk, hk.data(), kbytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        cudaFreeAsync(d, s);
        return cuda_fail(e);
    }
    // Copies from pageable host memory are staged before cudaMemcpyAsync
    // returns, so the host vector may die when this call returns.
    if (table) {
        rc = batch_prepare_sptable();
        if (rc == DES3_OK)
            rc = launch_batch_sptable(dj, njobs, dk, batch_units(jobs, njobs, kSegBlocks), shape.ctas_per_sm,
                                      shape.threads, s);
    } else {
        rc = batch_prepare();
        if (rc == DES3_OK) rc = launch_batch(dj, njobs, dk, ntiles, shape.ctas_per_sm, shape.threads, s);
    }
    e = cudaFreeAsync(d, s);
    if (rc != DES3_OK) return rc;
    return e == cudaSuccess ? DES3_OK : cuda_fail(e);
}

int des3_batch_plan_create(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs, uint32_t njobs, int kernel,
                           des3_batch_plan_t** plan) {
    if (!plan) return DES3_EINVAL;
    *plan = nullptr;
    if (kernel != DES3_KERNEL_AUTO && kernel != DES3_KERNEL_BITSLICE && kernel != DES3_KERNEL_SPTABLE)
        return DES3_EINVAL;
    int rc = check_keys(keys, nkeys);
    if (rc != DES3_OK) return rc;
    uint64_t ntiles = 0, total = 0;
    if ((rc = batch_validate(jobs, njobs, nkeys, &ntiles, &total)) != DES3_OK) return rc;
    DeviceInfo di;
    if ((rc = current_device_info(&di)) != DES3_OK) return rc;
    des3_batch_plan* p = new des3_batch_plan();
    p->device = di.device;
    p->njobs = njobs;
    p->ntiles = ntiles;
    p->total_bytes = total;
    const BatchShape shape = choose_batch_shape(jobs, njobs, ntiles, total, kernel, di.sms);
    p->shape = shape;
    const bool table = shape.kernel == DES3_KERNEL_SPTABLE;
    std::vector<BatchTileJob> hj(njobs);
    batch_fill_jobs(jobs, njobs, hj.data(), table ? kSegBlocks : kTileBlocks);
    std::vector<uint32_t> hk((size_t)nkeys * 2 * (table ? kSpKeyStride : kKeyBitsStride));
    if (table) batch_fill_spkeys(keys, nkeys, hk.data());
    else batch_fill_keys(keys, nkeys, hk.data());
    const size_t jbytes = (sizeof(BatchTileJob) * njobs + 255) / 256 * 256;
    const size_t kbytes = hk.size() * sizeof(uint32_t);
    cudaError_t e = cudaSuccess;
    cudaStream_t cs = nullptr;
    auto fail = [&](int code) {
        if (cs) cudaStreamDestroy(cs);
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        if (p->d_mem) cudaFree(p->d_mem);
        delete p;
        return code;
    };
    if (jbytes + kbytes > 0) {
        e = cudaMalloc(&p->d_mem, jbytes + kbytes);
        if (e == cudaErrorMemoryAllocation) return fail(DES3_ENOMEM);
        if (e != cudaSuccess) return fail(cuda_fail(e));
        if ((e = cudaMemcpy(p->d_mem, hj.data(), sizeof(BatchTileJob) * njobs, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(cuda_fail(e));
        if (kbytes && (e = cudaMemcpy(static_cast<char*>(p->d_mem) + jbytes, hk.data(), kbytes, cudaMemcpyHostToDevice)) !=
                          cudaSuccess)
            return fail(cuda_fail(e));
    }
    if ((rc = table ? batch_prepare_sptable() : batch_prepare()) != DES3_OK) return fail(rc);
    // capture the launch into a graph on a private stream
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return fail(cuda_fail(e));
    const BatchTileJob* dj = static_cast<BatchTileJob*>(p->d_mem);
    const uint32_t* dk = reinterpret_cast<const uint32_t*>(static_cast<char*>(p->d_mem) + jbytes);
    rc = table ? launch_batch_sptable(dj, njobs, dk, batch_units(jobs, njobs, kSegBlocks), shape.ctas_per_sm,
                                      shape.threads, cs)
               : launch_batch(dj, njobs, dk, ntiles, shape.ctas_per_sm, shape.threads, cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (rc != DES3_OK) return fail(rc);
    if (e != cudaSuccess) return fail(cuda_fail(e));
    if ((e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess) return fail(cuda_fail(e));
    cudaStreamDestroy(cs);
    *plan = p;
    return DES3_OK;
}

int des3_batch_plan_launch(des3_batch_plan_t* plan, des3_stream_t stream) {
    if (!plan || !plan->exec) return DES3_EINVAL;
    cudaError_t e = cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? DES3_OK : cuda_fail(e);
}

int des3_batch_plan_info(const des3_batch_plan_t* plan, uint64_t* total_bytes, uint64_t* tiles) {
    if (!plan) return DES3_EINVAL;
    if (total_bytes) *total_bytes = plan->total_bytes;
    if (tiles) *tiles = plan->ntiles;
    return DES3_OK;
}

int des3_batch_choose(const des3_job_t* jobs, uint32_t njobs, uint32_t sms, int* kernel, uint32_t* threads,
                      uint32_t* ctas_per_sm) {
    if ((njobs && !jobs) || sms == 0 || sms > 4096) return DES3_EINVAL;
    uint64_t tiles = 0, total = 0;
    for (uint32_t i = 0; i < njobs; i++) {
        if (jobs[i].nbytes % 8) return DES3_EINVAL;
        tiles += (jobs[i].nbytes / 8 + kTileBlocks - 1) / kTileBlocks;
        total += jobs[i].nbytes;
    }
    const BatchShape shape = choose_batch_shape(jobs, njobs, tiles, total, DES3_KERNEL_AUTO, (int)sms);
    if (kernel) *kernel = shape.kernel;
    if (threads) *threads = (uint32_t)shape.threads;
    if (ctas_per_sm) *ctas_per_sm = (uint32_t)shape.ctas_per_sm;
    return DES3_OK;
}

int des3_batch_plan_kernel(const des3_batch_plan_t* plan, int* kernel, uint32_t* threads, uint32_t* ctas_per_sm) {
    if (!plan) return DES3_EINVAL;
    if (kernel) *kernel = plan->shape.kernel;
    if (threads) *threads = (uint32_t)plan->shape.threads;
    if (ctas_per_sm) *ctas_per_sm = (uint32_t)plan->shape.ctas_per_sm;
    return DES3_OK;
}

int des3_batch_plan_destroy(des3_batch_plan_t* plan) {
    if (!plan) return DES3_OK;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    if (plan->d_mem) cudaFree(plan->d_mem);
    delete plan;
    return DES3_OK;
}

}  // extern "C"
