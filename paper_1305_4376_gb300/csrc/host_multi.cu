// host_multi.cu -- des3_ecb_host_multi: one host buffer split into contiguous
// block ranges, each range streamed through its own device by des3_ecb_host.
//
// The paper notes (Sec. III) that a second graphics card could raise the
// throughput, at the cost of dividing the work between the cards.  In ECB
// every 64-bit block is processed on its own (abstract), so the division is
// a split of the block index range with no exchange at all: no device reads
// another's memory, there is no peer access and no collective.  The host
// link of each device carries only its own range, which is what the host
// pipeline is bound by.
#include <cuda_runtime.h>

#include <thread>
#include <vector>  // std::thread and std::vector may throw; nothing escapes the C ABI

#include "internal.h"

using namespace des3;

extern "C" int des3_range_split(uint64_t nblocks, uint32_t nparts, uint64_t granule, uint64_t* first) {
    if (nparts == 0 || granule == 0 || !first) return DES3_EINVAL;
    const uint64_t units = nblocks / granule + (nblocks % granule ? 1 : 0);
    const uint64_t base = units / nparts, extra = units % nparts;
    for (uint32_t i = 0; i <= nparts; i++) {
        const uint64_t u = (uint64_t)i * base + (i < extra ? i : extra);
        const uint64_t b = u * granule;
        first[i] = b < nblocks ? b : nblocks;
    }
    return DES3_OK;
}

extern "C" int des3_ecb_host_multi(const des3_ks_t* ks, const void* h_in, void* h_out, size_t nbytes, int decrypt,
                                   uint32_t ndev, const int* devices, void* const* d_work,
                                   const size_t* work_bytes) {
    if (!ks || ((!h_in || !h_out) && nbytes)) return DES3_EINVAL;
    if (ks->magic != DES3_KS_MAGIC) return DES3_EKEY;
    if (nbytes % 8 || (decrypt != 0 && decrypt != 1)) return DES3_EINVAL;
    if (ndev == 0 || ndev > 64 || !devices || !d_work || !work_bytes) return DES3_EINVAL;
    if (nbytes == 0) return DES3_OK;
    if (h_in != h_out) {
        const uintptr_t x = reinterpret_cast<uintptr_t>(h_in), y = reinterpret_cast<uintptr_t>(h_out);
        if (x < y + nbytes && y < x + nbytes) return DES3_EINVAL;
    }
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return e == cudaErrorNoDevice ? DES3_ENODEV : cuda_fail(e);
    std::vector<uint64_t> first(ndev + 1);
    des3_range_split(nbytes / 8, ndev, kTileBlocks, first.data());
    for (uint32_t i = 0; i < ndev; i++) {
        if (devices[i] < 0 || devices[i] >= count) return DES3_ENODEV;
        if (first[i + 1] == first[i]) continue;  // an empty range needs no workspace
        if (!d_work[i]) return DES3_EINVAL;
        for (uint32_t j = 0; j < i; j++)  // two ranges in flight in one workspace would race
            if (first[j + 1] > first[j] && d_work[j] == d_work[i]) return DES3_EINVAL;
    }
    // one host thread per range: each makes its device current, runs the
    // pipeline on a stream of its own and waits for it, so the ranges run at
    // the same time even when the host memory is pageable (whose copies the
    // runtime stages synchronously)
    std::vector<int> rc(ndev, DES3_OK);
    std::vector<int> cuda_err(ndev, 0);  // a worker's CUDA error, for the caller's des3_last_cuda_error
    std::vector<std::thread> workers;
    const char* src = static_cast<const char*>(h_in);
    char* dst = static_cast<char*>(h_out);
    for (uint32_t i = 0; i < ndev; i++) {
        const uint64_t b0 = first[i], b1 = first[i + 1];
        if (b1 == b0) continue;
        auto work = [&, i, b0, b1] {
            cudaError_t err = cudaSetDevice(devices[i]);
            cudaStream_t st = nullptr;
            if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (err != cudaSuccess) {
                rc[i] = DES3_ECUDA;
                cuda_err[i] = (int)err;
                return;
            }
            int r = des3_ecb_host(ks, src + 8 * b0, dst + 8 * b0, 8 * (b1 - b0), decrypt, d_work[i], work_bytes[i],
                                  reinterpret_cast<des3_stream_t>(st));
            err = cudaStreamSynchronize(st);
            if (r == DES3_OK && err != cudaSuccess) r = cuda_fail(err);
            cudaStreamDestroy(st);
            rc[i] = r;
            cuda_err[i] = des3_last_cuda_error();
        };
        try {
            workers.emplace_back(work);
        } catch (...) {  // no thread to be had: this range fails, the others finish
            rc[i] = DES3_ENOMEM;
        }
    }
    for (std::thread& t : workers) t.join();
    for (uint32_t i = 0; i < ndev; i++) {
        if (rc[i] == DES3_ECUDA) return cuda_fail((cudaError_t)cuda_err[i]);
        if (rc[i] != DES3_OK) return rc[i];
    }
    return DES3_OK;
}
