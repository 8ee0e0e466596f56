// host_pipe.cu -- des3_ecb_host: 3DES-EDE ECB of a HOST buffer through a
// device workspace, with the transfers overlapped with the cipher.
//
// The paper copies the whole file to the device once, runs every kernel, and
// copies it back (Sec. II.B), and it leaves the transfer time out of its
// measurements (Sec. III).  Here the buffer is cut into chunks that cycle
// through NBUF slots of the workspace on NBUF private streams: chunk i is
// copied in on stream i % NBUF, transformed there and copied back out, so
// the host-to-device copy of one chunk, the kernel of another and the
// device-to-host copy of a third run at the same time.  The caller's stream
// is joined at both ends with events, so the call is ordered and
// asynchronous like the device calls.
#include <mutex>

#include "internal.h"
#include "tuning.h"

namespace des3 {
namespace {

constexpr int kSlots = 3;
constexpr size_t kMinWork = 2u << 20;
constexpr size_t kRampBytes = 4u << 20;  // first and last chunk sizes

struct PipeStreams {
    bool ready = false;
    cudaStream_t s[kSlots];
};

std::mutex g_pipe_mu;
PipeStreams g_pipe[64];

int pipe_streams(int dev, cudaStream_t* out) {
    std::lock_guard<std::mutex> g(g_pipe_mu);
    if (dev < 0 || dev >= 64) return DES3_ENODEV;
    PipeStreams& p = g_pipe[dev];
    if (!p.ready) {
        for (int i = 0; i < kSlots; i++) {
            cudaError_t e = cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking);
            if (e != cudaSuccess) {
                for (int k = 0; k < i; k++) cudaStreamDestroy(p.s[k]);
                return cuda_fail(e);
            }
        }
        p.ready = true;
    }
    for (int i = 0; i < kSlots; i++) out[i] = p.s[i];
    return DES3_OK;
}

// Bytes of chunk i when `left` bytes remain.  The first chunks grow from
// kRampBytes to the slot size and the last ones shrink back, so the copy in
// before the first kernel and the copy out after the last one, which run
// alone, are short.  Every chunk but the last is a multiple of 8 KiB (one
// bitsliced tile).
size_t chunk_size(size_t i, size_t left, size_t slot) {
    size_t c = slot;
    if (i < 8 && (kRampBytes << i) < c) c = kRampBytes << i;  // ramp up: 4, 8, 16, ... MiB
    if (left > kRampBytes) {  // ramp down: never more than half of what is left
        size_t half = (left / 2) & ~(size_t)8191;
        if (half < kRampBytes) half = kRampBytes;
        if (half < c) c = half;
    }
    return c < left ? c : left;
}

}  // namespace
}  // namespace des3

using namespace des3;

extern "C" int des3_ecb_host(const des3_ks_t* ks, const void* h_in, void* h_out, size_t nbytes, int decrypt,
                             void* d_work, size_t work_bytes, des3_stream_t stream) {
    if (!ks || ((!h_in || !h_out) && nbytes)) return DES3_EINVAL;
    if (ks->magic != DES3_KS_MAGIC) return DES3_EKEY;
    if (nbytes % 8 || (decrypt != 0 && decrypt != 1)) return DES3_EINVAL;
    if (nbytes == 0) return DES3_OK;
    if (!d_work || work_bytes < kMinWork || (reinterpret_cast<uintptr_t>(d_work) & 255)) return DES3_EINVAL;
    if (h_in != h_out) {
        const uintptr_t x = reinterpret_cast<uintptr_t>(h_in), y = reinterpret_cast<uintptr_t>(h_out);
        if (x < y + nbytes && y < x + nbytes) return DES3_EINVAL;
    }
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    cudaStream_t ps[kSlots];
    if ((rc = pipe_streams(di.device, ps)) != DES3_OK) return rc;
    cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);

    // slot size: a multiple of 8 KiB (one bitsliced tile) and of 256 bytes
    size_t chunk = (work_bytes / kSlots) & ~(size_t)8191;
    const size_t want = tuned_host_chunk();
    if (chunk > want) chunk = want;
    if (chunk == 0) return DES3_EINVAL;

    cudaError_t e;
    cudaEvent_t start, done[kSlots];
    if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess) return cuda_fail(e);
    int made = 0;
    for (; made < kSlots; made++)
        if ((e = cudaEventCreateWithFlags(&done[made], cudaEventDisableTiming)) != cudaSuccess) break;
    auto cleanup = [&]() {
        cudaEventDestroy(start);
        for (int i = 0; i < made; i++) cudaEventDestroy(done[i]);
    };
    if (made < kSlots) {
        cleanup();
        return cuda_fail(e);
    }
    rc = DES3_OK;
    // everything starts after the work already queued on the caller's stream
    if ((e = cudaEventRecord(start, user)) != cudaSuccess) rc = cuda_fail(e);
    for (int i = 0; rc == DES3_OK && i < kSlots; i++)
        if ((e = cudaStreamWaitEvent(ps[i], start, 0)) != cudaSuccess) rc = cuda_fail(e);
    const uint64_t* rk = ks->rk[decrypt];
    const char* src = static_cast<const char*>(h_in);
    char* dst = static_cast<char*>(h_out);
    size_t off = 0;
    for (size_t i = 0; rc == DES3_OK && off < nbytes; i++) {
        const int slot = (int)(i % kSlots);
        const size_t n = chunk_size(i, nbytes - off, chunk);
        uint8_t* d = static_cast<uint8_t*>(d_work) + slot * chunk;
        cudaStream_t s = ps[slot];
        if ((e = cudaMemcpyAsync(d, src + off, n, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
            rc = cuda_fail(e);
            break;
        }
        rc = launch_single(rk, d, d, n / 8, DES3_KERNEL_AUTO, s, ks_rounds(ks));
        if (rc != DES3_OK) break;
        if ((e = cudaMemcpyAsync(dst + off, d, n, cudaMemcpyDeviceToHost, s)) != cudaSuccess) rc = cuda_fail(e);
        off += n;
    }
    // the caller's stream continues only when every slot has drained
    for (int i = 0; i < kSlots; i++) {
        if ((e = cudaEventRecord(done[i], ps[i])) != cudaSuccess) {
            if (rc == DES3_OK) rc = cuda_fail(e);
            continue;
        }
        if ((e = cudaStreamWaitEvent(user, done[i], 0)) != cudaSuccess && rc == DES3_OK) rc = cuda_fail(e);
    }
    cleanup();  // destruction is deferred by CUDA until the events complete
    return rc;
}
