// probe.cu -- des3_pipe_probe: throughput of the pipes the cipher kernels are
// bound by, on the current device, for roofline accounting.
//
// One launch puts 8 CTAs of 256 threads on every SM; each thread runs 8
// independent chains of `iters` x 16 instructions of one kind:
//   kind 0  lop3.b32            (integer ALU pipe: the bitsliced S-box gates)
//   kind 1  mad.lo.u32          (FMA pipe: key corrections, table addresses)
//   kind 2  lop3 and mad, 1:1
//   kind 3  ld.shared.u32       (shared-memory pipe: the SP-table lookups),
//           each lane walking its own bank, so a warp's load is one
//           conflict-free access
// Eight chains per thread and 64 warps per SM hide every latency, so the
// launch runs at the pipe's issue rate.  Thread 0 of CTA 0 records its SM
// clock cycles and global-timer nanoseconds between its first and last probe
// instruction, which gives the clock the probe ran at.
#include "internal.h"

namespace des3 {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;
constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;
constexpr int kProbeRows = 128;  // shared-memory rows of the load chains (128 x 32 words)

__device__ __forceinline__ uint32_t p_lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t p_mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}

__device__ __forceinline__ uint32_t p_lds(uint32_t addr) {
    uint32_t d;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(d) : "r"(addr));
    return d;
}

__device__ __forceinline__ uint64_t p_gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads, kProbeCtasPerSm)
    pipe_probe_kernel(uint32_t iters, unsigned long long* sink) {
    __shared__ uint32_t rows[kProbeRows * 32];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(rows);
    if (KIND == 3) {
        // row i of lane l holds the address of row (5 i + 1) mod 128 of lane l:
        // a cycle through all rows of the lane's own bank
        for (uint32_t i = threadIdx.x >> 5; i < kProbeRows; i += kProbeThreads / 32)
            rows[i * 32 + lane] = base + (((5 * i + 1) % kProbeRows) * 32 + lane) * 4;
        __syncthreads();
    }
    uint32_t a[kProbeChains];
#pragma unroll
    for (int i = 0; i < kProbeChains; i++)
        a[i] = KIND == 3 ? base + ((uint32_t)(16 * i) * 32 + lane) * 4 : threadIdx.x * (i + 3) + blockIdx.x;
    const uint64_t c0 = clock64(), t0 = p_gtimer();
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; u++) {
#pragma unroll
            for (int i = 0; i < kProbeChains; i++) {
                const uint32_t b = a[(i + 1) & 7], c = a[(i + 2) & 7];
                if (KIND == 0) a[i] = p_lop3(a[i], b, c);
                else if (KIND == 1) a[i] = p_mad(a[i], b, c);
                else if (KIND == 2) a[i] = (i & 1) ? p_mad(a[i], b, c) : p_lop3(a[i], b, c);
                else a[i] = p_lds(a[i]);
            }
        }
    }
    const uint64_t c1 = clock64(), t1 = p_gtimer();
    uint32_t r = 0;
#pragma unroll
    for (int i = 0; i < kProbeChains; i++) r ^= a[i];
    r = __reduce_xor_sync(0xFFFFFFFFu, r);
    if (lane == 0) atomicXor(sink, (unsigned long long)r);
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        sink[1] = c1 - c0;
        sink[2] = t1 - t0;
    }
}

}  // namespace
}  // namespace des3

using namespace des3;

extern "C" int des3_pipe_probe(int kind, uint32_t iters, void* d_sink, uint64_t* instructions, uint32_t* sms,
                               des3_stream_t stream) {
    if (kind < 0 || kind > 3 || iters == 0 || !d_sink || !instructions || !sms) return DES3_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_sink) & 7) return DES3_EINVAL;
    DeviceInfo di;
    int rc = current_device_info(&di);
    if (rc != DES3_OK) return rc;
    const unsigned grid = (unsigned)di.sms * kProbeCtasPerSm;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    auto* sink = static_cast<unsigned long long*>(d_sink);
    switch (kind) {
        case 0: pipe_probe_kernel<0><<<grid, kProbeThreads, 0, s>>>(iters, sink); break;
        case 1: pipe_probe_kernel<1><<<grid, kProbeThreads, 0, s>>>(iters, sink); break;
        case 2: pipe_probe_kernel<2><<<grid, kProbeThreads, 0, s>>>(iters, sink); break;
        default: pipe_probe_kernel<3><<<grid, kProbeThreads, 0, s>>>(iters, sink); break;
    }
    *instructions = (uint64_t)grid * kProbeThreads * kProbeChains * kProbeUnroll * iters;
    *sms = (uint32_t)di.sms;
    return check_launch();
}
