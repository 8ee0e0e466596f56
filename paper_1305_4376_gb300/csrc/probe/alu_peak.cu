// alu_peak.cu -- throughput of the integer pipes on every SM: LOP3 (ALU
// pipe), IMAD (FMA pipe) and a 1:1 mix.  This is where the ALU roofline of
// the bitsliced kernel comes from (instructions per SM per clock, with the
// SM clock read from clock64 against the global nanosecond timer).
// Measures instructions per SM per clock using clock64 and globaltimer.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t lop(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d; asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}
__device__ __forceinline__ uint32_t mad(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d; asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d;
}
__device__ __forceinline__ uint64_t gtimer() { uint64_t t; asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t)); return t; }

template <int MODE>
__global__ void probe(uint32_t* out, int iters, unsigned long long* cyc, unsigned long long* ns) {
    uint32_t a[8];
    for (int i = 0; i < 8; i++) a[i] = threadIdx.x * (i + 3) + blockIdx.x;
    uint64_t c0 = clock64(), t0 = gtimer();
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++) {
#pragma unroll
            for (int i = 0; i < 8; i++) {
                if (MODE == 0) a[i] = lop(a[i], a[(i + 1) & 7], a[(i + 2) & 7]);
                else if (MODE == 1) a[i] = mad(a[i], a[(i + 1) & 7], a[(i + 2) & 7]);
                else a[i] = (i & 1) ? mad(a[i], a[(i + 1) & 7], a[(i + 2) & 7]) : lop(a[i], a[(i + 1) & 7], a[(i + 2) & 7]);
            }
        }
    }
    uint64_t c1 = clock64(), t1 = gtimer();
    uint32_t r = 0;
    for (int i = 0; i < 8; i++) r ^= a[i];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
    if (threadIdx.x == 0 && blockIdx.x == 0) { *cyc = c1 - c0; *ns = t1 - t0; }
}

int main() {
    int sms = 0; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    cudaDeviceProp prop; cudaGetDeviceProperties(&prop, 0);
    printf("device %s sms %d cc %d.%d\n", prop.name, sms, prop.major, prop.minor);
    const int threads = 256, ctas = sms * 8, iters = 4000;
    uint32_t* out; cudaMalloc(&out, (size_t)ctas * threads * 4);
    unsigned long long *cyc, *ns; cudaMallocManaged(&cyc, 8); cudaMallocManaged(&ns, 8);
    const char* names[3] = {"lop3", "imad", "lop3+imad 1:1"};
    for (int mode = 0; mode < 3; mode++) {
        for (int rep = 0; rep < 3; rep++) {
            cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
            cudaEventRecord(e0);
            if (mode == 0) probe<0><<<ctas, threads>>>(out, iters, cyc, ns);
            else if (mode == 1) probe<1><<<ctas, threads>>>(out, iters, cyc, ns);
            else probe<2><<<ctas, threads>>>(out, iters, cyc, ns);
            cudaEventRecord(e1); cudaEventSynchronize(e1);
            float ms; cudaEventElapsedTime(&ms, e0, e1);
            double ops = (double)ctas * threads * iters * 16 * 8;
            double mhz = (double)*cyc / (double)*ns * 1e3;
            double per_sm_clk = ops / (ms * 1e-3) / sms / (mhz * 1e6);
            printf("%-14s %.3f ms  %.2f Tops/s  sm clock %.0f MHz  %.1f ops/SM/clk  err=%s\n", names[mode], ms,
                   ops / (ms * 1e-3) / 1e12, mhz, per_sm_clk, cudaGetErrorString(cudaGetLastError()));
        }
    }
    return 0;
}
