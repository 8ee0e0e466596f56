// c2c_peak.cu -- host<->device bandwidth on this machine, by the copy
// engines (cudaMemcpyAsync on 1..4 streams per direction) and by the SMs
// (a kernel that loads and stores pinned host memory through its device
// mapping).  The second is what a kernel working directly on pinned host
// buffers can reach; the first is the ceiling of a staged copy pipeline.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x)                                                                         \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess) {                                                      \
            printf("CUDA error %s at %s:%d\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return 1;                                                                 \
        }                                                                             \
    } while (0)

// dst[i] = src[i] for i < n16 (16-byte words), grid-stride; n16 fits every launch below
__global__ void copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, uint64_t n16) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
}

int main() {
    const size_t n = 1ull << 30;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    int pageable = 0, hostreg = 0;
    cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, 0);
    cudaDeviceGetAttribute(&hostreg, cudaDevAttrCanUseHostPointerForRegisteredMem, 0);
    printf("sms %d pageable_access %d host_pointer_for_registered %d\n", sms, pageable, hostreg);
    uint8_t *h1, *h2, *d1, *d2;
    CK(cudaHostAlloc((void**)&h1, n, cudaHostAllocMapped));
    CK(cudaHostAlloc((void**)&h2, n, cudaHostAllocMapped));
    CK(cudaMalloc((void**)&d1, n));
    CK(cudaMalloc((void**)&d2, n));
    uint8_t *hd1, *hd2;  // device views of the pinned buffers
    CK(cudaHostGetDevicePointer((void**)&hd1, h1, 0));
    CK(cudaHostGetDevicePointer((void**)&hd2, h2, 0));
    for (size_t i = 0; i < n; i += 4096) h1[i] = h2[i] = (uint8_t)i;
    CK(cudaMemset(d1, 1, n));
    CK(cudaMemset(d2, 2, n));
    cudaStream_t st[8];
    for (int i = 0; i < 8; i++) CK(cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = 5;

    // copy engines: k streams per direction, each moving n / k bytes per rep
    for (int mode = 0; mode < 3; mode++) {
        for (int k = 1; k <= 4; k *= 2) {
            CK(cudaDeviceSynchronize());
            CK(cudaEventRecord(e0, 0));
            for (int r = 0; r < reps; r++) {
                for (int j = 0; j < k; j++) {
                    const size_t off = j * (n / k), len = n / k;
                    if (mode == 0 || mode == 2) CK(cudaMemcpyAsync(d1 + off, h1 + off, len, cudaMemcpyHostToDevice, st[j]));
                    if (mode == 1 || mode == 2) CK(cudaMemcpyAsync(h2 + off, d2 + off, len, cudaMemcpyDeviceToHost, st[4 + j]));
                }
            }
            for (int j = 0; j < 8; j++) CK(cudaStreamSynchronize(st[j]));
            CK(cudaEventRecord(e1, 0));
            CK(cudaEventSynchronize(e1));
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            const char* name = mode == 0 ? "copy engine h2d" : mode == 1 ? "copy engine d2h" : "copy engine both, each way";
            printf("%-30s streams %d  %.1f GB/s\n", name, k, reps * (double)n / (ms * 1e-3) / 1e9);
        }
    }

    // SM loads and stores through the device mapping of pinned memory
    const uint64_t n16 = n / 16;
    struct { const char* name; const uint8_t* src; uint8_t* dst; } kc[3] = {
        {"kernel host->device", hd1, d1}, {"kernel device->host", d2, hd2}, {"kernel host->host", hd1, hd2}};
    for (int c = 0; c < 3; c++) {
        for (int per_sm = 4; per_sm <= 16; per_sm *= 2) {
            const int grid = sms * per_sm;
            copy16<<<grid, 256>>>((const uint4*)kc[c].src, (uint4*)kc[c].dst, n16);
            CK(cudaGetLastError());
            CK(cudaDeviceSynchronize());
            CK(cudaEventRecord(e0, 0));
            for (int r = 0; r < reps; r++) copy16<<<grid, 256>>>((const uint4*)kc[c].src, (uint4*)kc[c].dst, n16);
            CK(cudaEventRecord(e1, 0));
            CK(cudaEventSynchronize(e1));
            CK(cudaGetLastError());
            float ms = 0;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            printf("%-30s %2d CTAs/SM  %.1f GB/s (bytes copied; host->host moves each byte over the link twice)\n",
                   kc[c].name, per_sm, reps * (double)n / (ms * 1e-3) / 1e9);
        }
    }
    return 0;
}
