// tuning.cu -- size-class table for DES3_KERNEL_AUTO.
//
// The bitsliced kernel works on whole 1024-block tiles per warp, so below a
// few tiles it leaves most of the GPU idle; the table kernel spreads the same
// blocks over 32x more threads.  The threshold is the measured crossover.
#include "des3.h"
#include "tuning.h"

namespace des3 {

namespace {
uint64_t g_bitslice_min_blocks = 1u << 13;  // 64 KiB
}  // namespace

int tuned_kernel(uint64_t nblocks) {
    return nblocks >= g_bitslice_min_blocks ? DES3_KERNEL_BITSLICE : DES3_KERNEL_SPTABLE;
}

BatchShape tuned_batch_shape(uint64_t total_bytes, uint32_t njobs) {
    (void)total_bytes;
    (void)njobs;
    return BatchShape{2, 256};
}

size_t tuned_host_chunk() { return 64u << 20; }

}  // namespace des3
