// tuning.h -- launch-shape and kernel choices per size class.
#pragma once

#include <cstddef>
#include <cstdint>

namespace des3 {

// Kernel the AUTO setting uses for a single buffer of `nblocks` blocks.
int tuned_kernel(uint64_t nblocks);

// Launch shape of the persistent batched kernel.
struct BatchShape {
    int ctas_per_sm;
    int threads;
};
BatchShape tuned_batch_shape(uint64_t total_bytes, uint32_t njobs);

// Chunk size of the host-memory pipeline (bytes, a multiple of 8 KiB).
size_t tuned_host_chunk();

}  // namespace des3
