// tuning.h -- launch-shape and kernel choices per size class.
#pragma once

#include <cstddef>
#include <cstdint>

namespace des3 {

struct LaunchShape {
    int kernel;  // DES3_KERNEL_BITSLICE or DES3_KERNEL_SPTABLE
    int threads;
    int ctas_per_sm;
};

// Shape of a single-buffer call of `nbytes`; `kernel` is the caller's
// request (AUTO lets the table choose; an explicit kernel keeps the table's
// shape when it names the same kernel, else that kernel's default shape).
LaunchShape tuned_single(uint64_t nbytes, int kernel);

// Launch shape of the persistent batched kernel.
struct BatchShape {
    int ctas_per_sm;
    int threads;
};
BatchShape tuned_batch_shape(uint64_t total_bytes, uint32_t njobs);

// Chunk size of the host-memory pipeline (bytes, a multiple of 8 KiB).
size_t tuned_host_chunk();

// Resource limits of each kernel, shared by the launchers and des3_tune_set.
bool shape_fits(int table, int kernel, int threads, int ctas_per_sm);

}  // namespace des3
