// tuning.h -- launch-shape and kernel choices per size class.
#pragma once

#include <cstddef>
#include <cstdint>

#include "internal.h"

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

// Kernel and launch shape of a batch.  With allow_table false (the
// allocation-free call, whose key scratch only holds the bitsliced kernel's
// masks) a table-kernel entry gives way to the bitsliced default.
struct BatchShape {
    int ctas_per_sm;
    int threads;
    int kernel;  // DES3_KERNEL_BITSLICE or DES3_KERNEL_SPTABLE
};
BatchShape tuned_batch_shape(uint64_t total_bytes, uint32_t njobs, bool allow_table = false);
constexpr BatchShape kBitsliceBatchDefault{1, kBsThreadsPerSm, DES3_KERNEL_BITSLICE};
constexpr BatchShape kTableBatchDefault{3, 384, DES3_KERNEL_SPTABLE};

// Whether the batched table kernel is predicted faster than the bitsliced
// batch, both in their default shapes, for a batch of `ntiles` 1024-block
// tiles and `nsegs` 64-block segments on `sms` SMs.  The bitsliced batch pays
// for whole tiles, so a batch of jobs far below a tile does 1024 blocks of
// work per job; the table kernel pays per 64-block segment at a lower rate.
// Both times are counted in waves (one unit for every warp the grid holds)
// with per-wave costs measured on GB300; below one bitsliced wave the launch
// shape matters more than the kernel and the answer is false (the tuning
// table decides there).
bool batch_prefers_table(uint64_t ntiles, uint64_t nsegs, int sms);

// The automatic choice for a batch of `total_bytes` in `njobs` jobs,
// `ntiles` 1024-block tiles and `nsegs` 64-block segments on `sms` SMs: the
// tuning table's entry for the size class, except that a bitsliced entry
// gives way to the table kernel's default shape where batch_prefers_table.
BatchShape auto_batch_shape(uint64_t total_bytes, uint32_t njobs, uint64_t ntiles, uint64_t nsegs, int sms);

// Chunk size of the host-memory pipeline (bytes, a multiple of 8 KiB).
size_t tuned_host_chunk();

// Resource limits of each kernel, shared by the launchers and des3_tune_set.
bool shape_fits(int table, int kernel, int threads, int ctas_per_sm);

}  // namespace des3
