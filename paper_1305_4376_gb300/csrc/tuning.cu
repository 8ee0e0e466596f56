// tuning.cu -- size-class tables for DES3_KERNEL_AUTO and the batched calls.
//
// Defaults: the bitsliced kernel works on whole 1024-block tiles per warp, so
// below a few tiles per SM it leaves the GPU idle, and the table kernel (one
// block per thread, 32x more threads for the same bytes) wins; above that
// the bitsliced kernel wins by its lower instruction count.  The autotuner
// replaces these guesses with measured choices (des3_tune_set).
#include <mutex>

#include "common.cuh"
#include "des3.h"
#include "internal.h"
#include "tuning.h"

namespace des3 {

namespace {

std::mutex g_mu;
des3_tune_entry_t g_tab[2][DES3_TUNE_CLASSES];
bool g_init = false;

// The built-in tables are the autotuner's GB300 choices (the library runs on
// sm_103a only), each size class taking the nearest measured class's entry;
// a CPU test keeps them equal to the committed tuning file.
void defaults_locked() {
    auto set = [](des3_tune_entry_t& e, uint32_t c, int kernel, uint32_t threads, uint32_t ctas) {
        e.size_class = c;
        e.kernel = kernel;
        e.threads = threads;
        e.ctas_per_sm = ctas;
    };
    for (uint32_t c = 0; c < DES3_TUNE_CLASSES; c++) {
        des3_tune_entry_t& e = g_tab[DES3_TUNE_SINGLE][c];
        if (c <= 13) set(e, c, DES3_KERNEL_SPTABLE, 256, 3);         // up to 4 KiB
        else if (c <= 15) set(e, c, DES3_KERNEL_SPTABLE, 128, 2);    // 16 KiB
        else if (c <= 19) set(e, c, DES3_KERNEL_SPTABLE, 256, 3);    // 64 and 256 KiB
        else if (c <= 21) set(e, c, DES3_KERNEL_SPTABLE, 384, 3);    // 1 MiB
        else if (c <= 23) set(e, c, DES3_KERNEL_BITSLICE, 384, 1);   // 4 MiB
        else if (c <= 25) set(e, c, DES3_KERNEL_BITSLICE, 256, 1);   // 16 MiB
        else set(e, c, DES3_KERNEL_BITSLICE, kBsThreadsPerSm, 1);     // 64 MiB and more
        des3_tune_entry_t& b = g_tab[DES3_TUNE_BATCH][c];
        if (c <= 17) set(b, c, DES3_KERNEL_SPTABLE, 128, 3);         // 64 KiB in all
        else if (c <= 21) set(b, c, DES3_KERNEL_SPTABLE, 256, 3);    // 256 KiB to 1 MiB
        else if (c <= 23) set(b, c, DES3_KERNEL_BITSLICE, kBsThreadsPerSm, 1);  // 4 MiB
        else if (c <= 25) set(b, c, DES3_KERNEL_BITSLICE, 256, 1);   // 16 MiB
        else set(b, c, DES3_KERNEL_BITSLICE, kBsThreadsPerSm, 1);     // 64 MiB and more
    }
    g_init = true;
}

uint32_t size_class(uint64_t bytes) {
    uint32_t c = 0;
    while (c + 1 < DES3_TUNE_CLASSES && (bytes >> (c + 1)) != 0) c++;
    return c;
}

des3_tune_entry_t lookup(int table, uint64_t bytes) {
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_init) defaults_locked();
    return g_tab[table][size_class(bytes)];
}

}  // namespace

bool shape_fits(int table, int kernel, int threads, int ctas) {
    if (threads != 64 && threads != 128 && threads != 256 && threads != 384) return false;
    if (ctas < 1 || ctas > 8) return false;
    // the bitsliced kernels are compiled for kBsThreadsPerSm threads per SM
    // (up to 168 registers each), so at most that many of them fit on an SM
    if (table == DES3_TUNE_BATCH) {
        if (kernel == DES3_KERNEL_SPTABLE)  // 64.4 KiB of tables and keys plus 384 B of round keys per warp
            return ctas <= 3 && (65536 + 384 + (threads / 32) * 384) * ctas <= 227 * 1024;
        return kernel == DES3_KERNEL_BITSLICE && threads * ctas <= kBsThreadsPerSm &&
               (threads / 32) * kBsMaskWords * 4 * ctas <= 227 * 1024;  // kBsMaskWords key masks per warp
    }
    if (kernel == DES3_KERNEL_BITSLICE) return threads * ctas <= kBsThreadsPerSm;
    if (kernel == DES3_KERNEL_SPTABLE) return ctas <= 3;  // 64.4 KiB of tables and keys per CTA
    return false;
}

LaunchShape tuned_single(uint64_t nbytes, int kernel) {
    const des3_tune_entry_t e = lookup(DES3_TUNE_SINGLE, nbytes);
    if (kernel == DES3_KERNEL_AUTO || kernel == e.kernel) return LaunchShape{e.kernel, (int)e.threads, (int)e.ctas_per_sm};
    if (kernel == DES3_KERNEL_SPTABLE) return LaunchShape{DES3_KERNEL_SPTABLE, 384, 3};
    return LaunchShape{DES3_KERNEL_BITSLICE, kBsThreadsPerSm, 1};
}

BatchShape tuned_batch_shape(uint64_t total_bytes, uint32_t njobs, bool allow_table) {
    (void)njobs;
    const des3_tune_entry_t e = lookup(DES3_TUNE_BATCH, total_bytes);
    if (e.kernel == DES3_KERNEL_SPTABLE && !allow_table) return kBitsliceBatchDefault;
    return BatchShape{(int)e.ctas_per_sm, (int)e.threads, (int)e.kernel};
}

// Wave model of the two batched kernels, fitted on GB300 to graph-replayed
// batches of 4096 and 32768 equal jobs of 64 to 2248 blocks (fill of the
// last tile 6 % to 100 %, 1 to 216 waves): the bitsliced batch (384 x 1,
// 12 warps per SM) took 10 + 39.2 us per wave of tiles to within 5 %, the
// table kernel (384 x 3, 36 warps per SM) 6.3 + 18.0 us per wave of
// segments to within 2 %.  Waves count whole because every warp takes an
// equal contiguous share and the slowest warp ends the launch.
bool batch_prefers_table(uint64_t ntiles, uint64_t nsegs, int sms) {
    const uint64_t bs_warps = (uint64_t)sms * (kBitsliceBatchDefault.threads / 32) * kBitsliceBatchDefault.ctas_per_sm;
    const uint64_t sp_warps = (uint64_t)sms * (kTableBatchDefault.threads / 32) * kTableBatchDefault.ctas_per_sm;
    if (sms <= 0 || ntiles < bs_warps) return false;
    const double t_bs = 10.0 + 39.2 * (double)((ntiles + bs_warps - 1) / bs_warps);
    const double t_sp = 6.3 + 18.0 * (double)((nsegs + sp_warps - 1) / sp_warps);
    return t_sp < t_bs;
}

BatchShape auto_batch_shape(uint64_t total_bytes, uint32_t njobs, uint64_t ntiles, uint64_t nsegs, int sms) {
    const BatchShape shape = tuned_batch_shape(total_bytes, njobs, true);
    if (shape.kernel == DES3_KERNEL_BITSLICE && batch_prefers_table(ntiles, nsegs, sms)) return kTableBatchDefault;
    return shape;
}

size_t tuned_host_chunk() { return 64u << 20; }

}  // namespace des3

using namespace des3;

extern "C" {

int des3_tune_set(int table, const des3_tune_entry_t* entries, uint32_t n) {
    if (table != DES3_TUNE_SINGLE && table != DES3_TUNE_BATCH) return DES3_EINVAL;
    if (n && !entries) return DES3_EINVAL;
    for (uint32_t i = 0; i < n; i++) {
        const des3_tune_entry_t& e = entries[i];
        if (e.size_class >= DES3_TUNE_CLASSES) return DES3_EINVAL;
        if (!shape_fits(table, e.kernel, (int)e.threads, (int)e.ctas_per_sm)) return DES3_EINVAL;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_init) defaults_locked();
    for (uint32_t i = 0; i < n; i++) g_tab[table][entries[i].size_class] = entries[i];
    return DES3_OK;
}

int des3_tune_get(int table, uint32_t size_class_, des3_tune_entry_t* out) {
    if ((table != DES3_TUNE_SINGLE && table != DES3_TUNE_BATCH) || size_class_ >= DES3_TUNE_CLASSES || !out)
        return DES3_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_init) defaults_locked();
    *out = g_tab[table][size_class_];
    return DES3_OK;
}

int des3_tune_reset(void) {
    std::lock_guard<std::mutex> g(g_mu);
    defaults_locked();
    return DES3_OK;
}

}  // extern "C"
