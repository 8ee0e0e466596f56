/*
 * des3.h -- C ABI of the GB300 3DES-EDE ECB library (libdes3gpu.so).
 *
 * The operation follows "3DES ECB Optimized for Massively Parallel CUDA GPU
 * Architecture" (Swierczewski):
 *   - Sec. II.A: 3DES encryption is DES-encrypt with K1, DES-decrypt with K2,
 *     DES-encrypt with K3; decryption is the same steps in reverse
 *     (DES-decrypt K3, DES-encrypt K2, DES-decrypt K1).
 *   - Abstract and Fig. 2: ECB mode; every 64-bit block is processed
 *     independently.
 *   - Listing 1.1 and Sec. II.B: the data is an array of 64-bit blocks
 *     resident in device memory, processed in place with 48 precomputed
 *     round keys (3 keys x 16 rounds) prepared on the host.
 * DES itself (IP, 16 Feistel rounds with E, S1..S8 and P, IP^-1, and the
 * PC-1/PC-2 key schedule) is the standard the paper uses without printing it
 * (FIPS PUB 46-3).
 *
 * Byte order: a block is 8 bytes in memory order and byte 0 holds DES bits
 * 1..8, most significant bit first (the convention of every ECB
 * implementation, e.g. OpenSSL).  Keys are 24 bytes K1||K2||K3; the low bit
 * of every key byte is a parity bit and is ignored.  Two-key 3DES is
 * K1||K2||K1; K1=K2=K3 reduces to single DES.
 *
 * Conventions for every call:
 *   - Return value: DES3_OK (0) or a negative DES3_E* code; no exception or
 *     abort ever crosses this boundary.  des3_strerror() names a code.  When
 *     a CUDA call failed (DES3_ECUDA) des3_last_cuda_error() gives the CUDA
 *     error number of the calling thread's last failure.
 *   - Device calls are asynchronous on the given stream (NULL = legacy
 *     default stream): they return once the work is enqueued.  The caller
 *     synchronises on the stream before reading results or freeing buffers.
 *   - The caller owns every buffer and every des3_ks_t.  Pointers named d_*
 *     are device pointers (cudaMalloc, or anything the device can address);
 *     pointers named h_* are host pointers (pinned memory recommended).
 *   - Sizes are in bytes and must be multiples of 8 (ECB has no padding);
 *     nbytes == 0 is a no-op that returns DES3_OK.
 *   - d_in and d_out must both be 8-byte aligned.  They may be the same
 *     buffer (in place, as in the paper); any other overlap is DES3_EINVAL.
 *   - Calls on distinct streams may run concurrently from several host
 *     threads.
 */
#ifndef DES3_H
#define DES3_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* The CUDA runtime's stream handle type (cudaStream_t / CUstream). */
typedef struct CUstream_st* des3_stream_t;

/* ---- error codes ------------------------------------------------------ */
#define DES3_OK 0
#define DES3_EINVAL -1       /* null pointer, size not a multiple of 8, misalignment, partial overlap, bad flag */
#define DES3_EKEY -2         /* key schedule object not produced by des3_key_schedule */
#define DES3_ECUDA -3        /* a CUDA runtime call failed; see des3_last_cuda_error() */
#define DES3_ETIMEOUT -4     /* a bounded wait on the device gave up */
#define DES3_ENOMEM -5       /* an allocation or an admission budget was exceeded */
#define DES3_ENODEV -6       /* no usable CUDA device (or not an sm_103 GPU) */
#define DES3_EBUSY -7        /* the request queue is full; retry later */

/* ---- kernel selection ------------------------------------------------- */
#define DES3_KERNEL_AUTO 0     /* tuned default (per size class) */
#define DES3_KERNEL_BITSLICE 1 /* 32 blocks per thread as bit planes, S-boxes as LOP3 circuits */
#define DES3_KERNEL_SPTABLE 2  /* one block per thread, combined S+P tables in shared memory */

/* ---- key schedule (paper Listing 1.1: 48 round keys prepared on the host)
 *
 * rk[0][r], r = 0..47, are the round keys of 3DES encryption in the order
 * they are applied: K1's 16 round keys forward, K2's backward, K3's forward.
 * rk[1] is the same sequence reversed, which is 3DES decryption (Sec. II.A,
 * "performed identically only in reverse").  Each entry is a 48-bit DES
 * round key in its low 48 bits, round-key bit 1 (the one XORed into the first
 * E output bit, S1's first input) at bit 47.  The struct is plain data: copy
 * it freely, store it in device memory for the batched calls. */
#define DES3_KS_MAGIC 0x4B533344u /* "D3SK" little-endian */
typedef struct des3_ks {
    uint32_t magic;   /* DES3_KS_MAGIC once filled */
    uint32_t flags;   /* 0 for 3DES, DES3_KS_SINGLE_DES for single DES */
    uint64_t rk[2][48];
} des3_ks_t;

/* Fill *ks from a 24-byte key K1||K2||K3 (host memory).  Parity bits are
 * ignored; weak and semi-weak keys are accepted.  Pure host code, no GPU.
 * Errors: DES3_EINVAL for a null pointer. */
int des3_key_schedule(const uint8_t key[24], des3_ks_t* ks);

/* Single DES, the building block the paper composes three times (Sec. II.A):
 * fills *ks from an 8-byte key with rk[0][0..15] = K_1..K_16, rk[1][0..15] =
 * K_16..K_1 and flags = DES3_KS_SINGLE_DES.  Every call that takes a
 * des3_ks_t accepts it; the single-buffer ECB calls and des3_ecb_host then
 * run 16 rounds instead of 48, the other calls (modes, batches, server)
 * run it as 3DES with K1 = K2 = K3, which is the same cipher. */
#define DES3_KS_SINGLE_DES 1u
int des3_key_schedule_des(const uint8_t key[8], des3_ks_t* ks);

/* ---- single-buffer device calls (paper Sec. II.A, Listing 1.1) --------
 *
 * 3DES-EDE ECB encryption / decryption of nbytes bytes from d_in to d_out
 * (device memory), with the tuned default kernel.  ks points to HOST memory
 * and is read before the call returns.  Errors: DES3_EINVAL (null pointer,
 * nbytes % 8 != 0, an address not 8-byte aligned, partial overlap),
 * DES3_EKEY (ks not filled), DES3_ECUDA (launch failure). */
int des3_ecb_encrypt(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes,
                     des3_stream_t stream);
int des3_ecb_decrypt(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes,
                     des3_stream_t stream);

/* The same with an explicit direction (decrypt = 0 or 1) and kernel
 * (DES3_KERNEL_*).  All kernels give bit-identical results. */
int des3_ecb_crypt_ex(const des3_ks_t* ks, const void* d_in, void* d_out, size_t nbytes,
                      int decrypt, int kernel, des3_stream_t stream);

/* ---- CTR and CBC modes (NIST SP 800-38A) ---------------------------------
 *
 * The paper uses ECB only (abstract, Fig. 2).  These two modes reuse the same
 * 3DES block function and are just as parallel over blocks:
 *   - CTR: d_out_i = d_in_i xor E(T_i), T_i = counter + i modulo 2^64, the
 *     8-byte block read as a big-endian integer (the standard increment of
 *     the whole block).  The same call decrypts.  d_in may equal d_out.
 *   - CBC decryption: d_out_i = D(d_in_i) xor d_in_{i-1}, d_in_{-1} = iv.
 *     Every output block needs the previous INPUT block, so the buffers must
 *     not overlap at all (in place is DES3_EINVAL).  CBC encryption is
 *     sequential over blocks and is not offered.
 * counter / iv point to 8 bytes of host memory, read before the call
 * returns.  Both run the bitsliced kernel; errors as for des3_ecb_crypt_ex. */
int des3_ctr_crypt(const des3_ks_t* ks, const uint8_t counter[8], const void* d_in, void* d_out, size_t nbytes,
                   des3_stream_t stream);
int des3_cbc_decrypt(const des3_ks_t* ks, const uint8_t iv[8], const void* d_in, void* d_out, size_t nbytes,
                     des3_stream_t stream);

/* ---- host-memory call: copy in, encrypt, copy out ----------------------
 *
 * 3DES-EDE ECB of nbytes bytes from h_in to h_out (HOST memory), through the
 * caller's device workspace d_work of work_bytes bytes (at least 2 MiB,
 * 256-byte aligned).  The data is streamed in chunks: the copy of chunk i+1
 * to the device, the cipher on chunk i and the copy of chunk i-1 back to the
 * host overlap (paper Sec. II.B copies everything once and excludes the
 * transfers from its timings; this call keeps them and overlaps them with
 * the cipher, so it runs at the host link's speed).  The chunks grow from
 * 4 MiB to a third of the workspace (64 MiB at most) and shrink again at the
 * end.  h_in may equal h_out.  Asynchronous on `stream` like the device
 * calls; with pageable host memory the copies are staged synchronously by the
 * CUDA runtime.  Errors as for des3_ecb_crypt_ex, plus DES3_EINVAL when
 * work_bytes is too small. */
int des3_ecb_host(const des3_ks_t* ks, const void* h_in, void* h_out, size_t nbytes,
                  int decrypt, void* d_work, size_t work_bytes, des3_stream_t stream);

/* ---- host-memory call over several devices -------------------------------
 *
 * The paper remarks (Sec. III) that a second graphics card could raise the
 * throughput once the work is divided between the cards.  ECB processes
 * every 64-bit block on its own (abstract), so the division is a split of
 * the block range: des3_ecb_host_multi cuts the nbytes / 8 blocks of h_in
 * into ndev contiguous ranges with des3_range_split (granule: one bitsliced
 * tile, 1024 blocks) and runs des3_ecb_host on range i with devices[i] and
 * its workspace d_work[i] of work_bytes[i] bytes (device memory of
 * devices[i], at least 2 MiB, 256-byte aligned).  No device touches another
 * device's memory; there is no peer access and no collective.  One host
 * thread per non-empty range drives its device on a stream of its own, so the
 * ranges run at the same time.  The call is SYNCHRONOUS: it returns once
 * every range is written to h_out.  The caller's current device is kept.
 * A device may appear more than once (its ranges then share it); workspaces
 * of non-empty ranges must be distinct and must not overlap.  Ranges beyond
 * the block count are empty and need no workspace (d_work[i] may be null).
 * h_in may equal h_out.  Errors: as for des3_ecb_host, DES3_ENODEV for a
 * device id out of range, DES3_EINVAL for ndev == 0 or > 64, null arrays or
 * a workspace shared by two ranges; the first failing range's code is
 * returned. */
int des3_ecb_host_multi(const des3_ks_t* ks, const void* h_in, void* h_out, size_t nbytes, int decrypt,
                        uint32_t ndev, const int* devices, void* const* d_work, const size_t* work_bytes);

/* The split des3_ecb_host_multi uses, as plain host arithmetic: nblocks into
 * nparts contiguous ranges, range i = [first[i], first[i+1]), first[0] = 0,
 * first[nparts] = nblocks.  Every boundary is a multiple of granule blocks
 * (or nblocks itself); the granule counts of the ranges differ by at most
 * one, larger ranges first, and ranges past the end are empty.  first must
 * hold nparts + 1 entries.  Errors: DES3_EINVAL for nparts == 0, granule ==
 * 0 or a null first.  No GPU needed. */
int des3_range_split(uint64_t nblocks, uint32_t nparts, uint64_t granule, uint64_t* first);

/* ---- batched call (many buffers, one key schedule each) ----------------
 *
 * One persistent launch processes every job: job j transforms
 * jobs[j].nbytes bytes from jobs[j].d_in to jobs[j].d_out with the schedule
 * keys[jobs[j].key_index] in the direction given by flags bit 0
 * (DES3_JOB_DECRYPT).  The launch is the batched bitsliced kernel (jobs cut
 * into 1024-block tiles) or the batched table kernel (jobs cut into 64-block
 * segments, so that jobs far below one tile cost little), whichever the
 * DES3_TUNE_BATCH table names for the size class of the batch's total
 * bytes.  Where the table names the bitsliced kernel but the batch holds at
 * least one tile for every warp of the bitsliced grid and its jobs fill
 * their tiles so sparsely that a wave model (fitted on GB300) predicts the
 * table kernel faster, the table kernel runs in its default shape (384
 * threads, 3 CTAs per SM).  The arithmetic of each job is exactly that of a
 * single-buffer call.  Buffers of distinct jobs must not overlap (a job may
 * be in place). */
#define DES3_JOB_DECRYPT 1u
typedef struct des3_job {
    const void* d_in;
    void* d_out;
    uint64_t nbytes;
    uint32_t key_index;
    uint32_t flags;
} des3_job_t;

/* One-shot batch: keys (HOST array of nkeys schedules) and jobs (HOST array)
 * are uploaded (of the keys, only those some job names, expanded for the
 * chosen kernel) into device memory that the call allocates with
 * cudaMallocAsync on `stream` and frees again on the same stream.  The
 * upload comes from pageable host memory, so the call returns once the
 * tables are staged (which waits for work already queued on `stream`); the
 * launch itself is asynchronous.  Errors: DES3_EINVAL (bad job: null
 * pointer, size, alignment, key_index >= nkeys), DES3_EKEY, DES3_ENOMEM,
 * DES3_ECUDA. */
int des3_ecb_batch(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs, uint32_t njobs,
                   des3_stream_t stream);

/* Reusable batch plan: the job list is split into work tiles on the host
 * once, the tiles, jobs and keys are uploaded once into device memory the
 * plan owns, and the launch is captured in a CUDA graph.  Each
 * des3_batch_plan_launch replays the graph on `stream`; the buffers named by
 * the jobs must stay valid while a launch is in flight.  `kernel`:
 * DES3_KERNEL_AUTO makes the choice des3_ecb_batch makes, with the tuning
 * table as it stands at the time of creation; DES3_KERNEL_BITSLICE or
 * DES3_KERNEL_SPTABLE forces that batched kernel (with the table's shape
 * when the table names the same kernel, else the kernel's default shape).
 * Errors as for des3_ecb_batch. */
typedef struct des3_batch_plan des3_batch_plan_t;
int des3_batch_plan_create(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs,
                           uint32_t njobs, int kernel, des3_batch_plan_t** plan);
int des3_batch_plan_launch(des3_batch_plan_t* plan, des3_stream_t stream);
int des3_batch_plan_destroy(des3_batch_plan_t* plan);
/* Bytes of payload the plan covers and the number of 1024-block work tiles. */
int des3_batch_plan_info(const des3_batch_plan_t* plan, uint64_t* total_bytes, uint64_t* tiles);
/* The batched kernel the plan's graph launches (DES3_KERNEL_BITSLICE or
 * DES3_KERNEL_SPTABLE), its threads per CTA and CTAs per SM.  Any output
 * pointer may be null.  Errors: DES3_EINVAL for a null plan. */
int des3_batch_plan_kernel(const des3_batch_plan_t* plan, int* kernel, uint32_t* threads, uint32_t* ctas_per_sm);
/* The batched kernel and launch shape des3_ecb_batch (and a plan in
 * DES3_KERNEL_AUTO) would choose for these jobs on a device with `sms` SMs,
 * under the current tuning table.  Only the jobs' sizes are read: no buffer
 * is touched, no key is needed and no GPU is used.  Any output pointer may be
 * null.  Errors: DES3_EINVAL for null jobs with njobs > 0, a size that is not
 * a multiple of 8, or sms == 0 or > 4096. */
int des3_batch_choose(const des3_job_t* jobs, uint32_t njobs, uint32_t sms, int* kernel, uint32_t* threads,
                      uint32_t* ctas_per_sm);

/* ---- serving: continuous batching of requests ------------------------------
 *
 * An extension of the paper (which encrypts one file with one key):
 * a request server that keeps key schedules and buffers resident on the
 * device, admits requests against a byte budget, and batches whatever is
 * waiting into one persistent launch whenever one of its streams is free.
 * The launch is the bitsliced or the table batched kernel, chosen per batch
 * as des3_ecb_batch chooses.  Requests that arrive while others run on the
 * GPU join the next batch; batches on different streams overlap on the
 * device.  Each request's bytes are exactly those of a single-buffer call.
 *
 * A server owns: a device table of each key in both batched kernels' forms
 * (key_capacity keys, 832 + 768 bytes each), and per stream a device job
 * table and a pinned host staging table
 * (max_batch_requests jobs each).  All of it is allocated by
 * des3_server_create and freed by des3_server_destroy.  Request buffers are
 * the caller's device memory and must stay valid until the request
 * completes.  Every call is thread-safe. */
typedef struct des3_server des3_server_t;

typedef struct des3_server_config {
    uint64_t budget_bytes;        /* admission budget: payload bytes in flight (e.g. 16 GiB) */
    uint32_t max_inflight;        /* requests in flight at most (slots) */
    uint32_t max_queue;           /* requests waiting for admission at most; beyond: DES3_EBUSY */
    uint32_t nstreams;            /* batches that may run at once (1..16) */
    uint32_t max_batch_requests;  /* requests per launch at most */
    uint64_t max_batch_bytes;     /* payload bytes per launch at most */
    uint32_t key_capacity;        /* key schedules the device cache holds */
    uint32_t fault_every;         /* test hook: fail every n-th batch (0 = never) ... */
    uint32_t fault_stage;         /* ... at DES3_FAULT_AT_LAUNCH or DES3_FAULT_AT_COMPLETION */
} des3_server_config_t;
/* Test hook stages (no GPU fault is involved in either): AT_LAUNCH skips the
 * n-th batch's launch on the host; AT_COMPLETION lets its kernel run and then
 * reports the batch as failed, the way an error raised on the device while it
 * ran is reported.  Its requests complete with DES3_ECUDA either way. */
#define DES3_FAULT_AT_LAUNCH 0u
#define DES3_FAULT_AT_COMPLETION 1u

typedef struct des3_request {
    const void* d_in;
    void* d_out;
    uint64_t nbytes;      /* multiple of 8 */
    uint32_t key_id;      /* from des3_server_add_keys */
    uint32_t flags;       /* DES3_JOB_DECRYPT */
    uint64_t tag;         /* returned in the completion */
} des3_request_t;

typedef struct des3_completion {
    uint64_t ticket;
    uint64_t tag;
    int status;           /* DES3_OK, or the batch's error: a failed enqueue or an
                             error the device raised while the batch ran */
    uint32_t batch_size;  /* requests in the launch that carried it */
    double latency_s;     /* submit (or scheduled arrival) -> completion */
} des3_completion_t;

typedef struct des3_server_stats {
    uint64_t submitted, completed, failed, launches, bytes_completed;
    uint64_t inflight_bytes, inflight_requests, queued_requests;
    uint64_t table_launches; /* launches that ran the batched table kernel */
} des3_server_stats_t;

int des3_server_create(const des3_server_config_t* cfg, des3_server_t** server);
/* Uploads n key schedules into the device cache; their ids are
 * first_id .. first_id + n - 1.  DES3_ENOMEM when the cache is full.
 * Concurrent calls are serialised; the caller's current device is kept. */
int des3_server_add_keys(des3_server_t* server, const des3_ks_t* keys, uint32_t n, uint32_t* first_id);
/* Queues one request; returns at once.  DES3_EBUSY when max_queue requests
 * already wait; DES3_EINVAL for a bad request (size, alignment, key id, or a
 * request larger than the budget). */
int des3_server_submit(des3_server_t* server, const des3_request_t* req, uint64_t* ticket);
/* Moves up to max finished requests into out[]; *n receives the count. */
int des3_server_poll(des3_server_t* server, des3_completion_t* out, uint32_t max, uint32_t* n);
/* Waits until nothing is queued or in flight; DES3_ETIMEOUT after timeout_ms
 * (0 or negative: checks once without waiting). */
int des3_server_drain(des3_server_t* server, int timeout_ms);
int des3_server_stats(des3_server_t* server, des3_server_stats_t* out);
/* Benchmark driver: submits reqs[i] at arrival_s[i] seconds after the call
 * starts (the calling thread paces the arrivals in native code, so no
 * interpreter sits in the loop), waits for all of them, and writes each one's
 * latency measured from its scheduled arrival to latency_s[i] (negative if
 * it failed).  Completions of requests submitted by other calls are left for
 * des3_server_poll.  Returns DES3_OK, the first error, or DES3_ETIMEOUT when
 * the requests have not all finished timeout_ms after the last submission. */
int des3_server_replay(des3_server_t* server, const des3_request_t* reqs, const double* arrival_s, uint32_t n,
                       double* latency_s, int timeout_ms);
/* Stops the dispatcher, waits for the launches in flight, and frees the
 * server.  Requests still queued (not yet launched) are dropped without a
 * completion. */
int des3_server_destroy(des3_server_t* server);

/* ---- batched call without any allocation ---------------------------------
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc.  Some processes hand all device memory to their own
 * pool allocator at start-up and may not allocate outside it afterwards, and
 * some latency-sensitive code must not call cudaMalloc/cudaFree because those
 * calls can synchronise the whole device.  des3_ecb_batch allocates its job
 * and key tables with cudaMallocAsync; this variant instead keeps them in a
 * fixed scratch array compiled into the library (a file-scope __device__
 * array of DES3_NOALLOC_SCRATCH_BYTES bytes, about 872 KiB, that every GPU
 * which loads the library holds until the process exits).
 *
 * Semantics, arguments and results are those of des3_ecb_batch (same jobs,
 * same keys, bit-identical output).  Differences:
 *   - At most DES3_NOALLOC_MAX_JOBS jobs and DES3_NOALLOC_MAX_KEYS keys;
 *     more is rejected with DES3_EINVAL before anything is enqueued.
 *   - It calls no cudaMalloc, cudaFree or other allocating routine.  The job
 *     and key tables are staged in static host arrays and copied with
 *     cudaMemcpyAsync into the scratch array on `stream`, then the kernel runs
 *     on `stream`.
 *   - That copy comes from pageable host memory, so the call returns only
 *     after the work already queued on `stream` has finished and the tables
 *     are staged; other host threads calling it wait for that time (the
 *     staging arrays are shared, so calls are serialised on the host).
 *   - A `stream` that is being captured into a CUDA graph is refused with
 *     DES3_EINVAL before anything is enqueued: a captured copy would read the
 *     staging arrays when the graph is replayed, after later calls have
 *     overwritten them.
 *   - The first call on each device looks up the scratch array's device
 *     address (cudaGetSymbolAddress) with that device current, and looks it
 *     up again after the device's context has been replaced (for example by
 *     cudaDeviceReset).
 *   - Every call uses the same scratch array, which keeps the previous call's
 *     tables until overwritten; nothing in it needs to start at zero.  Calls
 *     whose work overlaps on the GPU (e.g. issued on different streams
 *     without ordering) race on the array and may produce wrong output:
 *     order them on one stream or with events. */
#define DES3_NOALLOC_MAX_JOBS 1024u
#define DES3_NOALLOC_MAX_KEYS 1024u
#define DES3_NOALLOC_SCRATCH_BYTES (40u * DES3_NOALLOC_MAX_JOBS + 832u * DES3_NOALLOC_MAX_KEYS)
int des3_ecb_batch_noalloc(const des3_ks_t* keys, uint32_t nkeys, const des3_job_t* jobs, uint32_t njobs,
                           des3_stream_t stream);

/* ---- launch tuning (size classes) --------------------------------------
 *
 * DES3_KERNEL_AUTO and the batched calls look up a table indexed by the size
 * class of the work, c = floor(log2(bytes)) (0..DES3_TUNE_CLASSES-1).  An
 * entry names the kernel (bitsliced or table; for the batch table, the
 * batched form of either), the CTA size and the number of persistent CTAs
 * per SM.  des3_ecb_batch_noalloc keeps the bitsliced kernel: where the
 * batch table names the table kernel it uses the bitsliced kernel's default
 * shape.  The library starts with built-in tables (the autotuner's GB300
 * choices); the autotuner (paper_1305_4376_gb300/autotune.py)
 * measures the candidates on the GPU and installs its choices with
 * des3_tune_set.  Tables are process-wide; setting one is thread-safe and
 * affects calls made afterwards.  Errors: DES3_EINVAL for an unknown table,
 * a class out of range, or a shape the kernel cannot launch (threads not 64,
 * 128, 256 or 384; more than 384 bitsliced threads per SM; more CTAs per SM
 * than shared memory allows, i.e. more than 3 for the table kernel). */
#define DES3_TUNE_CLASSES 40
#define DES3_TUNE_SINGLE 0 /* single-buffer calls, indexed by the buffer size */
#define DES3_TUNE_BATCH 1  /* batched calls and the server, indexed by the batch's total bytes */
typedef struct des3_tune_entry {
    uint32_t size_class;
    int32_t kernel;       /* DES3_KERNEL_BITSLICE or DES3_KERNEL_SPTABLE */
    uint32_t threads;     /* 64, 128, 256 or 384 (bitsliced kernels only) */
    uint32_t ctas_per_sm; /* 1..8, within the kernel's register and shared-memory limits */
} des3_tune_entry_t;
int des3_tune_set(int table, const des3_tune_entry_t* entries, uint32_t n);
int des3_tune_get(int table, uint32_t size_class, des3_tune_entry_t* out);
int des3_tune_reset(void);

/* ---- diagnostics ------------------------------------------------------ */

/* Static cost of a kernel, for roofline accounting, per 64-bit block as
 * written in the kernel source: instructions for the integer ALU pipe (LOP3,
 * shifts, byte permutes: S-box gates or table index arithmetic, state XORs,
 * transposes), instructions for the FMA pipe (multiply-adds), and
 * shared-memory loads.  sbox_gates is the total LOP3 gate count of the
 * bitsliced S1..S8 circuits (0 for the table kernel). */
typedef struct des3_kernel_info {
    double alu_ops_per_block;
    double fma_ops_per_block;
    double smem_loads_per_block;
    int sbox_gates;
    int blocks_per_thread;
} des3_kernel_info_t;
int des3_kernel_info(int kernel, des3_kernel_info_t* info);

/* Throughput probe of the pipes the kernels are bound by.  The paper has no
 * counterpart: it measures the roofline denominators on the running device
 * so that a benchmark can state them from the same run.
 *   kind 0: lop3.b32 (integer ALU pipe: the bitsliced kernel's gates)
 *   kind 1: mad.lo.u32 (FMA pipe)
 *   kind 2: lop3.b32 and mad.lo.u32, 1:1
 *   kind 3: ld.shared.u32, every lane in its own bank (shared-memory pipe:
 *           the table kernel's lookups)
 * One launch of 8 CTAs of 256 threads per SM on `stream`; every thread runs
 * 8 independent chains of iters x 16 instructions, so the launch runs at the
 * pipe's issue rate.  Time it with events on `stream`.  d_sink: at least 24
 * bytes of caller-owned device memory, 8-byte aligned; the launch XORs its
 * results into word 0 and writes, from thread 0 of CTA 0, the SM clock cycles
 * (word 1) and global-timer nanoseconds (word 2) between its first and last
 * probe instruction: their ratio is the SM clock during the probe.
 * *instructions receives the lane-instructions the launch executes and *sms
 * the device's SM count.  Errors: DES3_EINVAL (kind, iters == 0, a null or
 * misaligned pointer), DES3_ENODEV, DES3_ECUDA. */
int des3_pipe_probe(int kind, uint32_t iters, void* d_sink, uint64_t* instructions, uint32_t* sms,
                    des3_stream_t stream);

const char* des3_strerror(int code);
int des3_last_cuda_error(void);
/* Host-only self test of the library's internal permutation networks,
 * combined tables and S-box circuits against the standard's tables (all 64
 * inputs of every S-box).  Returns DES3_OK or DES3_EINVAL.  No GPU needed. */
int des3_self_test(void);
/* Library version as "major.minor.patch". */
const char* des3_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DES3_H */
