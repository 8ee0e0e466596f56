// serve.cu -- a continuous-batching request server over the batched kernel.
//
// Requests (device buffers + a cached key id + a direction) are queued by
// des3_server_submit.  One dispatcher thread admits queued requests in
// arrival order while the payload in flight stays within the byte budget and
// the request count within max_inflight, and as soon as one of the server's
// streams is free it sends everything admitted (up to the batch limits) to
// the GPU as ONE persistent launch of a batched kernel: the bitsliced batch
// or the batched table kernel, chosen per batch as a one-shot batched call
// chooses (auto_batch_shape), so a light load's small batches take the
// table kernel; the server keeps both kernels' forms of every key.  An event
// is recorded behind the launch, and a host function behind the event
// timestamps the batch and wakes the dispatcher.  The dispatcher then reads
// the batch's status from the event (so an error the kernel raised while it
// ran is reported, not only a failure to enqueue it), publishes the
// completions, releases the budget and frees the stream.  CUDA does not run
// host functions once its context has failed, so while batches are in flight
// the dispatcher also queries their events every millisecond.  A request
// that arrives while others are on the GPU joins the next batch, and batches
// on different streams overlap on the device.  The arithmetic of a request
// is the single-buffer kernel's, so its bytes do not depend on what it was
// batched with.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tuning.h"

namespace {

using des3::BatchTileJob;

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Req {
    des3_request_t r;
    uint64_t ticket;
    int64_t t_arrival;
};

struct Batch {
    des3_server* srv = nullptr;
    int stream_index = 0;
    int status = DES3_OK;   // enqueue status (DES3_OK once launched)
    uint64_t launch_no = 0;
    bool signalled = false;  // the host function behind the batch has run
    int64_t t_done = 0;      // when it ran (ns)
    std::vector<Req> reqs;
};

}  // namespace

struct des3_server {
    des3_server_config_t cfg{};
    int device = 0;
    uint32_t* d_keys = nullptr;    // packed masks of the bitsliced batch
    uint32_t* d_spkeys = nullptr;  // round-key words of the batched table kernel
    uint32_t nkeys = 0;
    int sms = 0;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // recorded behind each stream's batch
    std::vector<BatchTileJob*> d_jobs;
    std::vector<BatchTileJob*> h_jobs;
    std::vector<Batch> batches;
    std::vector<char> busy;
    std::mutex mu;
    std::mutex keys_mu;  // serialises des3_server_add_keys (reserve, upload, publish)
    std::condition_variable cv;
    std::deque<Req> queue;
    std::deque<des3_completion_t> done;
    uint64_t next_ticket = 1;
    uint64_t inflight_bytes = 0, inflight_reqs = 0;
    uint64_t submitted = 0, completed = 0, failed = 0, launches = 0, bytes_completed = 0;
    std::atomic<uint64_t> table_launches{0};  // batches launched on the table kernel
    bool stop = false;
    std::thread dispatcher;
};

namespace {

// Host function behind a batch: timestamps it and wakes the dispatcher.  It
// makes no CUDA call (host functions may not).
void CUDART_CB on_batch_signal(void* p) {
    Batch* b = static_cast<Batch*>(p);
    des3_server* s = b->srv;
    const int64_t t = now_ns();
    std::lock_guard<std::mutex> g(s->mu);
    b->signalled = true;
    b->t_done = t;
    s->cv.notify_all();
}

// Publishes the completions of batch `si` with `status`, releases its budget
// and frees its stream.  Called with s->mu held.
void complete_locked(des3_server* s, int si, int status) {
    Batch& b = s->batches[si];
    const int64_t t = b.signalled ? b.t_done : now_ns();
    for (const Req& q : b.reqs) {
        des3_completion_t c;
        c.ticket = q.ticket;
        c.tag = q.r.tag;
        c.status = status;
        c.batch_size = (uint32_t)b.reqs.size();
        c.latency_s = (double)(t - q.t_arrival) * 1e-9;
        s->done.push_back(c);
        s->inflight_bytes -= q.r.nbytes;
        s->inflight_reqs--;
        s->completed++;
        if (status != DES3_OK) s->failed++;
        else s->bytes_completed += q.r.nbytes;
    }
    b.reqs.clear();
    b.signalled = false;
    s->busy[si] = 0;
    s->cv.notify_all();
}

// The status of a finished batch from its event, or 1 while it is not
// finished.  A batch counts as finished once its host function has run
// (`signalled`), or earlier only when its event reports an error: then the
// context has failed and the host function will never run.  A successful
// batch is never completed before its host function, which would otherwise
// touch the slot's next batch.  Called without s->mu (it makes CUDA calls).
int batch_result(des3_server* s, int si, bool signalled, int enqueue_status, uint64_t launch_no) {
    int status = enqueue_status;
    const cudaError_t e = cudaEventQuery(s->events[si]);
    if (e == cudaErrorNotReady || (e == cudaSuccess && !signalled)) return 1;
    if (e != cudaSuccess && status == DES3_OK) status = des3::cuda_fail(e);
    // test hook: report the n-th batch as failed once its kernel has run
    if (status == DES3_OK && s->cfg.fault_every && s->cfg.fault_stage == DES3_FAULT_AT_COMPLETION &&
        launch_no % s->cfg.fault_every == 0)
        status = DES3_ECUDA;
    return status;
}

int free_stream(const des3_server* s) {
    for (size_t i = 0; i < s->busy.size(); i++)
        if (!s->busy[i]) return (int)i;
    return -1;
}

bool admissible(const des3_server* s) {
    if (s->queue.empty()) return false;
    const Req& q = s->queue.front();
    return s->inflight_bytes + q.r.nbytes <= s->cfg.budget_bytes && s->inflight_reqs < s->cfg.max_inflight;
}

// Builds the job table of batch `si` in pinned memory, uploads it and
// launches; the event and the host function are enqueued in every case.
void launch_one(des3_server* s, int si, cudaError_t device_error) {
    Batch& b = s->batches[si];
    cudaStream_t st = s->streams[si];
    BatchTileJob* hj = s->h_jobs[si];
    const uint32_t n = (uint32_t)b.reqs.size();
    uint64_t tiles = 0, segs = 0, bytes = 0;
    for (uint32_t i = 0; i < n; i++) {
        const uint64_t nb = b.reqs[i].r.nbytes / 8;
        tiles += (nb + des3::kTileBlocks - 1) / des3::kTileBlocks;
        segs += (nb + des3::kSegBlocks - 1) / des3::kSegBlocks;
        bytes += b.reqs[i].r.nbytes;
    }
    // the kernel for this batch, as a one-shot batched call would choose it
    const des3::BatchShape shape = des3::auto_batch_shape(bytes, n, tiles, segs, s->sms);
    const bool table = shape.kernel == DES3_KERNEL_SPTABLE;
    const uint64_t grain = table ? des3::kSegBlocks : des3::kTileBlocks;
    uint64_t units = 0;
    for (uint32_t i = 0; i < n; i++) {
        const des3_request_t& r = b.reqs[i].r;
        hj[i].in = static_cast<const uint8_t*>(r.d_in);
        hj[i].out = static_cast<uint8_t*>(r.d_out);
        hj[i].nblocks = r.nbytes / 8;
        hj[i].tile_begin = units;
        hj[i].key_index = r.key_id;
        hj[i].decrypt = r.flags & DES3_JOB_DECRYPT;
        units += (hj[i].nblocks + grain - 1) / grain;
    }
    int rc = DES3_OK;
    if (device_error != cudaSuccess) {
        rc = des3::cuda_fail(device_error);  // the dispatcher thread has no device: nothing is launched
    } else if (s->cfg.fault_every && s->cfg.fault_stage == DES3_FAULT_AT_LAUNCH &&
               b.launch_no % s->cfg.fault_every == 0) {
        rc = DES3_ECUDA;  // test hook, injected on the host: the launch is skipped
    } else {
        cudaError_t e = cudaMemcpyAsync(s->d_jobs[si], hj, sizeof(BatchTileJob) * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = des3::cuda_fail(e);
        if (rc == DES3_OK)
            rc = table ? des3::launch_batch_sptable(s->d_jobs[si], n, s->d_spkeys, units, shape.ctas_per_sm,
                                                    shape.threads, st)
                       : des3::launch_batch(s->d_jobs[si], n, s->d_keys, units, shape.ctas_per_sm, shape.threads, st);
        if (rc == DES3_OK && table) s->table_launches++;
    }
    b.status = rc;
    bool signal_now = device_error != cudaSuccess || cudaEventRecord(s->events[si], st) != cudaSuccess;
    if (!signal_now && cudaLaunchHostFunc(st, on_batch_signal, &b) != cudaSuccess) signal_now = true;
    if (signal_now) {
        // Nothing will signal the batch.  If anything was enqueued, wait for
        // the stream first, so that no completion is published while the
        // kernel may still write the requests' buffers; the batch then
        // completes with an error (the event holds no newer record).
        if (device_error == cudaSuccess) cudaStreamSynchronize(st);
        std::lock_guard<std::mutex> g(s->mu);
        b.signalled = true;
        b.t_done = now_ns();
        if (b.status == DES3_OK) b.status = DES3_ECUDA;
        s->cv.notify_all();
    }
}

bool any_signalled(const des3_server* s) {
    for (size_t i = 0; i < s->busy.size(); i++)
        if (s->busy[i] && s->batches[i].signalled) return true;
    return false;
}

bool any_busy(const des3_server* s) {
    for (char b : s->busy)
        if (b) return true;
    return false;
}

void dispatch_loop(des3_server* s) {
    const cudaError_t dev_err = cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    int64_t last_poll = now_ns();
    for (;;) {
        auto ready = [&] { return s->stop || any_signalled(s) || (free_stream(s) >= 0 && admissible(s)); };
        if (any_busy(s)) s->cv.wait_for(lk, std::chrono::milliseconds(1), ready);
        else s->cv.wait(lk, ready);
        if (s->stop) break;
        // finished batches first: their streams and budget free up.  Batches
        // whose host function has not run are polled for a context error at
        // most once a millisecond, not on every wake-up (every submission
        // wakes this thread).
        const int64_t t = now_ns();
        const bool poll_all = t - last_poll >= 1000000;
        if (poll_all) last_poll = t;
        for (size_t si = 0; si < s->busy.size(); si++) {
            if (!s->busy[si] || !(s->batches[si].signalled || poll_all)) continue;
            Batch& b = s->batches[si];
            const bool sig = b.signalled;
            const int enq = b.status;
            const uint64_t no = b.launch_no;
            lk.unlock();
            const int st = dev_err != cudaSuccess ? des3::cuda_fail(dev_err) : batch_result(s, (int)si, sig, enq, no);
            lk.lock();
            if (st != 1) complete_locked(s, (int)si, st);
        }
        const int si = free_stream(s);
        if (si < 0 || !admissible(s)) continue;
        Batch& b = s->batches[si];
        b.reqs.clear();
        b.signalled = false;
        uint64_t bytes = 0;
        while (admissible(s) && b.reqs.size() < s->cfg.max_batch_requests) {
            const Req& q = s->queue.front();
            if (!b.reqs.empty() && bytes + q.r.nbytes > s->cfg.max_batch_bytes) break;
            s->inflight_bytes += q.r.nbytes;
            s->inflight_reqs++;
            bytes += q.r.nbytes;
            b.reqs.push_back(q);
            s->queue.pop_front();
        }
        s->busy[si] = 1;
        b.launch_no = ++s->launches;
        lk.unlock();
        launch_one(s, si, dev_err);
        lk.lock();
    }
}

int check_request(const des3_server* s, const des3_request_t* r) {
    if (!r || r->nbytes % 8 || (r->flags & ~DES3_JOB_DECRYPT)) return DES3_EINVAL;
    if (r->key_id >= s->nkeys) return DES3_EINVAL;
    if (r->nbytes > s->cfg.budget_bytes) return DES3_EINVAL;
    if (r->nbytes == 0) return DES3_OK;
    if (!r->d_in || !r->d_out) return DES3_EINVAL;
    const uintptr_t x = reinterpret_cast<uintptr_t>(r->d_in), y = reinterpret_cast<uintptr_t>(r->d_out);
    if ((x | y) & 7) return DES3_EINVAL;
    if (x != y && x < y + r->nbytes && y < x + r->nbytes) return DES3_EINVAL;
    return DES3_OK;
}

int submit_at(des3_server* s, const des3_request_t* r, int64_t t_arrival, uint64_t* ticket) {
    int rc = check_request(s, r);
    if (rc != DES3_OK) return rc;
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return DES3_EINVAL;
    const uint64_t tk = s->next_ticket++;
    if (ticket) *ticket = tk;
    s->submitted++;
    if (r->nbytes == 0) {  // nothing to do: complete at once
        des3_completion_t c{tk, r->tag, DES3_OK, 0, (double)(now_ns() - t_arrival) * 1e-9};
        s->done.push_back(c);
        s->completed++;
        s->cv.notify_all();
        return DES3_OK;
    }
    if (s->queue.size() >= s->cfg.max_queue) {
        s->submitted--;
        s->next_ticket--;
        return DES3_EBUSY;
    }
    s->queue.push_back(Req{*r, tk, t_arrival});
    // The dispatcher can only act on a new request while a stream is free;
    // with every stream busy it is woken by the next finished batch (or its
    // millisecond poll), so near saturation submissions do not wake it.
    if (free_stream(s) >= 0) s->cv.notify_all();
    return DES3_OK;
}

void destroy_impl(des3_server* s) {
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamSynchronize(st);
    for (cudaStream_t st : s->streams)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : s->events)
        if (ev) cudaEventDestroy(ev);
    for (BatchTileJob* p : s->d_jobs)
        if (p) cudaFree(p);
    for (BatchTileJob* p : s->h_jobs)
        if (p) cudaFreeHost(p);
    if (s->d_keys) cudaFree(s->d_keys);
    if (s->d_spkeys) cudaFree(s->d_spkeys);
    delete s;
}

}  // namespace

extern "C" {

int des3_server_create(const des3_server_config_t* cfg, des3_server_t** out) {
    if (!cfg || !out) return DES3_EINVAL;
    *out = nullptr;
    if (cfg->budget_bytes == 0 || cfg->max_inflight == 0 || cfg->max_queue == 0 || cfg->nstreams == 0 ||
        cfg->nstreams > 16 || cfg->max_batch_requests == 0 || cfg->max_batch_bytes == 0 || cfg->key_capacity == 0 ||
        (cfg->fault_stage != DES3_FAULT_AT_LAUNCH && cfg->fault_stage != DES3_FAULT_AT_COMPLETION))
        return DES3_EINVAL;
    des3::DeviceInfo di;
    int rc = des3::current_device_info(&di);
    if (rc != DES3_OK) return rc;
    if ((rc = des3::batch_prepare()) != DES3_OK) return rc;
    if ((rc = des3::batch_prepare_sptable()) != DES3_OK) return rc;
    des3_server* s = new des3_server();
    s->cfg = *cfg;
    s->device = di.device;
    s->sms = di.sms;
    const uint32_t n = cfg->nstreams;
    s->streams.assign(n, nullptr);
    s->events.assign(n, nullptr);
    s->d_jobs.assign(n, nullptr);
    s->h_jobs.assign(n, nullptr);
    s->batches.resize(n);
    s->busy.assign(n, 0);
    cudaError_t e = cudaMalloc(&s->d_keys, (size_t)cfg->key_capacity * 2 * des3::kKeyBitsStride * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_spkeys, (size_t)cfg->key_capacity * 2 * des3::kSpKeyStride * 4);
    for (uint32_t i = 0; e == cudaSuccess && i < n; i++) {
        s->batches[i].srv = s;
        s->batches[i].stream_index = (int)i;
        s->batches[i].reqs.reserve(cfg->max_batch_requests);
        e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_jobs[i], sizeof(BatchTileJob) * cfg->max_batch_requests);
        if (e == cudaSuccess) e = cudaMallocHost(&s->h_jobs[i], sizeof(BatchTileJob) * cfg->max_batch_requests);
    }
    if (e != cudaSuccess) {
        rc = e == cudaErrorMemoryAllocation ? DES3_ENOMEM : des3::cuda_fail(e);
        destroy_impl(s);
        return rc;
    }
    s->dispatcher = std::thread(dispatch_loop, s);
    *out = s;
    return DES3_OK;
}

int des3_server_add_keys(des3_server_t* s, const des3_ks_t* keys, uint32_t n, uint32_t* first_id) {
    if (!s || (n && !keys)) return DES3_EINVAL;
    for (uint32_t i = 0; i < n; i++)
        if (keys[i].magic != DES3_KS_MAGIC) return DES3_EKEY;
    std::lock_guard<std::mutex> kg(s->keys_mu);
    uint32_t first;
    {
        std::lock_guard<std::mutex> g(s->mu);
        if ((uint64_t)s->nkeys + n > s->cfg.key_capacity) return DES3_ENOMEM;
        first = s->nkeys;
    }
    // both batched kernels' forms of every key: a batch may run on either
    std::vector<uint32_t> bits((size_t)n * 2 * des3::kKeyBitsStride);
    des3::batch_fill_keys(keys, n, bits.data());
    std::vector<uint32_t> words((size_t)n * 2 * des3::kSpKeyStride);
    des3::batch_fill_spkeys(keys, n, words.data());
    // upload on the server's device, leaving the caller's current device as it was
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != s->device) e = cudaSetDevice(s->device);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_keys + (size_t)first * 2 * des3::kKeyBitsStride, bits.data(),
                       bits.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_spkeys + (size_t)first * 2 * des3::kSpKeyStride, words.data(),
                       words.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (prev != s->device) cudaSetDevice(prev);
    if (e != cudaSuccess) return des3::cuda_fail(e);
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->nkeys = first + n;  // visible to submitters only once uploaded
    }
    if (first_id) *first_id = first;
    return DES3_OK;
}

int des3_server_submit(des3_server_t* s, const des3_request_t* req, uint64_t* ticket) {
    if (!s) return DES3_EINVAL;
    return submit_at(s, req, now_ns(), ticket);
}

int des3_server_poll(des3_server_t* s, des3_completion_t* out, uint32_t max, uint32_t* n) {
    if (!s || !n || (max && !out)) return DES3_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    uint32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n = k;
    return DES3_OK;
}

int des3_server_drain(des3_server_t* s, int timeout_ms) {
    if (!s) return DES3_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                                   [&] { return s->queue.empty() && s->inflight_reqs == 0; });
    return ok ? DES3_OK : DES3_ETIMEOUT;
}

int des3_server_stats(des3_server_t* s, des3_server_stats_t* o) {
    if (!s || !o) return DES3_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    o->submitted = s->submitted;
    o->completed = s->completed;
    o->failed = s->failed;
    o->launches = s->launches;
    o->bytes_completed = s->bytes_completed;
    o->inflight_bytes = s->inflight_bytes;
    o->inflight_requests = s->inflight_reqs;
    o->queued_requests = s->queue.size();
    o->table_launches = s->table_launches.load();
    return DES3_OK;
}

int des3_server_replay(des3_server_t* s, const des3_request_t* reqs, const double* arrival_s, uint32_t n,
                       double* latency_s, int timeout_ms) {
    if (!s || (n && (!reqs || !arrival_s || !latency_s))) return DES3_EINVAL;
    std::unordered_map<uint64_t, uint32_t> index;
    index.reserve(n * 2 + 1);
    for (uint32_t i = 0; i < n; i++) latency_s[i] = -1.0;
    const int64_t t0 = now_ns() + 1000000;  // start 1 ms from now
    int first_err = DES3_OK;
    for (uint32_t i = 0; i < n; i++) {
        const int64_t target = t0 + (int64_t)(arrival_s[i] * 1e9);
        for (int64_t t = now_ns(); t < target; t = now_ns())
            if (target - t > 200000) std::this_thread::sleep_for(std::chrono::microseconds(50));
        uint64_t tk = 0;
        int rc;
        // a full queue means overload: keep the scheduled arrival time and retry
        while ((rc = submit_at(s, &reqs[i], target, &tk)) == DES3_EBUSY) std::this_thread::yield();
        if (rc != DES3_OK) {
            if (first_err == DES3_OK) first_err = rc;
            continue;
        }
        index[tk] = i;
    }
    // collect the completions of our tickets; others go back to the queue
    // of finished requests for the caller's own des3_server_poll
    const int64_t deadline = now_ns() + (int64_t)timeout_ms * 1000000;
    size_t got = 0;
    std::vector<des3_completion_t> buf(256), others;
    auto give_back = [&]() {
        if (others.empty()) return;
        std::lock_guard<std::mutex> g(s->mu);
        for (const des3_completion_t& c : others) s->done.push_back(c);
        others.clear();
    };
    while (got < index.size()) {
        uint32_t k = 0;
        des3_server_poll(s, buf.data(), (uint32_t)buf.size(), &k);
        for (uint32_t j = 0; j < k; j++) {
            auto it = index.find(buf[j].ticket);
            if (it == index.end()) {
                others.push_back(buf[j]);
                continue;
            }
            latency_s[it->second] = buf[j].status == DES3_OK ? buf[j].latency_s : -1.0;
            if (buf[j].status != DES3_OK && first_err == DES3_OK) first_err = buf[j].status;
            got++;
        }
        if (k == 0) {
            if (now_ns() > deadline) {
                give_back();
                return DES3_ETIMEOUT;
            }
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait_for(lk, std::chrono::microseconds(200), [&] { return !s->done.empty(); });
        }
    }
    give_back();
    return first_err;
}

int des3_server_destroy(des3_server_t* s) {
    if (!s) return DES3_OK;
    destroy_impl(s);
    return DES3_OK;
}

}  // extern "C"
