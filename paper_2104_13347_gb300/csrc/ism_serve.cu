// ism_serve.cu -- continuous batching of RIR + convolution requests.
//
// A background thread owns all CUDA work of a server:
//  * admission: requests wait in FIFO order until their device footprint
//    (RIRs + source + outputs) fits under max_hbm_bytes next to what is in
//    use, and a stream slot is free;
//  * batching: the admitted head of the queue (up to max_batch requests) is
//    packed into one device block and one ragged launch of each kernel
//    (K1 taps, convolution, noise) on the slot's stream, so batches on
//    different streams overlap on the GPU while new requests keep arriving;
//  * completion: an event per batch, polled with cudaEventQuery (never a
//    blocking wait), marks the batch's requests done and records latency.
// Every request's RIR windows, convolution tiles and noise streams (keyed
// by its noise id, or its ticket) are the same work items whatever else is
// in its batch, so a result is the same alone or in any mix up to FP32
// rounding (the RIR sums use shared-memory atomics).  The device is selected lazily
// by the thread: if it cannot be used, requests fail with ISM_ERR_CUDA and a
// message, which poll/wait report.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ism_internal.h"

namespace ism {
int validate_room(const ism_room &r, int64_t idx);
}

using namespace ism;

namespace {

using Clock = std::chrono::steady_clock;

enum State { QUEUED, RUNNING, DONE, FAILED };

// Page-locked host blocks by power-of-two size class, kept for reuse:
// cudaHostAlloc and cudaFreeHost are slow and cudaFreeHost can wait for the
// device, so a request's source copy and a batch's statistics readback take
// a cached block.  At most kMaxCached bytes stay cached; blocks beyond that
// are freed.  A block that cudaHostAlloc could not provide comes from malloc
// (pageable: its copies do not overlap) and is freed on return.
class PinnedPool {
  public:
    static constexpr size_t kMaxCached = size_t(1) << 30;
    struct Block {
        void *ptr = nullptr;
        size_t cls = 0;      // size class, bytes
        bool pinned = false;
    };
    Block get(size_t bytes) {
        size_t cls = 4096;
        while (cls < bytes) cls <<= 1;
        {
            std::lock_guard<std::mutex> lk(mu_);
            auto &v = free_[cls];
            if (!v.empty()) {
                Block b{v.back(), cls, true};
                v.pop_back();
                cached_ -= cls;
                return b;
            }
        }
        Block b{nullptr, cls, true};
        if (cudaHostAlloc(&b.ptr, cls, 0) != cudaSuccess) {
            cudaGetLastError();
            b.ptr = malloc(cls);
            b.pinned = false;
        }
        return b;
    }
    void put(const Block &b) {
        if (!b.ptr) return;
        if (!b.pinned) {
            free(b.ptr);
            return;
        }
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (cached_ + b.cls <= kMaxCached) {
                free_[b.cls].push_back(b.ptr);
                cached_ += b.cls;
                return;
            }
        }
        if (cudaFreeHost(b.ptr) != cudaSuccess) cudaGetLastError();
    }
    ~PinnedPool() {
        for (auto &kv : free_)
            for (void *p : kv.second)
                if (cudaFreeHost(p) != cudaSuccess) cudaGetLastError();
    }

  private:
    std::mutex mu_;
    std::map<size_t, std::vector<void *>> free_;
    size_t cached_ = 0;
};

struct Batch;

struct Req {
    uint64_t ticket;
    ism_room room;
    std::vector<double> mics;
    float *src_pinned = nullptr;  // the source copy (src_block.ptr)
    PinnedPool::Block src_block;
    int64_t src_len = 0;
    float snr_db = NAN;
    uint64_t noise_id = 0;
    int64_t bytes = 0;
    State state = QUEUED;
    bool released = false;
    int status = ISM_OK;
    std::string error;
    Clock::time_point t_submit, t_launch, t_done;
    Batch *batch = nullptr;
    int64_t h_off = 0, y_off = 0, src_off = 0;  // element offsets in the block
    int64_t y_len = 0;
};

struct Batch {
    int slot;
    char *block = nullptr;
    int64_t bytes = 0;
    cudaEvent_t done = nullptr;
    cudaEvent_t start = nullptr;      // timing: recorded before the batch's first copy
    long long *stats_host = nullptr;  // stats_block.ptr
    PinnedPool::Block stats_block;
    int64_t n_rirs = 0;
    int64_t mic_samples = 0;
    std::vector<std::shared_ptr<Req>> reqs;
    int refs = 0;
    bool complete = false;
};

int64_t align_elems(int64_t n) { return (n + 63) & ~int64_t(63); }

}  // namespace

struct ism_server {
    ism_serve_config cfg;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> queue;
    std::unordered_map<uint64_t, std::shared_ptr<Req>> reqs;
    std::vector<std::unique_ptr<Batch>> batches;  // in flight or awaiting release
    std::vector<cudaStream_t> streams;
    std::vector<bool> slot_busy;
    uint64_t next_ticket = 1;
    int64_t outstanding = 0;  // submitted, not released
    bool stop = false;
    bool dev_ok = false, dev_failed = false;
    std::string dev_error;
    ism_serve_stats st;
    std::thread th;

    int64_t bytes_in_use = 0;
    PinnedPool pool;                     // sources and statistics readbacks
    std::vector<cudaEvent_t> free_events;  // completion events for reuse (mu)
    std::vector<cudaEvent_t> free_timing;  // timing events for reuse (mu)

    void loop();
    bool setup_device();
    void launch(std::vector<std::shared_ptr<Req>> &take);
    void finish_batches();
    void free_released();
};

bool ism_server::setup_device() {
    if (dev_ok) return true;
    if (dev_failed) return false;
    cudaError_t e = cudaSetDevice(cfg.device);
    if (e == cudaSuccess) {
        for (int i = 0; i < cfg.n_streams && e == cudaSuccess; ++i) {
            cudaStream_t s;
            e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e == cudaSuccess) streams.push_back(s);
        }
    }
    if (e != cudaSuccess) {
        dev_failed = true;
        dev_error = std::string("device ") + std::to_string(cfg.device) + ": " +
                    cudaGetErrorString(e);
        cudaGetLastError();
        return false;
    }
    slot_busy.assign(streams.size(), false);
    dev_ok = true;
    return true;
}

static int64_t req_bytes(const ism_request &r) {
    const int64_t M = r.room.n_mics, L = r.room.rir_len, T = r.src_len;
    return 4 * (align_elems(M * L) + align_elems(T) + align_elems(M * (T + L - 1))) +
           16 * M + 4096;
}

void ism_server::launch(std::vector<std::shared_ptr<Req>> &take) {
    // called with mu held; drops it around CUDA work
    NvtxRange nr("ism.serve.batch");
    const auto t_host0 = Clock::now();
    int slot = -1;
    for (size_t i = 0; i < slot_busy.size(); ++i)
        if (!slot_busy[i]) { slot = (int)i; break; }
    auto b = std::make_unique<Batch>();
    b->slot = slot;
    int64_t off = 0, n_rirs = 0;
    for (auto &r : take) {
        const int64_t M = r->room.n_mics, L = r->room.rir_len, T = r->src_len;
        r->h_off = off; off += align_elems(M * L);
        r->src_off = off; off += align_elems(T);
        r->y_off = off; r->y_len = T + L - 1; off += align_elems(M * r->y_len);
        n_rirs += M;
        b->mic_samples += M * r->y_len;
        r->state = RUNNING;
        r->t_launch = Clock::now();
        r->batch = b.get();
        b->bytes += r->bytes;
    }
    const int64_t stats_off = off;
    off += align_elems(2 * 2 * n_rirs);  // int64 pairs, counted in floats
    b->n_rirs = n_rirs;
    b->reqs = take;
    b->refs = (int)take.size();
    slot_busy[slot] = true;
    bytes_in_use += b->bytes;
    st.bytes_in_use = bytes_in_use;
    st.bytes_peak = std::max(st.bytes_peak, bytes_in_use);
    st.batches++;
    st.in_flight += (int64_t)take.size();
    st.queued -= (int64_t)take.size();
    Batch *bp = b.get();
    batches.push_back(std::move(b));
    mu.unlock();

    cudaStream_t s = streams[slot];
    int status = ISM_OK;
    std::string err;
    auto cerr = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && status == ISM_OK) {
            status = ISM_ERR_CUDA;
            err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    void *blk = nullptr;
    if (take_injection(ISM_INJECT_SERVE_ALLOC)) {  // test aid: the allocator fails
        status = ISM_ERR_OUT_OF_MEMORY;
        err = "device block of the batch (injected allocation failure)";
    } else if (int st2 = scratch_alloc(&blk, (size_t)off * 4, s)) {
        status = st2;
        err = ism_last_error_string();
    }
    bp->block = (char *)blk;
    float *base = (float *)blk;
    if (status == ISM_OK) {
        bp->stats_block = pool.get(16 * n_rirs + 16);
        bp->stats_host = (long long *)bp->stats_block.ptr;
        if (!bp->stats_host) {
            status = ISM_ERR_OUT_OF_MEMORY;
            err = "statistics readback buffer";
        }
    }
    if (status == ISM_OK) {
        {
            std::lock_guard<std::mutex> lk2(mu);
            if (!free_events.empty()) {
                bp->done = free_events.back();
                free_events.pop_back();
            }
        }
        if (!bp->done) cerr(cudaEventCreateWithFlags(&bp->done, 0), "event");
        {
            std::lock_guard<std::mutex> lk2(mu);
            if (!free_timing.empty()) {
                bp->start = free_timing.back();
                free_timing.pop_back();
            }
        }
        if (!bp->start && status == ISM_OK)
            cerr(cudaEventCreateWithFlags(&bp->start, 0), "event");
        if (status == ISM_OK) cerr(cudaEventRecord(bp->start, s), "event record");
    }
    if (status == ISM_OK) {
        for (auto &r : take)
            cerr(cudaMemcpyAsync(base + r->src_off, r->src_pinned, 4 * r->src_len,
                                 cudaMemcpyHostToDevice, s), "source upload");
        cerr(cudaMemsetAsync(base + stats_off, 0, 16 * n_rirs, s), "stats memset");
    }
    if (status == ISM_OK) {
        std::vector<ism_room> rooms;
        std::vector<int64_t> hoffs;
        std::vector<ism_conv_job> jobs;
        for (auto &r : take) {
            ism_room rm = r->room;
            rm.mics = r->mics.data();
            rooms.push_back(rm);
            for (int m = 0; m < rm.n_mics; ++m) hoffs.push_back(r->h_off + (int64_t)m * rm.rir_len);
            ism_conv_job j;
            memset(&j, 0, sizeof(j));
            j.n_mics = rm.n_mics;
            j.rir_len = rm.rir_len;
            j.src_len = r->src_len;
            j.h_offset = r->h_off;
            j.src_offset = r->src_off;
            j.y_offset = r->y_off;
            j.snr_db = r->snr_db;
            j.noise_id = r->noise_id ? r->noise_id : r->ticket;
            jobs.push_back(j);
        }
        ism_rir_opts o;
        memset(&o, 0, sizeof(o));
        o.window = 1024;  // fixed: the same work items whatever the mix
        o.stats_dev = (int64_t *)(base + stats_off);
        int rc = ism_rir_batch_ex(rooms.data(), (int64_t)rooms.size(), base, hoffs.data(), &o, s);
        if (rc == ISM_OK)
            rc = convolve_batch(jobs.data(), (int64_t)jobs.size(), base, base, base, cfg.seed,
                                cfg.precision, s);
        if (rc != ISM_OK) {
            status = rc;
            err = ism_last_error_string();
        }
    }
    if (status == ISM_OK) {
        cerr(cudaMemcpyAsync(bp->stats_host, base + stats_off, 16 * n_rirs,
                             cudaMemcpyDeviceToHost, s), "stats readback");
        cerr(cudaEventRecord(bp->done, s), "event record");
    }
    mu.lock();
    st.launch_host_ns +=
        std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t_host0).count();
    if (status != ISM_OK) {
        // the batch failed to launch: its requests fail, its memory is freed
        // once every launched operation on the stream has finished
        cudaStreamSynchronize(s);
        cudaGetLastError();
        for (auto &r : take) {
            r->state = FAILED;
            r->status = status;
            r->error = err;
            r->t_done = Clock::now();
        }
        bp->complete = true;
        slot_busy[slot] = false;
        st.in_flight -= (int64_t)take.size();
        cv_done.notify_all();
    }
}

void ism_server::finish_batches() {
    // called with mu held
    for (auto &b : batches) {
        if (b->complete) continue;
        cudaError_t e = cudaEventQuery(b->done);
        if (e == cudaErrorNotReady) continue;
        const auto now = Clock::now();
        // kernel errors of the batch's convolution (its status cell; the
        // slot's stream runs one batch at a time)
        int kst = ISM_OK;
        std::string kmsg;
        if (e == cudaSuccess) {
            kst = status_collect(streams[b->slot], false);
            if (kst) kmsg = std::string("batch failed: ") + ism_last_error_string();
        }
        for (auto &r : b->reqs) {
            if (e == cudaSuccess && kst == ISM_OK) {
                r->state = DONE;
            } else if (e == cudaSuccess) {
                r->state = FAILED;
                r->status = kst;
                r->error = kmsg;
            } else {
                r->state = FAILED;
                r->status = ISM_ERR_CUDA;
                r->error = std::string("batch failed: ") + cudaGetErrorString(e);
            }
            r->t_done = now;
        }
        if (e == cudaSuccess && kst == ISM_OK) {
            for (int64_t i = 0; i < b->n_rirs; ++i) st.taps += b->stats_host[2 * i + 1];
            st.mic_samples += b->mic_samples;
            float ms = 0.f;
            if (b->start && cudaEventElapsedTime(&ms, b->start, b->done) == cudaSuccess)
                st.batch_device_ns += (int64_t)(1e6 * (double)ms);
        }
        cudaGetLastError();
        b->complete = true;
        slot_busy[b->slot] = false;
        st.completed += (int64_t)b->reqs.size();
        st.in_flight -= (int64_t)b->reqs.size();
        cv_done.notify_all();
    }
}

void ism_server::free_released() {
    // called with mu held: free the memory of batches whose requests are
    // all released (and that are complete)
    for (size_t i = 0; i < batches.size();) {
        Batch *b = batches[i].get();
        if (b->complete && b->refs == 0) {
            if (b->block) scratch_free(b->block, streams[b->slot]);
            pool.put(b->stats_block);
            if (b->done) free_events.push_back(b->done);
            if (b->start) free_timing.push_back(b->start);
            bytes_in_use -= b->bytes;
            st.bytes_in_use = bytes_in_use;
            batches.erase(batches.begin() + i);
        } else {
            ++i;
        }
    }
}

void ism_server::loop() {
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        if (stop && queue.empty()) {
            bool busy = false;
            for (auto &b : batches) busy |= !b->complete;
            if (!busy) break;
        }
        if (!queue.empty() && !setup_device()) {
            // no usable device: fail everything waiting
            while (!queue.empty()) {
                auto r = queue.front();
                queue.pop_front();
                r->state = FAILED;
                r->status = ISM_ERR_CUDA;
                r->error = dev_error;
                r->t_done = Clock::now();
                st.queued--;
            }
            cv_done.notify_all();
        }
        if (dev_ok) {
            finish_batches();
            free_released();
            // admit the FIFO head while memory and a slot allow
            bool slot = std::find(slot_busy.begin(), slot_busy.end(), false) != slot_busy.end();
            if (slot && !queue.empty()) {
                std::vector<std::shared_ptr<Req>> take;
                int64_t avail = cfg.max_hbm_bytes - bytes_in_use;
                while (!queue.empty() && (int)take.size() < cfg.max_batch &&
                       queue.front()->bytes <= avail) {
                    avail -= queue.front()->bytes;
                    take.push_back(queue.front());
                    queue.pop_front();
                }
                if (!take.empty()) {
                    launch(take);
                    continue;
                }
            }
        }
        bool inflight = false;
        for (auto &b : batches) inflight |= !b->complete;
        if (inflight)
            cv_work.wait_for(lk, std::chrono::microseconds(50));
        else
            cv_work.wait_for(lk, std::chrono::milliseconds(20));
    }
}

extern "C" {

int ism_serve_create(const ism_serve_config *config, ism_server **out) {
    set_error("");
    if (!config || !out) return fail(ISM_ERR_INVALID_ARG, "NULL config or out");
    ism_serve_config c = *config;
    if (c.max_hbm_bytes < 0 || c.max_batch < 0 || c.n_streams < 0 || c.max_queue < 0)
        return fail(ISM_ERR_INVALID_ARG, "negative config value");
    if (c.precision != ISM_F32 && c.precision != ISM_BF16X3)
        return fail(ISM_ERR_INVALID_ARG, "unknown precision");
    if (c.max_hbm_bytes == 0) c.max_hbm_bytes = (int64_t)8 << 30;
    if (c.max_batch == 0) c.max_batch = 64;
    if (c.n_streams == 0) c.n_streams = 2;
    if (c.n_streams > 16) return fail(ISM_ERR_INVALID_ARG, "n_streams above 16");
    if (c.max_queue == 0) c.max_queue = 4096;
    auto *s = new ism_server();
    s->cfg = c;
    memset(&s->st, 0, sizeof(s->st));
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return ISM_OK;
}

int ism_serve_submit(ism_server *s, const ism_request *rq, uint64_t *ticket) {
    set_error("");
    if (!s || !rq || !ticket) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    if (int st = validate_room(rq->room, 0)) return st;
    if (rq->src_len < 1 || !rq->src_host) return fail(ISM_ERR_INVALID_ARG, "empty source");
    if (rq->src_len > kMaxSignal) return fail(ISM_ERR_INVALID_ARG, "src_len above 2^40");
    if (!isnan(rq->snr_db) && !isfinite(rq->snr_db))
        return fail(ISM_ERR_INVALID_ARG, "snr must be finite or NaN");
    const int64_t bytes = req_bytes(*rq);
    auto r = std::make_shared<Req>();
    r->room = rq->room;
    r->mics.assign(rq->room.mics, rq->room.mics + 3 * rq->room.n_mics);
    r->room.mics = nullptr;
    r->src_len = rq->src_len;
    r->snr_db = rq->snr_db;
    r->noise_id = rq->noise_id;
    r->bytes = bytes;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (bytes > s->cfg.max_hbm_bytes) {
            s->st.rejected_busy++;
            return fail(ISM_ERR_BUSY, "request needs more device memory than the server may hold");
        }
        if (s->outstanding >= s->cfg.max_queue) {
            s->st.rejected_busy++;
            return fail(ISM_ERR_BUSY, "too many outstanding requests");
        }
        if (s->stop) return fail(ISM_ERR_BUSY, "server is stopping");
    }
    // page-locked copy of the source (host memory only; no device needed)
    r->src_block = s->pool.get((size_t)4 * rq->src_len);
    r->src_pinned = (float *)r->src_block.ptr;
    if (!r->src_pinned) return fail(ISM_ERR_OUT_OF_MEMORY, "host source copy");
    memcpy(r->src_pinned, rq->src_host, 4 * rq->src_len);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->ticket = s->next_ticket++;
        r->t_submit = Clock::now();
        s->reqs[r->ticket] = r;
        s->queue.push_back(r);
        s->outstanding++;
        s->st.submitted++;
        s->st.queued++;
        *ticket = r->ticket;
    }
    s->cv_work.notify_one();
    return ISM_OK;
}

static int fill_result(const Req &r, ism_result *out) {
    if (r.state == FAILED) return fail(r.status, r.error);
    if (r.state != DONE) return ISM_PENDING;
    if (out) {
        memset(out, 0, sizeof(*out));
        float *base = (float *)r.batch->block;
        out->h_dev = base + r.h_off;
        out->y_dev = base + r.y_off;
        out->n_mics = r.room.n_mics;
        out->rir_len = r.room.rir_len;
        out->y_len = r.y_len;
        out->queue_s = std::chrono::duration<double>(r.t_launch - r.t_submit).count();
        out->latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
    }
    return ISM_OK;
}

int ism_serve_poll(ism_server *s, uint64_t ticket, ism_result *out) {
    if (!s) return fail(ISM_ERR_INVALID_ARG, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(ISM_ERR_UNKNOWN_TICKET, "unknown ticket");
    return fill_result(*it->second, out);
}

int ism_serve_wait(ism_server *s, uint64_t ticket, double timeout_s, ism_result *out) {
    if (!s) return fail(ISM_ERR_INVALID_ARG, "NULL server");
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(ISM_ERR_UNKNOWN_TICKET, "unknown ticket");
        int st = fill_result(*it->second, out);
        if (st != ISM_PENDING) return st;
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            it = s->reqs.find(ticket);
            if (it != s->reqs.end() && fill_result(*it->second, out) != ISM_PENDING)
                return fill_result(*it->second, out);
            return fail(ISM_ERR_TIMEOUT, "wait deadline passed");
        }
    }
}

int ism_serve_copy(ism_server *s, uint64_t ticket, float *h_out, float *y_out, void *stream) {
    if (!s) return fail(ISM_ERR_INVALID_ARG, "NULL server");
    ism_result r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(ISM_ERR_UNKNOWN_TICKET, "unknown ticket");
        const int st = fill_result(*it->second, &r);
        if (st != ISM_OK) return st;
    }
    cudaStream_t cs = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (h_out)
        e = cudaMemcpyAsync(h_out, r.h_dev, sizeof(float) * r.n_mics * r.rir_len, cudaMemcpyDefault,
                            cs);
    if (e == cudaSuccess && y_out)
        e = cudaMemcpyAsync(y_out, r.y_dev, sizeof(float) * r.n_mics * r.y_len, cudaMemcpyDefault,
                            cs);
    if (e != cudaSuccess) return cuda_fail(e, "ism_serve_copy");
    return ISM_OK;
}

int ism_serve_release(ism_server *s, uint64_t ticket) {
    if (!s) return fail(ISM_ERR_INVALID_ARG, "NULL server");
    std::shared_ptr<Req> r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->reqs.find(ticket);
        if (it == s->reqs.end()) return fail(ISM_ERR_UNKNOWN_TICKET, "unknown ticket");
        r = it->second;
        if (r->state == QUEUED || r->state == RUNNING) return ISM_PENDING;
        s->reqs.erase(it);
        s->outstanding--;
        if (r->batch) r->batch->refs--;
    }
    s->cv_work.notify_one();
    s->pool.put(r->src_block);
    r->src_block = PinnedPool::Block{};
    r->src_pinned = nullptr;
    return ISM_OK;
}

int ism_serve_stats_get(ism_server *s, ism_serve_stats *out) {
    if (!s || !out) return fail(ISM_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    return ISM_OK;
}

int ism_serve_destroy(ism_server *s) {
    if (!s) return fail(ISM_ERR_INVALID_ARG, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        // requests never launched fail now
        for (auto &r : s->queue) {
            r->state = FAILED;
            r->status = ISM_ERR_BUSY;
            r->error = "server destroyed";
        }
        s->queue.clear();
    }
    s->cv_work.notify_all();
    s->th.join();
    for (auto &b : s->batches) {
        if (b->block) scratch_free(b->block, s->streams[b->slot]);
        s->pool.put(b->stats_block);
        if (b->done) cudaEventDestroy(b->done);
        if (b->start) cudaEventDestroy(b->start);
    }
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t e : s->free_events) cudaEventDestroy(e);
    for (cudaEvent_t e : s->free_timing) cudaEventDestroy(e);
    for (auto &kv : s->reqs) s->pool.put(kv.second->src_block);
    delete s;  // frees the cached page-locked blocks
    return ISM_OK;
}

}  // extern "C"
