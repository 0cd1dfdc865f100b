// ism_status.cu -- kernel status of asynchronous calls.
//
// The tensor-core convolution kernels bound every wait (see
// ism_conv_tc.cu): a wait that runs out makes the kernel stop, write zeros
// for the outputs it did not finish and set the call's status cell.  The cell
// is an int in page-locked, device-mapped host memory, so the kernel's store
// needs no copy back: once the event the call recorded after its launches
// has completed, the host reads it.  Failed calls are remembered per
// (device, stream) until reported: by ism_stream_status, by the next
// ism_convolve_batch on the stream, by ism_dataset_batch (which waits for its
// streams) and by the server (which reads its batch's cells when the batch's
// completion event fires).
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "ism_internal.h"

namespace ism {
namespace {

constexpr int kMaxDev = 64;
constexpr int kCellsPerPage = 1024;  // one 4 KiB page of ints

struct Pending {
    int device;
    cudaStream_t stream;
    int cell;
    cudaEvent_t ev;
    bool owned;  // the cell belongs to a plan: read and cleared, not freed
};

std::mutex g_mu;
std::vector<int *> g_pages[kMaxDev];   // host addresses (device-mapped)
std::vector<int *> g_dpages[kMaxDev];  // the same pages' device addresses
std::vector<int> g_free[kMaxDev];
std::vector<cudaEvent_t> g_events[kMaxDev];
std::vector<Pending> g_pending;
std::map<std::pair<int, cudaStream_t>, int> g_failed;  // failed calls not yet reported
std::atomic<int> g_inject{0};

int *host_cell(int device, int cell) { return g_pages[device][cell / kCellsPerPage] + cell % kCellsPerPage; }

// Moves every completed call into g_failed (when its cell is set) and frees
// its cell and event.  Called with g_mu held.
void reap_locked() {
    for (size_t i = 0; i < g_pending.size();) {
        Pending &p = g_pending[i];
        const cudaError_t q = cudaEventQuery(p.ev);
        if (q == cudaErrorNotReady) {
            cudaGetLastError();
            ++i;
            continue;
        }
        // completed (or failed with a CUDA error, which the caller's own
        // synchronisation reports): read the cell
        if (q != cudaSuccess) cudaGetLastError();
        volatile int *c = host_cell(p.device, p.cell);
        if (*c) g_failed[{p.device, p.stream}]++;
        *c = 0;
        if (!p.owned) g_free[p.device].push_back(p.cell);
        g_events[p.device].push_back(p.ev);
        g_pending[i] = g_pending.back();
        g_pending.pop_back();
    }
}

int current_device(int *d) {
    cudaError_t e = cudaGetDevice(d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (*d < 0 || *d >= kMaxDev) return fail(ISM_ERR_INTERNAL, "device ordinal out of range");
    return ISM_OK;
}

}  // namespace

int status_begin(StatusTicket *t) {
    int d = 0;
    if (int st = current_device(&d)) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_free[d].empty()) {
        void *p = nullptr;
        cudaError_t e = cudaHostAlloc(&p, kCellsPerPage * sizeof(int),
                                      cudaHostAllocMapped | cudaHostAllocPortable);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(status cells)");
        void *dp = nullptr;
        e = cudaHostGetDevicePointer(&dp, p, 0);
        if (e != cudaSuccess) {
            cudaFreeHost(p);
            return cuda_fail(e, "cudaHostGetDevicePointer(status cells)");
        }
        const int base = (int)g_pages[d].size() * kCellsPerPage;
        g_pages[d].push_back((int *)p);
        g_dpages[d].push_back((int *)dp);
        for (int i = kCellsPerPage - 1; i >= 0; --i) {
            ((volatile int *)p)[i] = 0;
            g_free[d].push_back(base + i);
        }
    }
    t->device = d;
    t->cell = g_free[d].back();
    g_free[d].pop_back();
    *(volatile int *)host_cell(d, t->cell) = 0;
    t->dev = g_dpages[d][t->cell / kCellsPerPage] + t->cell % kCellsPerPage;
    return ISM_OK;
}

int status_end(const StatusTicket &t, cudaStream_t stream, bool ok, bool owned) {
    if (t.cell < 0) return ISM_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!ok) {  // nothing was enqueued with this cell
        if (!owned) g_free[t.device].push_back(t.cell);
        return ISM_OK;
    }
    cudaEvent_t ev = nullptr;
    if (!g_events[t.device].empty()) {
        ev = g_events[t.device].back();
        g_events[t.device].pop_back();
    } else {
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            // the kernels are enqueued: keep the cell out of use (it may
            // still be written) and report the failure
            return cuda_fail(e, "cudaEventCreate(status)");
        }
    }
    cudaError_t e = cudaEventRecord(ev, stream);
    if (e != cudaSuccess) {
        g_events[t.device].push_back(ev);
        return cuda_fail(e, "cudaEventRecord(status)");
    }
    g_pending.push_back(Pending{t.device, stream, t.cell, ev, owned});
    return ISM_OK;
}

void status_release(const StatusTicket &t) {
    if (t.cell < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    // the owner has waited for its work: reap its entries, then free the cell
    for (auto &p : g_pending)
        if (p.device == t.device && p.cell == t.cell && cudaEventSynchronize(p.ev) != cudaSuccess)
            cudaGetLastError();
    reap_locked();
    g_free[t.device].push_back(t.cell);
}

int status_collect(cudaStream_t stream, bool wait) {
    int d = 0;
    if (int st = current_device(&d)) return st;
    if (wait) {
        std::vector<cudaEvent_t> evs;
        {
            std::lock_guard<std::mutex> lk(g_mu);
            for (auto &p : g_pending)
                if (p.device == d && p.stream == stream) evs.push_back(p.ev);
        }
        // the events stay pending (not recycled) until reaped below
        for (cudaEvent_t ev : evs)
            if (cudaEventSynchronize(ev) != cudaSuccess) cudaGetLastError();
    }
    std::lock_guard<std::mutex> lk(g_mu);
    reap_locked();
    auto it = g_failed.find({d, stream});
    if (it == g_failed.end()) return ISM_OK;
    const int n = it->second;
    g_failed.erase(it);
    return fail(ISM_ERR_INTERNAL,
                std::to_string(n) + " earlier call(s) on this stream stopped a tensor-core "
                "convolution kernel after a wait ran out; their outputs are incomplete");
}

int take_injection(int what) {
    int cur = g_inject.load();
    while (cur & what)
        if (g_inject.compare_exchange_weak(cur, cur & ~what)) return 1;
    return 0;
}

}  // namespace ism

extern "C" int ism_stream_status(void *stream) {
    ism::set_error("");
    return ism::status_collect((cudaStream_t)stream, true);
}

extern "C" int ism_debug_bounds(uint32_t *flags) {
    ism::set_error("");
    if (!flags) return ism::fail(ISM_ERR_INVALID_ARG, "NULL flags");
    unsigned int f = 0u;
    if (int st = ism::oob_read_rir(&f)) return st;
    if (int st = ism::oob_read_conv(&f)) return st;
    if (int st = ism::oob_read_conv_tc(&f)) return st;
    *flags = f;
    return ISM_OK;
}

extern "C" int ism_debug_inject(int32_t what) {
    ism::set_error("");
    if (what != 0 && what != ISM_INJECT_CONV_WAIT && what != ISM_INJECT_SERVE_ALLOC)
        return ism::fail(ISM_ERR_INVALID_ARG, "unknown injection");
    if (what == 0) ism::g_inject.store(0);
    else ism::g_inject.fetch_or(what);
    return ISM_OK;
}
