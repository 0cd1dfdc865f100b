// ism_noalloc.cu -- ism_rir_batch_noalloc: the RIR batch without any
// allocation.
//
// Some callers cannot allocate device memory when they compute RIRs: their
// device memory is already reserved by another allocator (a framework's
// caching allocator that owns the whole GPU), or they run in a latency-bound
// loop where cudaMalloc's implicit synchronisation and unbounded cost are not
// acceptable.  This entry point runs the same image-source kernel as
// ism_rir_batch, but its scratch (the per-RIR job table and the work
// counters) lives in the fixed device array below instead of a stream-ordered
// allocation, and the job table reaches the device as the kernel arguments of
// small store kernels (chunks of kChunk jobs, by value) instead of through a
// pinned staging block, so no host memory is read after the call returns.  It
// calls no cudaMalloc, cudaFree, cudaHostAlloc or other allocating routine.
//
// The array is a file-scope __device__ symbol: every GPU that loads this
// library holds its 2 MiB until the process exits.  In host code its name is
// only a host-side stand-in, so its device address is taken once per device
// (cudaGetSymbolAddress, with that device current) on the first call made on
// that device; make that first call before any stream capture.  Every call
// shares the array and it keeps the last call's contents: the counters are
// cleared at the start of each call, and calls that overlap on the GPU (on
// different streams) race on it, so serialise them.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "ism_internal.h"

using namespace ism;

namespace {

constexpr size_t kScratchBytes = size_t(2) << 20;  // 2 MiB
constexpr size_t kCounterBytes = 256;              // one counter per filter kind
static_assert(kCounterBytes + (size_t)ISM_NOALLOC_MAX_RIRS * sizeof(RirJob) <= kScratchBytes,
              "the fixed scratch must hold ISM_NOALLOC_MAX_RIRS jobs");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices];

// Device address of the fixed scratch on the current device (taken once).
int scratch_address(unsigned char **out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (d < 0 || d >= kMaxDevices) return fail(ISM_ERR_INTERNAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[d]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(fixed scratch)");
        g_scratch_addr[d] = (unsigned char *)p;
    }
    *out = g_scratch_addr[d];
    return ISM_OK;
}

constexpr int kChunk = 128;  // jobs per store kernel (18 KB of kernel arguments)

// One chunk of the job table, passed by value as a kernel argument.
struct JobChunk {
    RirJob job[kChunk];
};
static_assert(sizeof(JobChunk) + 64 <= 32764, "kernel argument limit");

// Writes n jobs of a chunk to dst; the first chunk of a launch also clears
// the work counter of the image-source kernel that follows.
__global__ void __launch_bounds__(kChunk)
k_store_jobs(RirJob *__restrict__ dst, const __grid_constant__ JobChunk chunk, int n,
             unsigned int *__restrict__ counter) {
    const int i = threadIdx.x;
    if (i < n) dst[i] = chunk.job[i];
    if (counter && i == 0) *counter = 0u;
}

}  // namespace

extern "C" int ism_rir_batch_noalloc(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                                     const int64_t *h_offsets, void *stream_v) {
    set_error("");
    if (n_rooms < 0) return fail(ISM_ERR_INVALID_ARG, "n_rooms < 0");
    if (n_rooms == 0) return ISM_OK;
    if (!rooms || !h_dev) return fail(ISM_ERR_INVALID_ARG, "NULL rooms or h_dev");
    cudaStream_t stream = (cudaStream_t)stream_v;
    for (int64_t r = 0; r < n_rooms; ++r)
        if (int st = validate_room(rooms[r], r)) return st;
    const int W = auto_window(rooms, n_rooms);  // ism_rir_batch's default windows

    int64_t count[2] = {0, 0};
    int max_order[2] = {0, 0}, max_taps[2] = {1, 1}, wmax[2] = {0, 0};
    for (int64_t r = 0; r < n_rooms; ++r) {
        const ism_room &R = rooms[r];
        const int k = R.fd_kind;
        count[k] += R.n_mics;
        for (int m = 0; m < R.n_mics; ++m) max_order[k] = std::max(max_order[k], room_order(R, m));
        max_taps[k] = std::max(max_taps[k], R.n_taps);
        wmax[k] = std::max(wmax[k], (int)((R.rir_len + W - 1) / W));
    }
    if (count[0] + count[1] > ISM_NOALLOC_MAX_RIRS)
        return fail(ISM_ERR_INVALID_ARG,
                    "ism_rir_batch_noalloc: " + std::to_string(count[0] + count[1]) +
                        " RIRs exceed its fixed scratch of " +
                        std::to_string(ISM_NOALLOC_MAX_RIRS) + " RIRs per call");
    for (int k = 0; k < 2; ++k)
        if (count[k] && rir_smem_bytes(W, max_order[k], max_taps[k]) > kMaxDynSmem)
            return fail(ISM_ERR_INVALID_ARG, "window/order/taps need too much shared memory");

    if (h_offsets) {  // checked before anything is launched
        const int64_t n_rirs = count[0] + count[1];
        for (int64_t j = 0; j < n_rirs; ++j)
            if (h_offsets[j] < 0) return fail(ISM_ERR_INVALID_ARG, "negative h offset");
    }

    unsigned char *base = nullptr;
    if (int st = scratch_address(&base)) return st;
    RirJob *jobs_dev[2] = {(RirJob *)(base + kCounterBytes),
                           (RirJob *)(base + kCounterBytes) + count[0]};
    unsigned int *counter_dev[2] = {(unsigned int *)base, (unsigned int *)(base + 16)};

    // job tables, chunk by chunk as kernel arguments (the counter of kind k
    // is cleared by its first chunk)
    JobChunk buf;
    for (int k = 0; k < 2; ++k) {
        if (!count[k]) continue;
        int64_t j = 0, packed = 0, done = 0;
        int nb = 0;
        auto store = [&]() -> int {
            k_store_jobs<<<1, kChunk, 0, stream>>>(jobs_dev[k] + done, buf, nb,
                                                    done == 0 ? counter_dev[k] : nullptr);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "launch k_store_jobs");
            done += nb;
            nb = 0;
            return ISM_OK;
        };
        for (int64_t r = 0; r < n_rooms; ++r) {
            const ism_room &R = rooms[r];
            for (int m = 0; m < R.n_mics; ++m, ++j) {
                const int64_t off = h_offsets ? h_offsets[j] : packed;
                packed += R.rir_len;
                if (R.fd_kind != k) continue;
                RirJob &J = buf.job[nb++];
                memset(&J, 0, sizeof(J));
                for (int a = 0; a < 3; ++a) {
                    J.src[a] = R.src[a];
                    J.mic[a] = R.mics[3 * m + a];
                    J.dims[a] = R.dims[a];
                }
                J.q = R.fs / R.c;
                for (int w = 0; w < 6; ++w) J.beta[w] = (float)R.beta[w];
                J.order = room_order(R, m);
                J.n_taps = R.n_taps;
                J.fd_kind = k;
                J.rir_len = R.rir_len;
                J.n_windows = (int32_t)((R.rir_len + W - 1) / W);
                J.h_offset = off;
                J.stat_index = j;
                if (nb == kChunk)
                    if (int st = store()) return st;
            }
        }
        if (nb)
            if (int st = store()) return st;
        RirLaunch L{jobs_dev[k], (int)count[k], wmax[k], W, max_order[k], max_taps[k], k,
                    h_dev, nullptr, counter_dev[k], nullptr, 0};
        if (int st = launch_rir(L, stream)) return st;
    }
    return ISM_OK;
}
