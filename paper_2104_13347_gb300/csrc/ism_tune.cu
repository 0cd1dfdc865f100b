// ism_tune.cu -- the window autotuner of the image-source kernel.
//
// A call of ism_rir_batch_ex with window = ISM_WINDOW_TUNE takes the output
// window W (samples per work item) that ran fastest for its bucket.  The
// bucket of a call is what the best window depends on: the filter (kinds and
// tap counts present), the largest lattice order, the sampling rate, the
// RIR length (power-of-two class) and the batch size (power-of-two class of
// the RIR count), plus the kernel variant.  On the first call of a bucket the
// tuner runs the call itself once per candidate window (1 untimed + 2 timed
// runs each, CUDA events on the call's stream, the host waiting for them),
// keeps the fastest and runs the call a last time with it, so the outputs
// are those of the chosen window.  Choices are kept for the process and,
// when the environment variable ISM_TUNE_CACHE names a file, appended to it
// and read back by later processes: a bucket tuned once keeps its window, so
// its RIRs stay bitwise reproducible (the sparse path's fixed-point scale is
// per window).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "ism_internal.h"

namespace ism {
namespace {

struct TuneKey {
    int variant, kinds, taps0, taps1, order, fs, len2, rirs2;
    bool operator<(const TuneKey &o) const {
        const int a[8] = {variant, kinds, taps0, taps1, order, fs, len2, rirs2};
        const int b[8] = {o.variant, o.kinds, o.taps0, o.taps1, o.order, o.fs, o.len2, o.rirs2};
        return std::lexicographical_compare(a, a + 8, b, b + 8);
    }
};

std::mutex g_mu;
std::map<TuneKey, int> g_table;
std::set<std::string> g_loaded;  // cache files read so far

int ceil_log2(int64_t x) {
    int k = 0;
    while (((int64_t)1 << k) < x) ++k;
    return k;
}
int floor_log2(int64_t x) {
    int k = 0;
    while (((int64_t)2 << k) <= x) ++k;
    return k;
}

TuneKey make_key(const ism_room *rooms, int64_t n_rooms, int variant) {
    TuneKey k{variant, 0, 0, 0, 0, 0, 0, 0};
    int64_t n_rirs = 0, max_len = 1;
    double fs = 0.0;
    for (int64_t r = 0; r < n_rooms; ++r) {
        const ism_room &R = rooms[r];
        k.kinds |= 1 << R.fd_kind;
        if (R.fd_kind == ISM_FD_HANN_SINC) k.taps0 = std::max(k.taps0, R.n_taps);
        else k.taps1 = std::max(k.taps1, R.n_taps);
        for (int m = 0; m < R.n_mics; ++m) k.order = std::max(k.order, room_order(R, m));
        n_rirs += R.n_mics;
        max_len = std::max(max_len, R.rir_len);
        fs = std::max(fs, R.fs);
    }
    k.fs = (int)lrint(fs);
    k.len2 = ceil_log2(max_len);
    k.rirs2 = floor_log2(std::max<int64_t>(n_rirs, 1));
    return k;
}

const char *cache_path() {
    const char *p = getenv("ISM_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

// Reads the cache file once per path (with g_mu held).  Lines:
//   ism-tune 1 <variant> <kinds> <taps0> <taps1> <order> <fs> <len2> <rirs2> <window> <ms>
void load_locked() {
    const char *p = cache_path();
    if (!p || g_loaded.count(p)) return;
    g_loaded.insert(p);
    FILE *f = fopen(p, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        TuneKey k;
        int ver = 0, w = 0;
        double ms = 0.0;
        if (sscanf(line, "ism-tune %d %d %d %d %d %d %d %d %d %d %lf", &ver, &k.variant, &k.kinds,
                   &k.taps0, &k.taps1, &k.order, &k.fs, &k.len2, &k.rirs2, &w, &ms) == 11 &&
            ver == 1 && w >= 32 && w <= 8192 && w % 32 == 0)
            g_table[k] = w;  // a later line for the same bucket wins
    }
    fclose(f);
}

void store_locked(const TuneKey &k, int w, double ms) {
    g_table[k] = w;
    const char *p = cache_path();
    if (!p) return;
    FILE *f = fopen(p, "a");
    if (!f) return;  // the choice still holds for this process
    fprintf(f, "ism-tune 1 %d %d %d %d %d %d %d %d %d %.6f\n", k.variant, k.kinds, k.taps0,
            k.taps1, k.order, k.fs, k.len2, k.rirs2, w, ms);
    fclose(f);
}

int lookup(const TuneKey &k) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_locked();
    auto it = g_table.find(k);
    return it == g_table.end() ? 0 : it->second;
}

}  // namespace

int rir_window_tuned(const ism_room *rooms, int64_t n_rooms, int variant) {
    return lookup(make_key(rooms, n_rooms, variant));
}

int rir_batch_tuned(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                    const int64_t *h_offsets, const ism_rir_opts &opts, cudaStream_t stream) {
    const TuneKey key = make_key(rooms, n_rooms, opts.variant);
    ism_rir_opts o = opts;
    int W = lookup(key);
    if (W > 0) {
        o.window = W;
        return ism_rir_batch_ex(rooms, n_rooms, h_dev, h_offsets, &o, (void *)stream);
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(stream, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return fail(ISM_ERR_INVALID_ARG,
                    "ISM_WINDOW_TUNE: this bucket is not tuned yet, and tuning cannot run "
                    "while the stream is being captured");
    // candidates: the automatic window and the usual batch windows, limited
    // to twice the longest RIR
    int64_t max_len = 1;
    for (int64_t r = 0; r < n_rooms; ++r) max_len = std::max(max_len, rooms[r].rir_len);
    std::vector<int> cand = {auto_window(rooms, n_rooms), 256, 512, 768, 1024, 1536, 2048};
    if (cand[0] < 256) {
        cand.push_back(64);
        cand.push_back(128);
    }
    const int64_t cap_w = std::max<int64_t>(64, ((2 * max_len + 31) / 32) * 32);
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    cudaEvent_t ev[2];
    if ((e = cudaEventCreate(&ev[0])) != cudaSuccess) return cuda_fail(e, "cudaEventCreate(tune)");
    if ((e = cudaEventCreate(&ev[1])) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return cuda_fail(e, "cudaEventCreate(tune)");
    }
    ism_rir_opts t = opts;
    t.stats_dev = nullptr;  // statistics accumulate: only the final run adds them
    int best = 0;
    float best_ms = 0.f;
    int st = ISM_OK;
    for (int w : cand) {
        if (w > cap_w && w != cand[0]) continue;
        t.window = w;
        // untimed run: kernel attributes, occupancy queries, caches
        int rc = ism_rir_batch_ex(rooms, n_rooms, h_dev, h_offsets, &t, (void *)stream);
        if (rc == ISM_ERR_INVALID_ARG) continue;  // this window does not fit the kernel
        if (rc) { st = rc; break; }
        cudaEventRecord(ev[0], stream);
        for (int i = 0; i < 2 && !rc; ++i)
            rc = ism_rir_batch_ex(rooms, n_rooms, h_dev, h_offsets, &t, (void *)stream);
        cudaEventRecord(ev[1], stream);
        if (rc) { st = rc; break; }
        if ((e = cudaEventSynchronize(ev[1])) != cudaSuccess) { st = cuda_fail(e, "tune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[0], ev[1]);
        ms *= 0.5f;
        if (!best || ms < best_ms) {
            best = w;
            best_ms = ms;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (st) return st;
    if (!best) return fail(ISM_ERR_INVALID_ARG, "no window fits the kernel for this batch");
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_locked();
        // another thread may have tuned the bucket meanwhile: keep its choice
        auto it = g_table.find(key);
        if (it != g_table.end()) best = it->second;
        else store_locked(key, best, best_ms);
    }
    o.window = best;
    return ism_rir_batch_ex(rooms, n_rooms, h_dev, h_offsets, &o, (void *)stream);
}

}  // namespace ism

extern "C" int ism_rir_tuned_window(const ism_room *rooms, int64_t n_rooms,
                                    const ism_rir_opts *opts, int32_t *window) {
    ism::set_error("");
    if (!window || n_rooms < 0 || (n_rooms > 0 && !rooms))
        return ism::fail(ISM_ERR_INVALID_ARG, "bad arguments");
    for (int64_t r = 0; r < n_rooms; ++r)
        if (int st = ism::validate_room(rooms[r], r)) return st;
    *window = n_rooms ? ism::rir_window_tuned(rooms, n_rooms, opts ? opts->variant : 0) : 0;
    return ISM_OK;
}
