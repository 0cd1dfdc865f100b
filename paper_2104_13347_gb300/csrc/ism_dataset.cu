// ism_dataset.cu -- the dataset step with host buffers (ism_dataset_batch):
// RIRs, convolution and noise for a batch of rooms, sources read from and
// microphone signals written to host memory, the copies of one chunk of
// rooms overlapping the kernels of the next (arXiv 2104.13347, Sec. II.A:
// the dataset is the batch convolution of recordings with the simulated
// RIRs).
//
// Pipeline over chunks k = 0, 1, ... with two device buffer sets (k mod 2)
// and four streams:
//   up:         [wait compute(k-2)] sources of chunk k -> src_d[k%2]
//   comp[k%2]:  [wait up(k), down(k-2)] RIRs -> h_d, convolution + noise -> y_d
//   down:       [wait comp(k)] y_d (and h_d) -> host
// Consecutive chunks compute on different streams, so the RIR kernel of
// chunk k+1 fills the SMs that the tail of chunk k's convolution leaves.
// Every kernel is the batch entry points' own (ism_rir_batch_ex,
// ism_convolve_batch); the RIR window is chosen once for the whole batch
// (ism_rir_batch's automatic rule over all rooms) and room i keeps noise id
// base + i, so the outputs do not depend on the chunking.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ism_internal.h"

using namespace ism;

namespace {

struct Pipe {
    cudaStream_t up = nullptr, comp[2] = {}, down = nullptr;
    cudaEvent_t ev_alloc = nullptr, ev_comp1 = nullptr, up_done[2] = {}, comp_done[2] = {},
                down_done[2] = {};
    void *buf = nullptr;
    ~Pipe() {
        // every stream is synchronised before the pipe goes out of scope;
        // the buffer is freed on comp[0] after comp[1]'s work
        if (buf && comp[0]) {
            if (comp[1] && ev_comp1) {
                cudaEventRecord(ev_comp1, comp[1]);
                cudaStreamWaitEvent(comp[0], ev_comp1, 0);
            }
            scratch_free(buf, comp[0]);
        }
        for (int s = 0; s < 2; ++s)
            if (comp[s]) cudaStreamSynchronize(comp[s]);
        for (int s = 0; s < 2; ++s) {
            if (up_done[s]) cudaEventDestroy(up_done[s]);
            if (comp_done[s]) cudaEventDestroy(comp_done[s]);
            if (down_done[s]) cudaEventDestroy(down_done[s]);
        }
        if (ev_alloc) cudaEventDestroy(ev_alloc);
        if (ev_comp1) cudaEventDestroy(ev_comp1);
        if (up) cudaStreamDestroy(up);
        for (int s = 0; s < 2; ++s)
            if (comp[s]) cudaStreamDestroy(comp[s]);
        if (down) cudaStreamDestroy(down);
    }
};

int copy_async(void *dst, const void *src, size_t bytes, cudaMemcpyKind kind, cudaStream_t s) {
    if (!bytes) return ISM_OK;
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, s);
    return e == cudaSuccess ? ISM_OK : cuda_fail(e, "cudaMemcpyAsync");
}

}  // namespace

extern "C" int ism_dataset_batch(const ism_room *rooms, int64_t n_rooms, const float *src_host,
                                 const int64_t *src_lens, const int64_t *src_offsets,
                                 const float *snr_db, uint64_t seed, uint64_t noise_id_base,
                                 int32_t precision, float *y_host, const int64_t *y_offsets,
                                 float *h_host, const int64_t *h_offsets, int64_t chunk_rooms) {
    set_error("");
    if (n_rooms < 0) return fail(ISM_ERR_INVALID_ARG, "n_rooms < 0");
    if (n_rooms == 0) return ISM_OK;
    if (!rooms || !src_host || !src_lens || !y_host)
        return fail(ISM_ERR_INVALID_ARG, "NULL rooms, sources, lengths or outputs");
    if (precision != ISM_F32 && precision != ISM_BF16X3)
        return fail(ISM_ERR_INVALID_ARG, "unknown precision");
    if (chunk_rooms < 0) return fail(ISM_ERR_INVALID_ARG, "chunk_rooms < 0");
    // per-room sizes and host offsets
    std::vector<int64_t> so(n_rooms), yo(n_rooms), ho(n_rooms), ylen(n_rooms), hlen(n_rooms);
    int64_t sp = 0, yp = 0, hp = 0, y_total = 0;
    for (int64_t i = 0; i < n_rooms; ++i) {
        const ism_room &R = rooms[i];
        if (int st = validate_room(R, i)) return st;
        if (src_lens[i] < 1 || src_lens[i] > kMaxSignal)
            return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(i) + ": src_len must lie in [1, 2^40]");
        ylen[i] = (int64_t)R.n_mics * (src_lens[i] + R.rir_len - 1);
        hlen[i] = (int64_t)R.n_mics * R.rir_len;
        so[i] = src_offsets ? src_offsets[i] : sp;
        yo[i] = y_offsets ? y_offsets[i] : yp;
        ho[i] = h_offsets ? h_offsets[i] : hp;
        if (so[i] < 0 || yo[i] < 0 || ho[i] < 0)
            return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(i) + ": negative offset");
        sp += src_lens[i];
        yp += ylen[i];
        hp += hlen[i];
        y_total += ylen[i];
    }
    // chunks of consecutive rooms.  Automatic, split-BF16 (every room on the
    // persistent tensor-core convolution, one CTA per SM walking the chunk's
    // tiles): chunks cut at whole rounds of tiles over the SMs, so that no
    // chunk but the last ends with a partly filled round -- main chunks of R
    // rounds (R = rounds / 4.5, at most 9), then a chunk of R / 3 rounds and
    // the rest, which keeps the last chunk's download (the one copy nothing
    // hides) short.  1024 8-mic rooms with 1 s sources and 8192-sample RIRs
    // (40.4 rounds): 228, 228, 228, 228, 76 and 36 rooms, 12.55 ms end to end
    // against 13.3 ms (12.7-13.9 from call to call) for six chunks of six
    // rounds and the rest; chunks of 12 rounds, or not cut at whole rounds,
    // were slower still (13.2-13.6 ms).  FP32: K >= 6 chunks of about 128
    // MiB of signals each, balanced by signal length (ragged rooms).  With
    // two compute streams the tails of consecutive chunks overlap.
    std::vector<int64_t> cb;  // chunk boundaries
    const int64_t target = (128ll << 20) / 4;  // floats of signals per chunk
    const int64_t K = std::min<int64_t>(n_rooms,
                                        std::max<int64_t>((y_total + target - 1) / target, 6));
    std::vector<int64_t> tiles;
    if (chunk_rooms == 0 && precision == ISM_BF16X3) {
        tiles.resize(n_rooms);
        int64_t total = 0;
        for (int64_t i = 0; i < n_rooms && !tiles.empty(); ++i) {
            const ism_room &R = rooms[i];
            tiles[i] = conv_bf16x3_persistent_tiles(R.n_mics, R.rir_len, src_lens[i] + R.rir_len - 1);
            if (tiles[i] < 0) tiles.clear();
            else total += tiles[i];
        }
        const int64_t sms = device_sm_count();
        if (!tiles.empty() && sms > 0) {
            const double rounds = (double)total / (double)sms;
            const int64_t R = std::min<int64_t>(9, std::max<int64_t>(1, llround(rounds / 4.5)));
            const int64_t Tr = std::max<int64_t>(1, R / 3);
            const int64_t n_main = rounds > (double)R + 1.5 ? (int64_t)((rounds - 1.5) / R) : 0;
            std::vector<int64_t> caps(n_main, R * sms);  // tiles per chunk
            if (rounds - (double)(n_main * R) > (double)(Tr + 1)) caps.push_back(Tr * sms);
            int64_t acc = 0;
            size_t ci = 0;
            for (int64_t r = 0; r < n_rooms; ++r) {
                if (r == 0) {
                    cb.push_back(r);
                } else if (ci < caps.size() && acc + tiles[r] > caps[ci]) {
                    cb.push_back(r);
                    acc = 0;
                    ++ci;
                }
                acc += tiles[r];
            }
        }
    }
    if (!cb.empty()) {
        // cut by tile rounds above
    } else if (chunk_rooms > 0) {
        for (int64_t r = 0; r < n_rooms; r += chunk_rooms) cb.push_back(r);
    } else {
        int64_t r = 0;
        double acc = 0.0;
        for (int64_t c = 0; c < K && r < n_rooms; ++c) {
            cb.push_back(r);
            const double goal = (double)(c + 1) / (double)K * (double)y_total;
            do { acc += (double)ylen[r]; ++r; } while (r < n_rooms && acc < goal);
        }
    }
    cb.push_back(n_rooms);
    const int n_chunks = (int)cb.size() - 1;
    int64_t max_s = 0, max_y = 0, max_h = 0;
    for (int c = 0; c < n_chunks; ++c) {
        int64_t s = 0, y = 0, h = 0;
        for (int64_t i = cb[c]; i < cb[c + 1]; ++i) { s += src_lens[i]; y += ylen[i]; h += hlen[i]; }
        max_s = std::max(max_s, s);
        max_y = std::max(max_y, y);
        max_h = std::max(max_h, h);
    }
    auto al = [](int64_t n) { return (size_t)((n * 4 + 255) & ~(int64_t)255); };
    const size_t set_bytes = al(max_s) + al(max_y) + al(max_h);

    Pipe P;
    cudaError_t e = cudaSuccess;
    if ((e = cudaStreamCreateWithFlags(&P.up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&P.comp[0], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&P.comp[1], cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&P.down, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&P.ev_alloc, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&P.ev_comp1, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "dataset streams");
    for (int s = 0; s < 2; ++s)
        if ((e = cudaEventCreateWithFlags(&P.up_done[s], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&P.comp_done[s], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&P.down_done[s], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "dataset events");
    if (int st = scratch_alloc(&P.buf, 2 * set_bytes, P.comp[0])) return st;
    cudaEventRecord(P.ev_alloc, P.comp[0]);
    cudaStreamWaitEvent(P.up, P.ev_alloc, 0);
    cudaStreamWaitEvent(P.comp[1], P.ev_alloc, 0);
    cudaStreamWaitEvent(P.down, P.ev_alloc, 0);
    auto src_d = [&](int s) { return (float *)((char *)P.buf + s * set_bytes); };
    auto y_d = [&](int s) { return (float *)((char *)P.buf + s * set_bytes + al(max_s)); };
    auto h_d = [&](int s) { return (float *)((char *)P.buf + s * set_bytes + al(max_s) + al(max_y)); };

    // one RIR window for every chunk: the sparse path's fixed-point scale is
    // per window, so the window fixes the last bits of the RIRs
    ism_rir_opts ro;
    memset(&ro, 0, sizeof(ro));
    ro.window = auto_window(rooms, n_rooms);

    int st = ISM_OK;
    std::vector<ism_conv_job> jobs;
    NvtxRange nr("ism.dataset");
    for (int c = 0; c < n_chunks && !st; ++c) {
        NvtxRange cr("ism.dataset.chunk");
        const int s = c & 1;
        const int64_t r0 = cb[c], r1 = cb[c + 1];
        // sources of the chunk, packed in src_d[s]
        if (c >= 2) cudaStreamWaitEvent(P.up, P.comp_done[s], 0);
        {
            int64_t o = 0;
            for (int64_t i = r0; i < r1 && !st; ) {
                // one copy per run of rooms that are contiguous on the host
                int64_t j = i + 1, n = src_lens[i];
                while (j < r1 && so[j] == so[j - 1] + src_lens[j - 1]) n += src_lens[j++];
                st = copy_async(src_d(s) + o, src_host + so[i], (size_t)n * 4,
                                cudaMemcpyHostToDevice, P.up);
                o += n;
                i = j;
            }
        }
        if (st) break;
        cudaEventRecord(P.up_done[s], P.up);
        // kernels of the chunk, on the buffer set's own compute stream
        cudaStream_t cs = P.comp[s];
        cudaStreamWaitEvent(cs, P.up_done[s], 0);
        if (c >= 2) cudaStreamWaitEvent(cs, P.down_done[s], 0);
        st = ism_rir_batch_ex(rooms + r0, r1 - r0, h_d(s), nullptr, &ro, cs);
        if (st) break;
        jobs.assign((size_t)(r1 - r0), ism_conv_job{});
        {
            int64_t hoff = 0, soff = 0, yoff = 0;
            for (int64_t i = r0; i < r1; ++i) {
                ism_conv_job &J = jobs[(size_t)(i - r0)];
                J.n_mics = rooms[i].n_mics;
                J.rir_len = rooms[i].rir_len;
                J.src_len = src_lens[i];
                J.h_offset = hoff;
                J.src_offset = soff;
                J.y_offset = yoff;
                J.snr_db = snr_db ? snr_db[i] : NAN;
                J.noise_id = noise_id_base + (uint64_t)i;
                hoff += hlen[i];
                soff += src_lens[i];
                yoff += ylen[i];
            }
        }
        st = ism_convolve_batch(jobs.data(), r1 - r0, h_d(s), src_d(s), y_d(s), seed, precision,
                                cs);
        if (st) break;
        cudaEventRecord(P.comp_done[s], cs);
        // outputs of the chunk
        cudaStreamWaitEvent(P.down, P.comp_done[s], 0);
        {
            int64_t o = 0;
            for (int64_t i = r0; i < r1 && !st; ) {
                int64_t j = i + 1, n = ylen[i];
                while (j < r1 && yo[j] == yo[j - 1] + ylen[j - 1]) n += ylen[j++];
                st = copy_async(y_host + yo[i], y_d(s) + o, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                P.down);
                o += n;
                i = j;
            }
            o = 0;
            for (int64_t i = r0; h_host && i < r1 && !st; ) {
                int64_t j = i + 1, n = hlen[i];
                while (j < r1 && ho[j] == ho[j - 1] + hlen[j - 1]) n += hlen[j++];
                st = copy_async(h_host + ho[i], h_d(s) + o, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                P.down);
                o += n;
                i = j;
            }
        }
        if (st) break;
        cudaEventRecord(P.down_done[s], P.down);
    }
    // drain every stream (also after an error); the pipe frees the buffer
    const cudaError_t e1 = cudaStreamSynchronize(P.up);
    const cudaError_t e2 = cudaStreamSynchronize(P.down);
    const cudaError_t e3 = cudaStreamSynchronize(P.comp[0]);
    const cudaError_t e4 = cudaStreamSynchronize(P.comp[1]);
    if (!st && e1 != cudaSuccess) st = cuda_fail(e1, "dataset upload");
    if (!st && e2 != cudaSuccess) st = cuda_fail(e2, "dataset download");
    if (!st && e3 != cudaSuccess) st = cuda_fail(e3, "dataset kernels");
    if (!st && e4 != cudaSuccess) st = cuda_fail(e4, "dataset kernels");
    // kernel errors of the chunks' convolutions (the streams are drained)
    for (int s = 0; s < 2; ++s) {
        const int ks = status_collect(P.comp[s], false);
        if (!st) st = ks;
    }
    return st;
}
