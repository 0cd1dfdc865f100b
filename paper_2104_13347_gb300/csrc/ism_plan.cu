// ism_plan.cu -- plans: the dataset step of a fixed batch shape captured
// once into CUDA graphs and replayed (Sec. II.A: RIRs of a batch of rooms,
// their convolution with the source signals, Sec. III.A noise).
//
// A plan fixes the shape of a batch -- the rooms' microphone counts, RIR
// lengths, filters and source lengths, a lattice-order capacity -- and the
// device buffers (h, sources, y, packed).  At creation it prepares the
// launches the batch entry points would make for that shape, takes one
// device block for every descriptor and scratch array, and captures two
// graphs: each starts with the copies of the per-run descriptors (RIR jobs,
// convolution jobs) from its own page-locked staging buffer, followed by
// the K1 table and sparse kernels, the convolution and the noise kernels.  A
// run writes the new rooms' descriptors into the staging buffer of the
// graph it launches, alternating between the two, so the host prepares run
// k + 1 while run k executes (it waits only for run k - 1 before reusing its
// buffer).  The kernels and their launch shapes are the batch entry points'
// own: a run's outputs are bitwise those of ism_rir_batch_ex (same window)
// and ism_convolve_batch on the same rooms.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "ism_internal.h"

using namespace ism;

struct ism_plan {
    int device = -1;
    ism_plan_config cfg{};
    int64_t n_rooms = 0;
    std::vector<ism_room> shape;  // per room: n_mics, rir_len, n_taps, fd_kind
    std::vector<int64_t> src_lens;
    int W = 0;
    std::vector<int> caps;  // lattice-order capacity per RIR
    bool conv = false;
    float *h_dev = nullptr;
    const float *src_dev = nullptr;
    float *y_dev = nullptr;
    RirPrep prep;
    ConvPlan cplan;
    std::vector<ConvJob> cjobs;
    int64_t n_part = 0;
    char *dblock = nullptr;
    size_t off_rir[kRirGroups] = {}, off_cj = 0, off_tiles = 0, off_part = 0, d_bytes = 0;
    size_t s_rir[kRirGroups] = {}, s_cj = 0, stage_bytes = 0;
    void *pinned[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    bool used[2] = {false, false};
    int next = 0;
    StatusTicket cell;

    ~ism_plan() {
        for (int k = 0; k < 2; ++k)
            if (done[k] && used[k]) cudaEventSynchronize(done[k]);
        status_release(cell);
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (done[k]) cudaEventDestroy(done[k]);
            if (pinned[k]) cudaFreeHost(pinned[k]);
        }
        if (dblock) cudaFree(dblock);
        cudaGetLastError();
    }
};

namespace {

size_t al256(size_t n) { return (n + 255) & ~(size_t)255; }

// The convolution jobs of a run (packed buffers), with its SNRs and noise
// ids; n_part = total noise partial slots.
void make_conv_jobs(const ism_plan &P, const float *snr_db, uint64_t noise_id_base,
                    std::vector<ConvJob> *out, int64_t *n_part) {
    out->assign((size_t)P.n_rooms, ConvJob{});
    int64_t ho = 0, so = 0, yo = 0, np = 0;
    for (int64_t i = 0; i < P.n_rooms; ++i) {
        ConvJob &c = (*out)[(size_t)i];
        const ism_room &R = P.shape[(size_t)i];
        c.rir_len = R.rir_len;
        c.src_len = P.src_lens[(size_t)i];
        c.h_offset = ho;
        c.src_offset = so;
        c.y_offset = yo;
        c.y_len = c.src_len + c.rir_len - 1;
        c.noise_id = noise_id_base + (uint64_t)i;
        c.n_mics = R.n_mics;
        c.snr_db = snr_db ? snr_db[i] : NAN;
        c.part_offset = np;
        np += conv_partials_per_job(R.n_mics, c.y_len);
        ho += (int64_t)R.n_mics * R.rir_len;
        so += c.src_len;
        yo += (int64_t)R.n_mics * c.y_len;
    }
    *n_part = np;
}

ConvLaunch plan_conv_launch(ism_plan &P) {
    ConvLaunch L;
    memset(&L, 0, sizeof(L));
    L.jobs_dev = (const ConvJob *)(P.dblock + P.off_cj);
    L.jobs_host = P.cjobs.data();
    L.n_jobs = (int)P.n_rooms;
    L.h_dev = P.h_dev;
    L.src_dev = P.src_dev;
    L.y_dev = P.y_dev;
    L.precision = P.cfg.precision;
    L.seed = P.cfg.seed;
    L.any_noise = 1;  // jobs without an SNR (NaN) skip the noise kernel's work
    L.noise_partials_dev = (double *)(P.dblock + P.off_part);
    L.err_dev = P.cell.dev;
    L.inject = 0;
    return L;
}

// The same launches as at creation?  (rooms already validated)
int same_launches(const RirPrep &a, const RirPrep &b) {
    for (int k = 0; k < kRirGroups; ++k) {
        const RirKindPrep &x = a.k[k], &y = b.k[k];
        if (x.jobs.size() != y.jobs.size() || x.sparse != y.sparse || x.up_bytes != y.up_bytes ||
            x.total() != y.total() || x.chunks != y.chunks || x.max_order != y.max_order ||
            x.max_taps != y.max_taps || x.wmax != y.wmax || x.max_cheb != y.max_cheb ||
            x.min_cheb != y.min_cheb)
            return fail(ISM_ERR_INVALID_ARG, "the rooms do not fit the plan's launches");
    }
    return ISM_OK;
}

int check_shape(const ism_plan &P, const ism_room *rooms, int64_t n_rooms) {
    if (n_rooms != P.n_rooms) return fail(ISM_ERR_INVALID_ARG, "room count differs from the plan's");
    for (int64_t i = 0; i < n_rooms; ++i) {
        if (int st = validate_room(rooms[i], i)) return st;
        const ism_room &R = rooms[i], &S = P.shape[(size_t)i];
        if (R.n_mics != S.n_mics || R.rir_len != S.rir_len || R.n_taps != S.n_taps ||
            R.fd_kind != S.fd_kind)
            return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(i) +
                                                 ": mics, RIR length or filter differ from the plan's");
    }
    return ISM_OK;
}

// Writes run descriptors into staging buffer k.
void stage(ism_plan &P, int k, const RirPrep &rp, const std::vector<ConvJob> &cj) {
    char *st = (char *)P.pinned[k];
    for (int kind = 0; kind < kRirGroups; ++kind)
        if (!rp.k[kind].jobs.empty())
            memcpy(st + P.s_rir[kind], rp.k[kind].blob.data(), rp.k[kind].up_bytes);
    if (P.conv) memcpy(st + P.s_cj, cj.data(), cj.size() * sizeof(ConvJob));
}

}  // namespace

extern "C" {

int ism_plan_create(const ism_room *rooms, int64_t n_rooms, const int64_t *src_lens,
                    const ism_plan_config *config, float *h_dev, const float *src_dev,
                    float *y_dev, ism_plan **out) {
    set_error("");
    if (!out || !rooms || n_rooms < 1 || !h_dev)
        return fail(ISM_ERR_INVALID_ARG, "NULL rooms, h_dev or out, or no rooms");
    *out = nullptr;
    ism_plan_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    if (config) cfg = *config;
    if (src_lens && (!src_dev || !y_dev))
        return fail(ISM_ERR_INVALID_ARG, "a plan with sources needs src_dev and y_dev");
    if (cfg.precision != ISM_F32 && cfg.precision != ISM_BF16X3)
        return fail(ISM_ERR_INVALID_ARG, "unknown precision");
    if (cfg.variant != ISM_RIR_SPARSE && cfg.variant != ISM_RIR_DIRECT)
        return fail(ISM_ERR_INVALID_ARG, "unknown variant");
    if (cfg.window != 0 && cfg.window != ISM_WINDOW_TUNE &&
        (cfg.window % 32 != 0 || cfg.window < 32 || cfg.window > 8192))
        return fail(ISM_ERR_INVALID_ARG,
                    "window must be a multiple of 32 in [32, 8192], 0 or ISM_WINDOW_TUNE");
    if (cfg.max_order < 0 || cfg.max_order > 200)
        return fail(ISM_ERR_INVALID_ARG, "max_order must lie in [0, 200]");
    for (int64_t i = 0; i < n_rooms; ++i) {
        if (int st = validate_room(rooms[i], i)) return st;
        if (src_lens && (src_lens[i] < 1 || src_lens[i] > kMaxSignal))
            return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(i) + ": src_len must lie in [1, 2^40]");
    }
    std::unique_ptr<ism_plan> P(new ism_plan());
    cudaError_t e = cudaGetDevice(&P->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    P->cfg = cfg;
    P->n_rooms = n_rooms;
    P->h_dev = h_dev;
    P->src_dev = src_dev;
    P->y_dev = y_dev;
    P->conv = src_lens != nullptr;
    for (int64_t i = 0; i < n_rooms; ++i) {
        ism_room S = rooms[i];
        S.mics = nullptr;
        P->shape.push_back(S);
        P->src_lens.push_back(src_lens ? src_lens[i] : 0);
    }
    // window and order capacity
    int W = cfg.window;
    if (W == ISM_WINDOW_TUNE) W = rir_window_tuned(rooms, n_rooms, cfg.variant);
    if (W <= 0) W = auto_window(rooms, n_rooms);
    P->W = W;
    for (int64_t i = 0; i < n_rooms; ++i)
        for (int m = 0; m < rooms[i].n_mics; ++m)
            P->caps.push_back(cfg.max_order > 0 ? std::max(cfg.max_order, room_order(rooms[i], m))
                                                : room_order(rooms[i], m));
    ism_rir_opts o;
    memset(&o, 0, sizeof(o));
    o.window = W;
    o.variant = cfg.variant;
    if (int st = rir_prepare(rooms, n_rooms, nullptr, o, W, P->caps.data(), &P->prep)) return st;
    if (P->conv) {
        make_conv_jobs(*P, nullptr, 0, &P->cjobs, &P->n_part);
        for (auto &c : P->cjobs)
            if ((c.n_mics + (int64_t)kConvMG - 1) / kConvMG * ((c.y_len + kConvTT - 1) / kConvTT) >
                0x3fffffff)
                return fail(ISM_ERR_INVALID_ARG, "too many convolution tiles");
    }
    // device block: [kind 0 | kind 1 | conv jobs | tiles | noise partials]
    size_t o_ = 0;
    for (int kind = 0; kind < kRirGroups; ++kind) {
        P->off_rir[kind] = o_;
        if (!P->prep.k[kind].jobs.empty()) o_ += al256(P->prep.k[kind].total());
    }
    ConvLaunch L;
    if (P->conv) {
        P->off_cj = o_;
        o_ += al256(P->cjobs.size() * sizeof(ConvJob));
        P->dblock = nullptr;
        L = plan_conv_launch(*P);  // jobs_host only, for the tiles
        if (int st = conv_plan(L, &P->cplan)) return st;
        P->off_tiles = o_;
        o_ += al256(P->cplan.tiles.size() * sizeof(ConvTile));
        P->off_part = o_;
        o_ += al256((size_t)P->n_part * sizeof(double));
    }
    P->d_bytes = std::max<size_t>(o_, 256);
    // staging: [kind 0 blob | kind 1 blob | conv jobs]
    size_t s_ = 0;
    for (int kind = 0; kind < kRirGroups; ++kind) {
        P->s_rir[kind] = s_;
        s_ += al256(P->prep.k[kind].up_bytes);
    }
    P->s_cj = s_;
    s_ += P->conv ? al256(P->cjobs.size() * sizeof(ConvJob)) : 0;
    P->stage_bytes = std::max<size_t>(s_, 256);

    e = cudaMalloc((void **)&P->dblock, P->d_bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ISM_ERR_OUT_OF_MEMORY, "plan device block");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(plan)");
    for (int k = 0; k < 2; ++k) {
        if ((e = cudaHostAlloc(&P->pinned[k], P->stage_bytes, cudaHostAllocDefault)) != cudaSuccess)
            return cuda_fail(e, "cudaHostAlloc(plan staging)");
        memset(P->pinned[k], 0, P->stage_bytes);
        if ((e = cudaEventCreateWithFlags(&P->done[k], cudaEventDisableTiming)) != cudaSuccess)
            return cuda_fail(e, "cudaEventCreate(plan)");
    }
    if (P->conv && P->cfg.precision == ISM_BF16X3)
        if (int st = status_begin(&P->cell)) return st;
    if (P->conv) {
        L = plan_conv_launch(*P);
        if (!P->cplan.tiles.empty() &&
            (e = cudaMemcpy(P->dblock + P->off_tiles, P->cplan.tiles.data(),
                            P->cplan.tiles.size() * sizeof(ConvTile), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
            return cuda_fail(e, "cudaMemcpy(plan tiles)");
    }
    // capture: one graph per staging buffer
    cudaStream_t cs = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate(plan)");
    int st = ISM_OK;
    for (int k = 0; k < 2 && !st; ++k) {
        if ((e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
            st = cuda_fail(e, "cudaStreamBeginCapture(plan)");
            break;
        }
        for (int kind = 0; kind < kRirGroups && !st; ++kind) {
            const RirKindPrep &K = P->prep.k[kind];
            if (K.jobs.empty()) continue;
            if ((e = cudaMemcpyAsync(P->dblock + P->off_rir[kind], (char *)P->pinned[k] + P->s_rir[kind],
                                     K.up_bytes, cudaMemcpyHostToDevice, cs)) != cudaSuccess)
                st = cuda_fail(e, "plan descriptor copy");
        }
        if (!st && P->conv &&
            (e = cudaMemcpyAsync(P->dblock + P->off_cj, (char *)P->pinned[k] + P->s_cj,
                                 P->cjobs.size() * sizeof(ConvJob), cudaMemcpyHostToDevice, cs)) !=
                cudaSuccess)
            st = cuda_fail(e, "plan descriptor copy");
        for (int kind = 0; kind < kRirGroups && !st; ++kind) {
            const RirKindPrep &K = P->prep.k[kind];
            if (K.jobs.empty()) continue;
            st = rir_enqueue(K, P->dblock + P->off_rir[kind], W, h_dev, nullptr, nullptr, cs);
        }
        if (!st && P->conv) {
            st = conv_enqueue(L, P->cplan, (const ConvTile *)(P->dblock + P->off_tiles), cs);
            if (!st) st = launch_noise(L, cs);
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cs, &g);
        if (!st && e != cudaSuccess) st = cuda_fail(e, "cudaStreamEndCapture(plan)");
        if (!st && (e = cudaGraphInstantiate(&P->exec[k], g, 0)) != cudaSuccess)
            st = cuda_fail(e, "cudaGraphInstantiate(plan)");
        if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    if (st) return st;
    *out = P.release();
    return ISM_OK;
}

int ism_plan_run(ism_plan *P, const ism_room *rooms, const float *snr_db, uint64_t noise_id_base,
                 void *stream_v) {
    set_error("");
    if (!P || !rooms) return fail(ISM_ERR_INVALID_ARG, "NULL plan or rooms");
    cudaStream_t stream = (cudaStream_t)stream_v;
    NvtxRange nr("ism.plan.run");
    int d = -1;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (d != P->device) return fail(ISM_ERR_INVALID_ARG, "the plan belongs to another device");
    if (int st = check_shape(*P, rooms, P->n_rooms)) return st;
    if (snr_db && P->conv)
        for (int64_t i = 0; i < P->n_rooms; ++i)
            if (!isnan(snr_db[i]) && !isfinite(snr_db[i]))
                return fail(ISM_ERR_INVALID_ARG, "snr must be finite or NaN");
    if (P->conv && P->cfg.precision == ISM_BF16X3)
        if (int st = status_collect(stream, false)) return st;
    ism_rir_opts o;
    memset(&o, 0, sizeof(o));
    o.window = P->W;
    o.variant = P->cfg.variant;
    RirPrep rp;
    if (int st = rir_prepare(rooms, P->n_rooms, nullptr, o, P->W, P->caps.data(), &rp)) return st;
    if (int st = same_launches(P->prep, rp)) return st;
    std::vector<ConvJob> cj;
    int64_t np = 0;
    if (P->conv) make_conv_jobs(*P, snr_db, noise_id_base, &cj, &np);
    const int k = P->next;
    if (P->used[k] && (e = cudaEventSynchronize(P->done[k])) != cudaSuccess)
        return cuda_fail(e, "plan: waiting for the staging buffer");
    stage(*P, k, rp, cj);
    if ((e = cudaGraphLaunch(P->exec[k], stream)) != cudaSuccess)
        return cuda_fail(e, "cudaGraphLaunch(plan)");
    if ((e = cudaEventRecord(P->done[k], stream)) != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord(plan)");
    P->used[k] = true;
    P->next = k ^ 1;
    if (P->cell.cell >= 0) return status_end(P->cell, stream, true, true);
    return ISM_OK;
}

int ism_plan_destroy(ism_plan *P) {
    if (!P) return fail(ISM_ERR_INVALID_ARG, "NULL plan");
    delete P;
    return ISM_OK;
}

}  // extern "C"
