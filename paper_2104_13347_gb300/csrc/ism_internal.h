// ism_internal.h -- shared declarations of the CUDA library (not part of
// the public ABI; include/ism.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ism.h"

namespace ism {

// NVTX range on the calling thread for the scope of the object (a profiler
// shows the library's host phases -- plan, K1, K2, noise, serve batches --
// on its timeline; without a profiler attached a range costs a branch).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// One RIR = (room, microphone) as the ISM kernel sees it.  FP64 geometry so
// that the per-axis image offsets round exactly as the definition
// (arXiv 2104.13347, Sec. II.A): offset = ((1-2p) s + (2q) L) - r.
struct alignas(16) RirJob {
    double src[3];
    double mic[3];
    double dims[3];
    double q;           // fs / c, samples per metre (FP64, rounded once)
    float beta[6];      // x0, x1, y0, y1, z0, z1
    int32_t order;      // N
    int32_t n_taps;
    int16_t fd_kind;    // ISM_FD_HANN_SINC / ISM_FD_LAGRANGE
    int16_t n_cheb;     // Chebyshev terms of the filter table (sparse kernel)
    int32_t n_windows;  // ceil(rir_len / W)
    int64_t rir_len;
    int64_t h_offset;   // element offset of h[0] in the output buffer
    int32_t stat_index; // RIR index in the caller's order (statistics slot)
    int32_t tab_offset; // offset of the filter's Chebyshev table (floats; P rows of
                        // round4(n_taps) taps, zero-padded)
};
static_assert(sizeof(RirJob) == 144, "RirJob layout");

// One room of a convolution batch on the device.
struct alignas(16) ConvJob {
    int64_t rir_len;
    int64_t src_len;
    int64_t h_offset;
    int64_t src_offset;
    int64_t y_offset;
    int64_t y_len;       // src_len + rir_len - 1
    uint64_t noise_id;   // identifies the room's noise streams (with the seed)
    int32_t n_mics;
    float snr_db;        // NaN = no noise
    int64_t part_offset; // first noise partial slot of the job
};

// Thread-local error message (ism_last_error_string).
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

// Pinned host staging for descriptor uploads.  Blocks are recycled once the
// copy that read them has completed (an event per block), so uploads never
// wait for earlier work on the stream.
int upload_async(void *dev_dst, const void *host_src, size_t bytes, cudaStream_t stream);

// Stream-ordered device scratch from the library's own memory pool (kept
// cached between calls).
int scratch_alloc(void **p, size_t bytes, cudaStream_t stream);
void scratch_free(void *p, cudaStream_t stream);

int device_sm_count();

// Largest dynamic shared memory a launch of this library asks for: the 227 KB
// a block may opt into, less 1 KB for the kernels' static shared memory (the
// convolution kernels declare 1 KB, their dynamic array's 1024-byte
// alignment; the image-source kernels less than 100 bytes).
constexpr size_t kMaxDynSmem = 227 * 1024 - 1024;

// Lattice order of RIR (room r, mic m): the room's order, or the
// delay-limited order for ISM_ORDER_AUTO (see ism.h).
int room_order(const ism_room &r, int m);

// Checks one room of a batch (index idx for the message); ISM_OK or the
// error status with the last-error string set.
int validate_room(const ism_room &r, int64_t idx);

// The default output window of a K1 call (see ism_api.cu).
int auto_window(const ism_room *rooms, int64_t n_rooms);
// Window autotuner (ism_tune.cu): the tuned window of a call's bucket (0 if
// not tuned yet), and ism_rir_batch_ex with window = ISM_WINDOW_TUNE.
int rir_window_tuned(const ism_room *rooms, int64_t n_rooms, int variant);
int rir_batch_tuned(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                    const int64_t *h_offsets, const ism_rir_opts &opts, cudaStream_t stream);

// K1: image-source taps.  jobs_dev has n_rirs jobs; every job's windows are
// processed; wmax = max n_windows.  counter_dev: one zeroed uint32 work
// counter.  max_order / max_taps size the shared memory and tap rows.
struct RirLaunch {
    const RirJob *jobs_dev;
    int n_rirs;
    int wmax;
    int window;
    int max_order;
    int max_taps;
    int fd_kind;          // all jobs of one launch share the filter kind
    float *h_dev;
    long long *stats_dev; // nullable
    unsigned int *counter_dev;
    int *err_dev;
    int grid;             // 0 = persistent (SMs x blocks/SM)
    const float *tabs_dev;  // sparse kernel: Chebyshev tables [p][n_taps]
    int max_cheb;           // sparse kernel: largest n_cheb of the jobs
    int min_cheb;           // sparse kernel: smallest n_cheb of the jobs
    int min_taps = 0;       // sparse kernel: smallest n_taps of the jobs
    // sparse kernel scratch: per RIR j, offs_dev[2 j] is the offset of its
    // sorted column list in cols_dev (room for TEj^2 entries, TEj = 2 (2 N_j
    // + 1)) and offs_dev[2 j + 1] the offset of its per-window rank ranges
    // in wr_dev (n_windows entries)
    uint32_t *cols_dev = nullptr;
    int2 *wr_dev = nullptr;
    const long long *offs_dev = nullptr;
    // sparse kernel: per-RIR tables (rir_tables_bytes(n_rirs, max_order)
    // bytes), or NULL to have the launch allocate them
    void *tables_dev = nullptr;
};
// Bytes of the sparse kernel's per-RIR tables for n_rirs RIRs of order at
// most max_order (16-byte multiple).
size_t rir_tables_bytes(long long n_rirs, int max_order);
// Entries of a sparse launch's column list for a RIR of order N.
inline long long rir_col_entries(int order) {
    const long long te = 2 * (2 * (long long)order + 1);
    return te * te;
}
// One K1 call prepared on the host, per filter kind: the jobs, the sparse
// path's Chebyshev tables and per-RIR offsets, its launches (chunks of the
// job list), and its device block: [jobs | counter | tables | offsets]
// (blob, uploaded) then [column lists | window ranges | per-RIR tables]
// (filled by the kernels).
struct RirKindPrep {
    int kind = 0;
    bool sparse = false;
    std::vector<RirJob> jobs;
    std::vector<int> caps;  // per job: the lattice order its layout is sized for
    std::vector<float> tabs;
    std::vector<long long> offs;
    std::vector<std::pair<size_t, size_t>> chunks;
    int max_order = 0, max_taps = 1, min_taps = 1 << 30, wmax = 0, max_cheb = 0, min_cheb = 0;
    size_t jb = 0, tb = 0, ob = 0, up_bytes = 0, cb = 0, wb = 0, gb = 0;
    std::vector<unsigned char> blob;
    size_t total() const { return up_bytes + cb + wb + gb; }
};
// Launch groups of a K1 call: 0 the Hann-sinc RIRs, 1 the Lagrange ones,
// 2 the Hann-sinc RIRs that end before their direct arrival (rint of the
// direct delay >= rir_len), which hold nothing but filter tails and take the
// direct per-tap kernel: the sparse path's truncation error is relative to
// the peak tap, so on a RIR made only of far tail taps it could pass the
// 1e-5 bar (on every other RIR the direct path's central taps dominate).
constexpr int kRirGroups = 3;
struct RirPrep {
    int W = 0;
    RirKindPrep k[kRirGroups];
};
// Host preparation of a K1 call at window W (rooms validated by the
// caller).  order_caps (nullable, one per RIR in the caller's order): the
// lattice order each RIR's layout and launch are sized for (a RIR above its
// capacity is an error), so that calls with other rooms of the same shape
// get the same launches; NULL = each RIR's own order.
int rir_prepare(const ism_room *rooms, int64_t n_rooms, const int64_t *h_offsets,
                const ism_rir_opts &o, int W, const int *order_caps, RirPrep *out);
// The launches of one kind, its device block at sp (blob already there).
int rir_enqueue(const RirKindPrep &K, char *sp, int W, float *h_dev, long long *stats,
                int *err_dev, cudaStream_t stream);

// Direct per-tap kernel (bitwise reproducible).
int launch_rir(const RirLaunch &L, cudaStream_t stream);
size_t rir_smem_bytes(int window, int max_order, int max_taps);
// Sparse integer-delay arrays + Chebyshev FIR kernel.
int launch_rir_sparse(const RirLaunch &L, cudaStream_t stream);
size_t rir_sparse_smem_bytes(int window, int max_order, int max_taps, int max_cheb);
constexpr int kMaxCheb = 16;

// Chebyshev table of a fractional-delay filter: coef[p * n_taps + j], tap j
// (first tap = 0) as a function of x in [-1, 1], x = 2f (Hann sinc, f the
// fraction in [-1/2, 1/2]) or x = 2f - 1 (Lagrange, f in [0, 1)).  n_cheb is
// the number of terms kept (<= kMaxCheb), or 0 if the filter needs more.
struct ChebTable {
    int n_cheb;
    std::vector<float> coef;
};
const ChebTable &cheb_table(int fd_kind, int n_taps);

// K2b / K2 / noise.
struct ConvLaunch {
    const ConvJob *jobs_dev;
    const ConvJob *jobs_host;  // same table on the host (for grid sizing)
    int n_jobs;
    const float *h_dev;
    const float *src_dev;
    float *y_dev;
    int precision;
    uint64_t seed;
    int any_noise;
    // sum of y^2 over the tile of mic group g and output block b of job j
    // in slot part_offset(j) + g * ceil(y_len / kConvTT) + b, written by the
    // convolution kernels when non-null (noise requested)
    double *noise_partials_dev;
    // split-BF16 only: the call's status cell (host-mapped; a kernel whose
    // bounded wait runs out sets it), and the test aid of ism_debug_inject
    int *err_dev;
    int inject;
};
// Noise-partial grid: one slot per 8 mics x 2048 outputs (the FP32
// kernel's tile; a tile of the split-BF16 kernel spans two slots).
// Size limits of the entry points: signal lengths (sources, the RIRs a
// convolution is given, a frame's source rows) up to 2^40 samples, and up
// to 65536 mics per room (a room's noise streams are keyed noise_id * 65536
// + mic).  Every size product the host forms then stays below 2^57.
constexpr int64_t kMaxSignal = (int64_t)1 << 40;
constexpr int kMaxMics = 65536;
constexpr int kConvMG = 8;     // mics per tile
constexpr int kConvTT = 2048;  // outputs per slot
__host__ __device__ inline int conv_partials_per_job(int n_mics, int64_t y_len) {
    return (int)((n_mics + kConvMG - 1) / kConvMG * ((y_len + kConvTT - 1) / kConvTT));
}
__host__ __device__ inline int conv_partial_slot(int mic0, int64_t t0, int64_t y_len) {
    return (int)(mic0 / kConvMG * ((y_len + kConvTT - 1) / kConvTT) + t0 / kConvTT);
}
// ism_convolve_batch (also called by the server's worker).
int convolve_batch(const ism_conv_job *jobs, int64_t n_jobs, const float *h_dev,
                   const float *src_dev, float *y_dev, uint64_t seed, int32_t precision,
                   void *stream);
int launch_conv_f32(const ConvLaunch &L, cudaStream_t stream);
int launch_conv_bf16x3(const ConvLaunch &L, cudaStream_t stream);
// One convolution tile: mics [mic0, mic0 + 8) of job `job`, outputs from t0.
struct ConvTile {
    int job;
    int mic0;
    int64_t t0;
};
// The tiles of a convolution call and its launch shapes (host), then its
// launches given the tiles in device memory (launch_conv_* = both, with the
// tiles uploaded through the staging blocks).  Split-BF16: the persistent
// kernel's 8-mic x 4096-output tiles, longest RIR first; FP32: 8-mic x
// 2048-output tiles.
struct ConvPlan {
    int precision = ISM_F32;
    std::vector<ConvTile> tiles;
    int64_t p_max_lh = 0;  // split-BF16: the longest RIR (shared-memory layout)
};
int conv_plan(const ConvLaunch &L, ConvPlan *P);
int conv_f32_plan(const ConvLaunch &L, ConvPlan *P);
int conv_bf16x3_plan(const ConvLaunch &L, ConvPlan *P);
int conv_f32_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                     cudaStream_t stream);
int conv_bf16x3_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                        cudaStream_t stream);
int conv_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                 cudaStream_t stream);
// Tiles the persistent split-BF16 kernel makes of a room (n_mics mics,
// RIRs of rir_len samples, signals of y_len = src_len + rir_len - 1), or -1
// when its RIRs are too long for that kernel.
int64_t conv_bf16x3_persistent_tiles(int n_mics, int64_t rir_len, int64_t y_len);
int launch_noise(const ConvLaunch &L, cudaStream_t stream);

// Bounds-checked build (-DISM_BOUNDS_CHECK, libism_checked.so): the kernels
// test the indices they compute from data -- table entries, sparse-array
// positions, FIR reads, column-list slots, window words, operand extents,
// output samples, noise slots -- and an index out of its range is recorded
// as a bit in the translation unit's device flag word and its access
// skipped (never a trap).  ism_debug_bounds reads and clears the flags.  In
// the normal build ISM_IN_RANGE is the constant true and costs nothing.
enum OobBit : unsigned {
    kOobTableIndex = 1u << 0,     // K1 sparse: z table entry of a candidate
    kOobSparsePos = 1u << 1,      // K1 sparse: sparse-array position
    kOobFirRead = 1u << 2,        // K1 sparse: FIR read of a sparse array
    kOobDeltaRead = 1u << 3,      // K1 sparse: integer-delay array read
    kOobColumnSlot = 1u << 4,     // K1 tables: sorted column-list slot
    kOobColumnEntry = 1u << 5,    // K1 sparse: column-list entry
    kOobDirectRow = 1u << 6,      // K1 direct: window row index
    kOobTcpWindow = 1u << 8,      // K2 persistent: source-window word
    kOobTcpOperand = 1u << 9,     // K2 persistent: B operand extent
    kOobTcpOutput = 1u << 10,     // K2 persistent: output sample
    kOobTcpPartial = 1u << 11,    // K2 persistent: noise-partial slot
    kOobNoise = 1u << 16,         // noise: output sample
    kOobConvF32 = 1u << 17,       // FP32 convolution: output sample or partial
};
// Per translation unit (no relocatable device code): reads and clears its
// flag word; ISM_ERR_INVALID_ARG in the normal build.
int oob_read_rir(unsigned int *flags);
int oob_read_conv(unsigned int *flags);
int oob_read_conv_tc(unsigned int *flags);

#ifdef __CUDACC__
#ifdef ISM_BOUNDS_CHECK
static __device__ unsigned int g_ism_oob;
__device__ __forceinline__ bool ism_oob_record(unsigned int bit) {
    atomicOr(&g_ism_oob, bit);
    return false;
}
#define ISM_IN_RANGE(cond, bit) ((cond) || ::ism::ism_oob_record(bit))
#define ISM_OOB_READER(name)                                                              \
    int oob_read_##name(unsigned int *flags) {                                            \
        unsigned int v = 0u;                                                              \
        cudaError_t e = cudaDeviceSynchronize();                                          \
        if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_ism_oob, sizeof(v));         \
        const unsigned int z = 0u;                                                        \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_ism_oob, &z, sizeof(z));           \
        if (e != cudaSuccess) return cuda_fail(e, "bounds flags");                        \
        *flags |= v;                                                                      \
        return ISM_OK;                                                                    \
    }
#else
#define ISM_IN_RANGE(cond, bit) true
#define ISM_OOB_READER(name)                                                              \
    int oob_read_##name(unsigned int *) {                                                 \
        return fail(ISM_ERR_INVALID_ARG, "not a bounds-checked build");                   \
    }
#endif

// s + e += v^2 in float-float: the square's rounding error from an FMA, the
// sum's from a two-sum (error-free transformations; the pair keeps ~2^-44
// relative accuracy over thousands of terms).
__device__ __forceinline__ void ff_accumulate_sq(float v, float &s, float &e) {
    const float p = __fmul_rn(v, v);
    const float pe = __fmaf_rn(v, v, -p);
    const float t = __fadd_rn(s, p);
    const float bb = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
    e = __fadd_rn(e, __fadd_rn(err, pe));
    s = t;
}

// Sum of x over the 32 lanes of a warp, FP64, fixed shuffle tree; valid in
// lane 0.
__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
#endif

// Kernel status of a call (ism_status.cu).  A call whose kernels contain
// bounded waits takes a status cell -- an int in page-locked, device-mapped
// host memory, zeroed by the host -- and passes its device address to them;
// a wait that runs out sets it.  After enqueueing, the call records an event
// on its stream; once the event has completed, the host reads the cell.
struct StatusTicket {
    int device = -1;
    int cell = -1;
    int *dev = nullptr;
};
int status_begin(StatusTicket *t);
// Records the ticket's completion event on `stream` (or, with ok = false,
// gives the cell back at once: nothing was enqueued).  owned: the cell stays
// with its owner (a plan, whose launches all use it) until status_release.
int status_end(const StatusTicket &t, cudaStream_t stream, bool ok, bool owned = false);
void status_release(const StatusTicket &t);
// ISM_ERR_INTERNAL (with the message set) if a call on `stream` (current
// device) whose kernels have completed reported an internal error since the
// last report; ISM_OK otherwise.  wait: first wait for every call on the
// stream that holds a status cell.
int status_collect(cudaStream_t stream, bool wait);
// Test aid (ism_debug_inject): 1 if injection `what` is pending (and
// clears it), else 0.
int take_injection(int what);

// SplitMix64 (Steele, Lea and Flood 2014): output i of the stream with
// state x is mix(x + (i+1) * gamma).
__host__ __device__ inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
constexpr uint64_t kSm64Gamma = 0x9E3779B97F4A7C15ULL;
__host__ __device__ inline uint64_t sm64_out(uint64_t state, uint64_t i) {
    return sm64_mix(state + (i + 1) * kSm64Gamma);
}

#ifdef __CUDACC__
// Box--Muller pair (Sec. III.A measurement noise) from one SplitMix64 output
// `bits`: u1 = (bits 63..40 + 1/2) 2^-24, u2 = (bits 39..16) 2^-24,
// r = scale sqrt(-2 ln u1), z0 = r cos(2 pi u2), z1 = r sin(2 pi u2).
//  -ln u1 = -ln(1 - t) with t = 1 - u1, exact in FP32 (a 24-bit integer
//   plus 1/2, scaled).  For t < 2^-6 the Taylor series t + t^2/2 + ... +
//   t^5/5 (remainder below 2e-10 relative); above, the hardware base-2
//   logarithm times ln 2, whose small absolute error is then far below
//   -ln u1 >= 0.0157 (r moves by under 1e-6).
//  cos, sin: the octant of the angle comes from the top 3 bits of u2; within
//   it, the distance x in [0, pi/4] to the nearest multiple of pi/2 (the
//   octant offset, reflected in odd octants, exactly, in integers) goes
//   through the Taylor series of sin to x^9 and of cos to x^8 (within 2e-9
//   and 3e-8), which the octant then swaps and negates.
__device__ __forceinline__ void box_muller(uint64_t bits, float scale, float &z0, float &z1) {
    const uint32_t k1 = (uint32_t)(bits >> 40);
    const uint32_t k2 = (uint32_t)(bits >> 16) & 0xFFFFFFu;
    const float u1 = ((float)k1 + 0.5f) * (1.0f / 16777216.0f);
    const float t = ((float)(0xFFFFFFu - k1) + 0.5f) * (1.0f / 16777216.0f);
    const float ser =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 0.2f, 0.25f), 0.33333333f), 0.5f), 1.f);
    const float lg = -__log2f(u1) * 0.69314718f;
    const float r2 = 2.f * (t < 0.015625f ? ser : lg);
    const float r = scale * (r2 * rsqrtf(r2));
    const uint32_t o = k2 >> 21, rem = k2 & 0x1FFFFFu;
    const uint32_t rr = (o & 1u) ? 0x200000u - rem : rem;
    const float x = (float)rr * (0.78539816f / 2097152.0f);
    const float x2 = x * x;
    const float sx = fmaf(x * x2,
                          fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 362880.f, -1.f / 5040.f), 1.f / 120.f),
                               -1.f / 6.f),
                          x);
    const float cx =
        fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 40320.f, -1.f / 720.f), 1.f / 24.f), -0.5f),
             1.f);
    const bool swap = ((o + 1u) >> 1) & 1u;
    const float c = swap ? sx : cx, s = swap ? cx : sx;
    z0 = r * __uint_as_float(__float_as_uint(c) ^ ((((o + 2u) >> 2) & 1u) << 31));
    z1 = r * __uint_as_float(__float_as_uint(s) ^ ((o >> 2) << 31));
}
#endif

}  // namespace ism
