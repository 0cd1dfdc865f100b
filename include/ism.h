/*
 * ism.h -- C ABI of the GB300 image-source RIR and convolution library
 * (libism.so).
 *
 * The library computes, on one GPU, the dataset-generation path of
 * arXiv 2104.13347, Sec. II.A: shoebox room impulse responses from the
 * image-source method with fractional delays, then the batch convolution of
 * source signals with those RIRs into multichannel microphone pressure, with
 * the additive Gaussian noise at a chosen SNR of Sec. III.A.
 *
 * Conventions shared by every entry point:
 *  - Plain C types only.  Pointers named *_dev are CUDA device pointers
 *    (e.g. from a torch tensor); everything else is host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Batch calls only enqueue work: they return once the work is
 *    queued, and outputs are valid after the stream reaches that point.
 *  - The caller owns every buffer it passes.  Host arrays may be freed once
 *    the call returns.  Device outputs must not be read or freed before the
 *    stream has passed the call.
 *  - Every call returns an ism_status.  On error nothing has been launched,
 *    and ism_last_error_string() (thread-local) says why.  No C++ exception
 *    crosses this boundary.
 *  - Lengths and offsets are counted in elements, not bytes.
 */
#ifndef ISM_H
#define ISM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ism_status {
    ISM_OK = 0,
    ISM_PENDING = 1,             /* serve: result not ready yet */
    ISM_ERR_INVALID_ARG = 2,     /* validation failed; nothing launched */
    ISM_ERR_OUT_OF_MEMORY = 3,   /* device scratch or serve pool exhausted */
    ISM_ERR_BUSY = 4,            /* serve: cannot admit the request now */
    ISM_ERR_TIMEOUT = 5,         /* serve: wait deadline passed */
    ISM_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    ISM_ERR_INTERNAL = 7,        /* a kernel reported an internal error */
    ISM_ERR_UNKNOWN_TICKET = 8   /* serve: ticket never issued or released */
} ism_status;

/* Fractional-delay filter.
 *  ISM_FD_HANN_SINC: n_taps = 2H+1 (odd) taps j = -H..H at k0 + j, where
 *    k0 = rint(tau), f = tau - k0, tap = sinc(j - f) * 0.5 (1 + cos(pi (j-f)/(H+1))).
 *  ISM_FD_LAGRANGE: the paper's 7th-order Lagrange filter (Sec. II.A),
 *    n_taps = P+1 (even) taps j = 0..P at floor(tau) - (P-1)/2 + j with
 *    coefficients prod_{i != j} (D - i)/(j - i), D = tau - floor(tau) + (P-1)/2. */
typedef enum ism_fd_kind { ISM_FD_HANN_SINC = 0, ISM_FD_LAGRANGE = 1 } ism_fd_kind;

/* Arithmetic of the convolution.
 *  ISM_F32: FP32 direct convolution on the CUDA cores.
 *  ISM_BF16X3: tensor-core convolution with each operand split into
 *    bf16 hi + lo parts, the cross products accumulated in FP32: hi.hi,
 *    hi.lo and lo.hi in a persistent kernel (one CTA per SM) for every RIR,
 *    batch and served (RIRs beyond 22464 samples in segments of that many
 *    taps, the accumulator carried across them).
 *    Rel-L2 error against FP64 below 1e-5 per (room, mic) on the dataset's
 *    rooms (8192-sample RIRs, 1 s sources at 16 kHz; the bf16 hi + lo split
 *    itself keeps about 16 bits of each operand).  The error grows with the
 *    number of terms of an output (FP32 tensor-core accumulation): about
 *    6e-5 for 48 kHz RIRs of about 1 s against 1 s sources. */
typedef enum ism_precision { ISM_F32 = 0, ISM_BF16X3 = 1 } ism_precision;

/* One shoebox room, following the problem statement of Sec. II.A.
 * dims    room size Lx, Ly, Lz in metres; the room is [0,Lx]x[0,Ly]x[0,Lz].
 * beta    pressure reflection coefficient of each wall, in [0, 1], ordered
 *         x=0, x=Lx, y=0, y=Ly, z=0, z=Lz.  An image reaching the mic after
 *         a reflections on one wall is damped by beta^a (0^0 = 1).
 * src     source position (metres), strictly inside the room.
 * mics    host array of 3*n_mics doubles (x,y,z per mic), strictly inside
 *         the room and not on the source; 1 <= n_mics <= 65536 (a room's
 *         noise streams are keyed noise_id * 65536 + mic).
 * order   lattice order N >= 0: images (u,v,w,l,m,n), u,v,w in {0,1},
 *         l,m,n in [-N, N], 8 (2N+1)^3 in all.  ISM_ORDER_AUTO (any
 *         negative value): per microphone, the smallest N whose lattice
 *         holds every image able to put a tap into [0, rir_len) -- the
 *         delay-limited image set of Sec. II.A (every reflection arriving
 *         within the response).  With d = (rir_len + n_taps) c / fs,
 *         N = max over axes a and parities p of
 *         floor((d + |(1-2p) src_a - mic_a|) / (2 dims_a)).
 * fs, c   sampling rate (Hz) and speed of sound (m/s), both > 0.
 * n_taps  fractional-delay filter length (see ism_fd_kind).
 * rir_len RIR length Lh >= 1 in samples; taps outside [0, Lh) are dropped. */
#define ISM_ORDER_AUTO (-1)

typedef struct ism_room {
    double dims[3];
    double beta[6];
    double src[3];
    const double *mics;
    int32_t n_mics;
    int32_t order;
    double fs;
    double c;
    int32_t n_taps;
    int32_t fd_kind;
    int64_t rir_len;
} ism_room;

/* How the taps are laid down.
 *  ISM_RIR_SPARSE (default): each image adds P Chebyshev coefficients of its
 *    fractional delay to sparse integer-delay arrays, and one FIR per output
 *    window applies the filter (P <= 16 terms; the expansion error is below
 *    1e-6 of the peak tap for the Hann sinc -- 8 terms for 81 taps, about
 *    1.2e-6 rel-L2 on a RIR -- and zero for the 8-tap Lagrange filter).  The sparse arrays are 32-bit fixed point summed
 *    with integer atomics, so the result does not depend on the order of
 *    the adds: repeated runs are bitwise equal.  The fixed-point scale is
 *    set per output window, so a different window may change the last bit.
 *  ISM_RIR_DIRECT: every tap of every image is evaluated from the filter's
 *    formula and accumulated in a fixed order (bitwise reproducible). */
typedef enum ism_rir_variant { ISM_RIR_SPARSE = 0, ISM_RIR_DIRECT = 1 } ism_rir_variant;

/* ism_rir_opts.window = ISM_WINDOW_TUNE: the window the library's autotuner
 * found fastest for the call's bucket -- the filter (kinds and tap counts),
 * the largest lattice order, the sampling rate, the RIR length (power-of-two
 * class), the number of RIRs (power-of-two class) and the variant.  The first
 * call of a bucket tunes it: it runs the call once per candidate window (64
 * to 2048 samples), timing each on `stream` with the host waiting, and
 * finishes with the fastest, whose outputs it leaves; it returns
 * ISM_ERR_INVALID_ARG if the stream is being captured then.  Choices are kept
 * for the process and, if the environment variable ISM_TUNE_CACHE names a
 * file, appended to it and read by later processes, so a tuned bucket keeps
 * its window (and its RIRs stay bitwise reproducible).  Not with per_room. */
#define ISM_WINDOW_TUNE (-1)

/* Options of ism_rir_batch_ex (zero-initialise for defaults). */
typedef struct ism_rir_opts {
    int32_t window;      /* output window per work item, samples (multiple of
                            32 in [32, 8192]); 0 = automatic: 1024, halved
                            down to 64 while the call has fewer than four
                            work items per SM; ISM_WINDOW_TUNE = autotuned
                            (above).  The automatic window depends on the
                            whole call, so pass a fixed window when a RIR
                            must be bitwise equal across calls of different
                            sizes */
    int32_t per_room;    /* 1 = one plain launch per room (the unbatched path) */
    int64_t *stats_dev;  /* optional device int64[2 * n_rirs]: per RIR, the
                            images with a tap in [0, Lh) and the taps that
                            landed in [0, Lh); accumulated (not overwritten),
                            so zero it first */
    int32_t variant;     /* ism_rir_variant */
    int32_t reserved;
} ism_rir_opts;

/* ism_rir_batch -- RIRs of a batch of rooms (Sec. II.A: image sources,
 * per-image delay split, wall dampings over spherical spreading, fractional
 * delay taps accumulated into h).
 *
 * rooms      host array of n_rooms rooms (n_rooms >= 0; 0 is a no-op).
 * h_dev      device float output; RIR j (rooms in order, mics in order
 *            within a room) occupies h_dev[h_offsets[j] .. + rir_len).
 * h_offsets  host int64 array with one offset per RIR, or NULL for the
 *            packed layout (each room's mics back to back, rooms back to
 *            back).  Ranges must not overlap.
 * Every output sample of every RIR is written (zeros where no tap lands).
 * The image delay tau = d fs / c is split with the same FP64 rounding rule
 * as the definition (ties to even), so integer delays and window counts are
 * exact; taps are accumulated in FP32.
 * Errors: ISM_ERR_INVALID_ARG for dims not finite and > 0, a source or mic
 * not strictly inside the room, a mic on the source, beta outside [0,1],
 * fs or c not finite and > 0, rir_len outside [1, 2^30], n_mics < 1, a tap
 * count outside the filter's range (Hann sinc: odd, 1..255; Lagrange: even,
 * 2..32), an unknown fd_kind, a lattice order above 200 (given, or that of
 * the delay-limited set), lattice delays beyond 8e6 samples, or a NULL
 * pointer; ISM_ERR_CUDA if a launch or scratch allocation fails. */
int ism_rir_batch(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                  const int64_t *h_offsets, void *stream);

/* As ism_rir_batch, with options (NULL = defaults). */
int ism_rir_batch_ex(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                     const int64_t *h_offsets, const ism_rir_opts *opts, void *stream);

/* The window ISM_WINDOW_TUNE would use for this call (same rooms and
 * options), or 0 if its bucket is not tuned yet (host only: reads the
 * ISM_TUNE_CACHE file if set, runs nothing).  Errors: ISM_ERR_INVALID_ARG for
 * invalid rooms or a NULL window. */
int ism_rir_tuned_window(const ism_room *rooms, int64_t n_rooms, const ism_rir_opts *opts,
                         int32_t *window);

/* Number of RIRs (sum of n_mics) and packed h length of a batch, for sizing
 * buffers; host only. */
int ism_rir_batch_size(const ism_room *rooms, int64_t n_rooms, int64_t *n_rirs,
                       int64_t *h_len);

/* Number of Chebyshev terms P the sparse path uses for a filter (host only,
 * no device work): *n_terms = P in [1, 16], or 0 when the filter needs more
 * terms and ism_rir_batch takes the direct path for it.  The per-output FIR
 * of the sparse path costs P * n_taps multiply-adds.
 * Errors: ISM_ERR_INVALID_ARG for an unknown filter, a tap count of the
 * wrong parity, or a NULL pointer. */
int ism_rir_filter_terms(int32_t fd_kind, int32_t n_taps, int32_t *n_terms);

/* Largest number of RIRs (sum of n_mics over the rooms) that one
 * ism_rir_batch_noalloc call accepts. */
#define ISM_NOALLOC_MAX_RIRS 14560

/* ism_rir_batch_noalloc -- ism_rir_batch for callers that cannot allocate.
 * The paper has no counterpart: this is a deployment variant of the same
 * image-source kernel.  It is meant for callers that must not allocate
 * device memory while they run -- their device memory is already owned by
 * another allocator (such as a framework's caching allocator that reserved
 * the whole GPU), or they sit in a latency-bound loop where cudaMalloc's
 * implicit synchronisation and unbounded cost are not acceptable.
 * Arguments and output layout are those of ism_rir_batch, and the results
 * agree with it to FP32 rounding: it runs the direct per-tap kernel
 * (ISM_RIR_DIRECT, which needs no per-RIR tables) on the same automatic
 * windows; no statistics.  The call allocates
 * nothing: its scratch is one fixed 2 MiB device array inside the library,
 * which every GPU that loads the library holds until the process exits.
 * Limits and rules:
 *  - at most ISM_NOALLOC_MAX_RIRS RIRs per call; more returns
 *    ISM_ERR_INVALID_ARG before anything is launched;
 *  - the first call on a device looks up the array's device address on that
 *    device (with it current); make that first call before any stream
 *    capture;
 *  - all calls share the array, which keeps the last call's contents; each
 *    call clears what must start at zero, but calls that overlap on the GPU
 *    (on different streams) race on it, so serialise them;
 *  - the job table reaches the device as the arguments of small kernels
 *    enqueued on `stream` (up to 128 RIRs each), so the call never waits for
 *    the stream and reads no host memory after it returns;
 *  - a negative offset in h_offsets returns ISM_ERR_INVALID_ARG before
 *    anything is launched. */
int ism_rir_batch_noalloc(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                          const int64_t *h_offsets, void *stream);

/* One room of a convolution batch (Sec. II.A, "batch convolutions" of the
 * RIRs with the source signals; Sec. III.A noise).
 * n_mics      RIRs of the room, stored back to back in h_dev starting at
 *             h_offset, each rir_len long.
 * src_offset  the room's source signal, src_len samples, in src_dev.
 * y_offset    output start; mic m writes y_dev[y_offset + m*(src_len +
 *             rir_len - 1) ...], the full linear convolution.
 * snr_db      noise level: each mic gets Gaussian noise of variance
 *             mean(y^2 over all of the room's mics and samples) / 10^(snr/10).
 *             NaN = no noise.
 * noise_id    identifies the room's noise streams (with the call's seed):
 *             the same (seed, noise_id) gives the same noise in any batch. */
typedef struct ism_conv_job {
    int32_t n_mics;
    int32_t reserved;
    int64_t rir_len;
    int64_t src_len;
    int64_t h_offset;
    int64_t src_offset;
    int64_t y_offset;
    float snr_db;
    int32_t reserved2;
    uint64_t noise_id;
} ism_conv_job;

/* ism_convolve_batch -- y = s * h for every mic of every job, plus noise.
 * jobs       host array of n_jobs jobs.
 * h_dev      device float RIRs; src_dev device float sources; y_dev device
 *            float outputs (must not overlap the inputs).
 * seed       noise seed: stream (noise_id, mic) has key
 *            out(seed, noise_id * 65536 + mic); samples 2k, 2k + 1 share
 *            SplitMix64 output k of that stream (u1 from bits 63..40, u2 from
 *            bits 39..16) and take the two Box--Muller branches.
 * precision  ISM_F32 or ISM_BF16X3.
 * Errors: ISM_ERR_INVALID_ARG (n_mics outside [1, 65536], rir_len or
 * src_len outside [1, 2^40], a negative offset, an SNR of +-inf, more than
 * 2^30 - 1 tiles of 8 mics x 2048 outputs in a job, NULL pointers, an unknown
 * precision), ISM_ERR_CUDA, ISM_ERR_OUT_OF_MEMORY (scratch). */
int ism_convolve_batch(const ism_conv_job *jobs, int64_t n_jobs, const float *h_dev,
                       const float *src_dev, float *y_dev, uint64_t seed,
                       int32_t precision, void *stream);

/* ism_dataset_batch -- the whole dataset step of Sec. II.A with host
 * buffers: the RIRs of every (room, mic), the convolution of each room's
 * source with its RIRs and the room's noise, from sources in host memory to
 * microphone signals in host memory.  The rooms run in chunks on the
 * library's own streams: while one chunk's kernels run, the next chunk's
 * sources are uploaded and the previous chunk's signals downloaded (the
 * host buffers must be page-locked for the copies to overlap; pageable
 * memory works but serializes).  Results do not depend on the chunking.
 * rooms, n_rooms  as ism_rir_batch (ISM_ORDER_AUTO included).
 * src_host        room i's source: src_lens[i] floats at
 *                 src_host + src_offsets[i] (src_offsets NULL: packed in
 *                 room order).
 * snr_db          host, one SNR per room (NaN: no noise), or NULL (no noise).
 * seed            noise seed; room i's noise id is noise_id_base + i.
 * precision       ISM_F32 or ISM_BF16X3.
 * y_host          room i's n_mics x (src_lens[i] + rir_len - 1) floats,
 *                 mic-major, at y_host + y_offsets[i] (NULL: packed).
 * h_host          nullable: the RIRs too, room i's n_mics x rir_len floats
 *                 at h_host + h_offsets[i] (NULL offsets: packed).
 * chunk_rooms     rooms per chunk, or 0: with ISM_BF16X3, chunks of
 *                 consecutive rooms whose convolution tiles fill whole
 *                 rounds over the SMs -- main chunks of R rounds (R = the
 *                 batch's rounds / 4.5, at most 9), then one of R / 3
 *                 rounds and the rest, so that the last chunk's download is
 *                 short; with ISM_F32, six or more chunks of about 128 MiB
 *                 of signals each, balanced by signal length.  Consecutive
 *                 chunks compute on two streams, so one chunk's RIR kernel
 *                 overlaps the previous chunk's convolution.  The outputs
 *                 do not depend on the chunking.
 * Returns when every output is in host memory.  Errors: those of
 * ism_rir_batch and ism_convolve_batch, ISM_ERR_INVALID_ARG for NULL
 * buffers or src_lens outside [1, 2^40], ISM_ERR_CUDA, ISM_ERR_OUT_OF_MEMORY. */
int ism_dataset_batch(const ism_room *rooms, int64_t n_rooms, const float *src_host,
                      const int64_t *src_lens, const int64_t *src_offsets,
                      const float *snr_db, uint64_t seed, uint64_t noise_id_base,
                      int32_t precision, float *y_host, const int64_t *y_offsets,
                      float *h_host, const int64_t *h_offsets, int64_t chunk_rooms);

/* ------------------------------------------------------------------------
 * Plans: the dataset step of Sec. II.A (RIRs, convolution) with the noise of
 * Sec. III.A, for a batch of fixed shape, captured once into CUDA graphs and
 * replayed.  A run costs the host one descriptor build and one graph launch
 * instead of the batch entry points' validation, staging and launches, and
 * its outputs are bitwise those of ism_rir_batch_ex (with the plan's window)
 * followed by ism_convolve_batch on the same rooms.
 * ------------------------------------------------------------------------ */
typedef struct ism_plan ism_plan;

typedef struct ism_plan_config {
    int32_t precision;   /* ISM_F32 or ISM_BF16X3 (convolution) */
    int32_t window;      /* K1 window: 0 = automatic for the creation rooms, a
                            multiple of 32 in [32, 8192], or ISM_WINDOW_TUNE
                            (the bucket's tuned window if it is tuned,
                            automatic otherwise; plans never tune) */
    int32_t max_order;   /* lattice-order capacity of every RIR, in
                            [0, 200]: 0 = each RIR's order at creation
                            (ISM_ORDER_AUTO rooms of later runs may need
                            more: give it here); never below a RIR's order
                            at creation */
    int32_t variant;     /* ism_rir_variant */
    uint64_t seed;       /* noise seed (see ism_convolve_batch) */
} ism_plan_config;

/* Creates a plan for batches shaped like `rooms`: the same number of rooms,
 * and per room the same n_mics, rir_len, n_taps and fd_kind (geometry,
 * walls, fs, c and order -- up to the capacity -- may change per run).
 * h_dev: device output, packed RIRs (as ism_rir_batch with NULL offsets).
 * src_lens: host, source length per room, or NULL for a plan of RIRs only;
 * src_dev: device sources packed in room order; y_dev: device output, room
 * i's n_mics x (src_lens[i] + rir_len - 1) samples, packed.  The buffers are
 * the caller's and must outlive the plan; the plan keeps its own device
 * block (descriptors and scratch) and two page-locked staging buffers, and
 * captures its graphs on a private stream (call it before capturing any
 * stream of your own).  Errors: ISM_ERR_INVALID_ARG (rooms, config,
 * src_lens outside [1, 2^40]),
 * ISM_ERR_OUT_OF_MEMORY, ISM_ERR_CUDA. */
int ism_plan_create(const ism_room *rooms, int64_t n_rooms, const int64_t *src_lens,
                    const ism_plan_config *config, float *h_dev, const float *src_dev,
                    float *y_dev, ism_plan **out);

/* Runs the plan on `stream` for `rooms` (same shape as at creation; the
 * current device must be the plan's): RIRs into h_dev and, for a plan with
 * sources, the signals into y_dev with room i's noise at snr_db[i] (host
 * array, NaN = none, or NULL = no noise) and noise id noise_id_base + i.
 * Enqueues and returns; the two staging buffers alternate, so a run waits
 * for the run before the previous one to finish before it overwrites its
 * staging buffer.  Errors: ISM_ERR_INVALID_ARG (a room of another shape, an
 * order above the capacity), ISM_ERR_INTERNAL (an earlier call on the stream
 * reported a kernel error, see ism_stream_status), ISM_ERR_CUDA. */
int ism_plan_run(ism_plan *plan, const ism_room *rooms, const float *snr_db,
                 uint64_t noise_id_base, void *stream);

/* A plan is not thread-safe: run it from one thread at a time. */

/* Waits for the plan's runs, then frees it. */
int ism_plan_destroy(ism_plan *plan);

/* ------------------------------------------------------------------------
 * Training frames: the network of the paper reads multichannel windows of
 * 1024 samples (23.2 ms at 44.1 kHz) of the convolved signals, with
 * measurement noise added at a chosen SNR as data augmentation
 * (Sec. II.B and III.A).  (The paper draws these windows inside its
 * training pipeline; this call is the batched GPU form of that step.)
 * ------------------------------------------------------------------------ */

/* One frame.
 * y_offset    element offset of the room's signals in y_dev: n_mics rows of
 *             y_len samples, mic-major, as ism_convolve_batch writes them.
 * y_len       samples per mic of the room's signals (>= 1).
 * t0          first sample of the frame; samples outside [0, y_len) read as
 *             0 (t0 may be negative or run past the end).
 * out_offset  element offset of the frame in frames_dev: n_mics rows of
 *             frame_len samples, mic-major.
 * noise_id    identifies the frame's noise streams (with the call's seed).
 * n_mics      microphones (rows) of the frame, >= 1.
 * snr_db      SNR of the added noise, relative to the frame's own mean
 *             power over its mics and samples: sigma^2 = P / 10^(snr/10),
 *             noise sigma z, z standard normal from SplitMix64 counters
 *             (stream key out(seed, noise_id * 65536 + mic); samples 2k and
 *             2k + 1 of the frame share output k: u1 from bits 63..40,
 *             u2 from bits 39..16, and take the two Box--Muller branches
 *             r cos(2 pi u2), r sin(2 pi u2)).  NaN or +inf: a clean copy. */
typedef struct ism_frame_job {
    int64_t y_offset;
    int64_t y_len;
    int64_t t0;
    int64_t out_offset;
    uint64_t noise_id;
    int32_t n_mics;
    float snr_db;
} ism_frame_job;

/* ism_frames_batch -- cut n_frames frames of frame_len samples and add their
 * noise.  jobs: host array; y_dev, frames_dev: device floats (must not
 * overlap).  Errors: ISM_ERR_INVALID_ARG (NULL pointers, frame_len < 1,
 * n_mics outside [1, 65536], y_len outside [1, 2^40], negative offsets,
 * SNR = -inf), ISM_ERR_CUDA,
 * ISM_ERR_OUT_OF_MEMORY (scratch). */
int ism_frames_batch(const ism_frame_job *jobs, int64_t n_frames, int32_t frame_len,
                     const float *y_dev, float *frames_dev, uint64_t seed, void *stream);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of RIR + convolution requests.
 * Requests of uneven sizes arrive at any time; a background thread admits
 * them while device memory (max_hbm_bytes) and slots allow, packs the
 * admitted ones into ragged batches, and runs them on its streams so that
 * batches overlap on the GPU.  Results stay on the device until released.
 * Each request's work items (RIR windows, convolution tiles, noise streams
 * keyed by its noise_id) are the same alone or mixed with others, bit for
 * bit (the sparse RIR path sums in fixed point, and the server always uses
 * 1024-sample RIR windows).  The server convolves with the kernels of
 * ism_convolve_batch, whose work for a job does not depend on the rest of
 * the batch: given the same RIRs, seed and noise ids its signals equal the
 * batch call's bit for bit.
 * ------------------------------------------------------------------------ */
typedef struct ism_server ism_server;

typedef struct ism_serve_config {
    int64_t max_hbm_bytes;   /* device bytes the server may hold (0 = 8 GiB) */
    int32_t max_batch;       /* requests per launch batch (0 = 64) */
    int32_t n_streams;       /* concurrent batches in flight (0 = 2) */
    int32_t precision;       /* ISM_F32 or ISM_BF16X3 */
    int32_t max_queue;       /* waiting requests before submit says BUSY (0 = 4096) */
    uint64_t seed;           /* noise seed */
    int32_t device;          /* CUDA device ordinal */
    int32_t reserved;
} ism_serve_config;

typedef struct ism_request {
    ism_room room;
    const float *src_host;   /* source signal, src_len floats; copied at submit */
    int64_t src_len;
    float snr_db;            /* NaN = no noise */
    int32_t reserved;
    uint64_t noise_id;       /* noise streams of the request (with the server
                                seed); 0 = use the ticket */
} ism_request;

typedef struct ism_result {
    const float *h_dev;      /* n_mics x rir_len, library-owned until release */
    const float *y_dev;      /* n_mics x y_len, library-owned until release */
    int32_t n_mics;
    int32_t reserved;
    int64_t rir_len;
    int64_t y_len;
    double queue_s;          /* submit -> launch */
    double latency_s;        /* submit -> result ready on the device */
} ism_result;

typedef struct ism_serve_stats {
    int64_t submitted, completed, rejected_busy, batches;
    int64_t queued, in_flight;
    int64_t bytes_in_use, bytes_peak;
    int64_t taps;            /* image-source taps that landed in the RIRs */
    int64_t mic_samples;     /* convolution outputs written */
    int64_t launch_host_ns;  /* host time the server thread spent launching
                                batches (allocation, uploads, launches) */
    int64_t batch_device_ns; /* device time of the finished batches, first
                                kernel to completion (CUDA events) */
} ism_serve_stats;

/* Creates a server on config->device.  Besides at most max_hbm_bytes of
 * device memory, the server keeps page-locked host blocks (request source
 * copies, statistics readbacks) in a cache for reuse, at most 1 GiB of
 * them, returned at ism_serve_destroy.  Errors: INVALID_ARG, CUDA. */
int ism_serve_create(const ism_serve_config *config, ism_server **out);

/* Validates and enqueues a request; returns its ticket.  The source is
 * copied into a page-locked host block before the call returns, so the
 * caller's buffer may be reused at once.  ISM_ERR_BUSY if the queue is full
 * or the request alone needs more than max_hbm_bytes; ISM_ERR_INVALID_ARG
 * for an invalid room or source (src_len outside [1, 2^40]);
 * ISM_ERR_OUT_OF_MEMORY if no host block
 * can be had. */
int ism_serve_submit(ism_server *server, const ism_request *request, uint64_t *ticket);

/* ISM_OK and the result if ready, ISM_PENDING if not yet,
 * ISM_ERR_UNKNOWN_TICKET if the ticket was never issued or is released,
 * ISM_ERR_CUDA / ISM_ERR_INTERNAL if the request's batch failed. */
int ism_serve_poll(ism_server *server, uint64_t ticket, ism_result *out);

/* As poll, blocking up to timeout_s seconds (ISM_ERR_TIMEOUT after). */
int ism_serve_wait(ism_server *server, uint64_t ticket, double timeout_s, ism_result *out);

/* Copies a finished request's RIRs (n_mics x rir_len) and microphone
 * signals (n_mics x y_len), mic-major, into caller buffers h_out / y_out
 * (device or host memory; either may be NULL), enqueued on `stream`; read
 * them once the stream has passed the copy.  Same status codes as poll
 * (ISM_PENDING if not finished yet). */
int ism_serve_copy(ism_server *server, uint64_t ticket, float *h_out, float *y_out,
                   void *stream);

/* Frees a finished request's device memory.  ISM_ERR_UNKNOWN_TICKET for an
 * unknown ticket, ISM_PENDING if it is still running (not released). */
int ism_serve_release(ism_server *server, uint64_t ticket);

int ism_serve_stats_get(ism_server *server, ism_serve_stats *out);

/* Stops the serving thread after in-flight batches finish and frees all
 * server memory; outstanding results become invalid. */
int ism_serve_destroy(ism_server *server);

/* ------------------------------------------------------------------------
 * Kernel-reported errors.  The split-BF16 tensor-core convolution kernels
 * bound every wait inside them (2 s): if one runs out, the kernel stops,
 * writes zeros for the outputs it did not finish and records the failure in
 * the call's status cell.  Batch calls return before their kernels run, so
 * the failure is reported once the call's work has completed, as
 * ISM_ERR_INTERNAL: by ism_stream_status on the call's stream, by the next
 * ism_convolve_batch on that stream (which then launches nothing), by
 * ism_dataset_batch (which waits for its work), and by ism_serve_poll /
 * ism_serve_wait for the requests of a served batch.
 * ------------------------------------------------------------------------ */

/* Waits for every earlier call on `stream` (current device) that holds a
 * status cell, then returns ISM_ERR_INTERNAL if any call on the stream
 * reported a kernel error since the last report (the report clears it),
 * ISM_OK otherwise. */
int ism_stream_status(void *stream);

/* Fault injection for tests of the error path (no counterpart in the paper).
 * ISM_INJECT_CONV_WAIT: the next split-BF16 convolution launch (any thread)
 * makes each of its CTAs' MMA issuer wait, before issuing anything, on a
 * barrier that nothing arrives at, with every wait of that launch limited to
 * 20 ms; the launch then stops as after a real timeout and its call reports
 * ISM_ERR_INTERNAL.  0 cancels a pending injection.  Nothing faults or hangs:
 * the waits are bounded and the kernels return. */
#define ISM_INJECT_CONV_WAIT 1
/* ISM_INJECT_SERVE_ALLOC: the next batch a server launches finds its device
 * allocation failing (the allocator is not called): the batch's requests
 * fail with ISM_ERR_OUT_OF_MEMORY, their memory budget is returned when they
 * are released, and later batches run normally.  Injections of different
 * kinds may be pending together. */
#define ISM_INJECT_SERVE_ALLOC 2
int ism_debug_inject(int32_t what);

/* Bounds-checked build (libism_checked.so, compiled with ISM_BOUNDS_CHECK):
 * the kernels test every index they compute from data (table entries,
 * sparse-array positions, FIR reads, column-list slots, window words,
 * operand extents, noise-partial slots); an index out of range sets a flag
 * bit and its access is skipped, never trapped.  ism_debug_bounds waits for
 * the device, returns the bits set since the last call in *flags and clears
 * them (no counterpart in the paper; a debugging aid).  In the normal build
 * it returns ISM_ERR_INVALID_ARG. */
int ism_debug_bounds(uint32_t *flags);

/* Message of the last error on the calling thread ("" if none). */
const char *ism_last_error_string(void);

/* Library version string. */
const char *ism_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ISM_H */
