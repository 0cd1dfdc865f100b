// ism_conv_tc.cu -- K2: the convolution y_m = s * h_m on the tcgen05 tensor
// cores, in split BF16 (each FP32 operand as bf16 hi + lo, FP32 accumulate).
//
// Convolution (arXiv 2104.13347, Sec. II.A: the dataset is built by batch
// convolution of the RIRs with source signals), for every mic m of a room:
//   y_m[t] = sum_k h_m[k] s[t - k],  t in [0, Ts + Lh - 1).
//
// Block-Toeplitz formulation: outputs of a tile are split into phases so
// that the source operand B is a Toeplitz matrix whose rows shift by 8
// elements = 16 bytes, read straight from a linear copy of the source in
// shared memory through a no-swizzle K-major descriptor with
// leading-dimension offset 16 B and stride offset 128 B (core matrices
// overlap), and the RIR operand A is materialised per chunk of taps in TMEM.
//
// k_conv_tcp (every split-BF16 call, batch and served): a persistent kernel,
// one CTA per SM.  A tile is 8 mics x 4096 outputs, 16 phases; the taps are
// split by parity so that both parity windows of the source are again
// 16-byte-shifted Toeplitz matrices.  Its 128 GEMM rows are (mic, phase) of
// one part, and the MMAs hi.hi, lo.hi and hi.lo accumulate into one FP32
// accumulator: the split-BF16 product without its lo.lo term (each lo part
// is within 2^-8 of its value, so lo.lo is within 2^-16 of the product: the
// order of the split's own representation error, and adding it back does
// not lower the largest rel-L2 error over the dataset's RIRs).  The A
// operands go straight from the producers' registers into TMEM
// (tcgen05.st), so shared memory carries only the source windows the MMAs
// read as B: one window per segment of up to P_SEG chunks of taps (one
// segment for RIRs up to 22464 samples, several for longer ones, the
// accumulator carried across them); two window buffers let the next
// segment's window conversion run under the current segment's MMAs.
//
// The raw RIR values of each chunk are staged with cp.async (zero-filled
// outside the RIR), converted once per value into bf16 hi / lo pairs, and
// each producer thread builds 16-byte rows of A with byte permutes.  Chunks
// whose source window is all zero padding are skipped.  Stages hand over
// through mbarriers (full: producer arrivals; empty: tcgen05.commit).  Every
// wait is bounded: on timeout the kernel records an error in the call's
// status cell (host-mapped memory the host reads once the call has
// completed), stops issuing, writes zeros for the outputs it did not finish,
// waits (bounded) for its own MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ism_internal.h"

namespace ism {

namespace {

constexpr int NN = 256;                // GEMM N: time groups of 16 outputs
constexpr int MG = 8;                  // mics per tile
static_assert(MG == kConvMG, "tile shape of the noise partials");
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any mbarrier wait

using Tile = ConvTile;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor: start address, leading and
// stride byte offsets (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;
    return d;
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) |
                            ((128u >> 4) << 24);

// Bounded waits of one launch: the call's status cell (host-mapped int,
// set to 1 when a wait runs out; may be null), the limit of every wait, and
// the test aid that makes the MMA issuer wait once on a barrier nothing
// arrives at (ism_debug_inject).
struct WaitCtl {
    int *err;
    unsigned long long limit_ns;
    int inject;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the given phase parity of an mbarrier, at most w.limit_ns; on
// timeout sets the call's status cell (host-mapped) and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const WaitCtl &w) {
    const unsigned long long t0 = global_ns();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > w.limit_ns) break;
    }
    if (w.err) {
        *reinterpret_cast<volatile int *>(w.err) = 1;
        __threadfence_system();
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
    // element with the lower k at the lower address (low half)
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float bf16_round(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const float *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}

// ===========================================================================
// k_conv_tcp: persistent convolution with three products, A in TMEM
// ===========================================================================
// A tile is 8 mics x 4096 outputs t = T0 + 16 n + p (n < 256, p < 16).
// With k = 2 kappa + b split by parity b, B_b[kappa][n] = s[c0 + b + 2 kappa
// + 16 n] is the Toeplitz matrix of the source's parity-b samples, whose
// rows again shift by 8 elements (16 bytes), and A_b[(m, p)][kappa] =
// h_m[Lh - 1 + p - b - 2 kappa].  GEMM row (TMEM lane) R = 64 (p % 2) +
// 8 m + p / 2 holds (mic m, phase p), so that each producer warp writes the
// 32 lanes of its own TMEM lane quadrant.  Per parity the MMAs hi.hi, lo.hi
// and hi.lo (A from TMEM, B from shared memory) accumulate into one
// 128 x 256 FP32 accumulator, so no hi / lo rows are merged in the epilogue.
//
// One CTA per SM walks its tiles (blockIdx.x, + gridDim.x, ...).  A tile's
// live chunks are cut into segments of P_SEG chunks ("units"), each with its
// own source window (word e of segment u starts at source sample c0 + 64 u_lo
// + 4 e, u_lo its first chunk); a tile without live chunks is one empty
// unit.  Warps 0-7 build the A operands of 64-tap chunks into four TMEM
// stages of 64 columns (warps 0-3 the hi parts, 4-7 the lo parts) and, a
// slice per chunk, convert the next unit's source window into the other of
// two window buffers (the slice's source values are loaded one chunk before
// they are stored); warp 8 allocates 512 TMEM columns (the accumulator in
// 0-255, the stages from 256) and one lane issues the MMAs; warps 9-12 drain
// the accumulator (write y, sum y^2), which the next tile's first MMA waits
// for.  Barriers: full / empty per stage; win[b] (the window buffer's unit
// has had its last MMA); accf (a tile's MMAs are done); acce (the
// accumulator is drained).  Every wait is bounded.
constexpr int P_PH = 16;                 // output phases per row set
constexpr int P_TT = P_PH * NN;          // outputs per tile (4096)
static_assert(P_TT == 2 * kConvTT, "a tile covers two noise-partial slots");
constexpr int P_KC = 64;                 // k values per chunk: 32 per parity
constexpr int P_NS = 4;                  // operand stages (in TMEM)
constexpr int P_ACOL = 256;              // TMEM column of stage 0 (after the accumulator)
constexpr int P_SCOL = 64;               // TMEM columns per stage: [parity][hi / lo][32 kappa / 2]
constexpr int P_STG = 8 * 80;            // raw RIR per chunk: 8 mics x 80 values
constexpr int P_PB = 4;                  // raw RIR staging buffers (ring)
constexpr int P_PD = 3;                  // chunks staged ahead
constexpr int P_CVW = 2 * 8 * 40;        // the chunk as bf16 pairs: [hi/lo][mic][40 words]
constexpr int P_NPROD = 256;             // producer threads (warps 0-7)
constexpr int P_NT = 416;                // 13 warps: producers, MMA (warp 8), epilogue (9-12)
constexpr int P_SEG = 352;               // chunks per segment window (22464 taps)

// OR of pred over the P_NPROD producer threads (named barrier 1); also a barrier.
__device__ __forceinline__ bool p_producers_any(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, 256, p;\n"
        "selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

struct PLayout {
    size_t stg, cv, win, win_bytes, total;
    int bl;
};

// Elements per [parity][hi / lo] array of the source window of n_ch chunks:
// chunk c of the window reads elements 32 c + [0, 32 + 8 (NN - 1)).
__host__ __device__ inline int p_window_len(int n_ch) {
    return (n_ch * 32 + 8 * (NN - 1) + 8 + 7) & ~7;
}

// Shared-memory layout for RIRs of at most max_lh samples: raw staging (P_PB
// chunks), two converted chunks, two segment windows of four [parity][hi /
// lo] arrays of bl elements (the A operands live in TMEM).
__host__ __device__ inline PLayout p_layout(int64_t max_lh) {
    PLayout L;
    const int64_t n_ch = (max_lh + 15 + P_KC - 1) / P_KC;
    L.bl = p_window_len(n_ch < P_SEG ? (int)n_ch : P_SEG);
    L.stg = 0;
    L.cv = L.stg + (size_t)P_STG * P_PB * 4;
    L.win = L.cv + (size_t)2 * P_CVW * 4;
    L.win_bytes = (size_t)4 * L.bl * 2;
    L.total = L.win + 2 * L.win_bytes;
    return L;
}

// Source samples s[i0 .. i0 + 3], zero outside [0, Ts).
__device__ __forceinline__ void load_source4(float (&x)[4], const float *sb, int64_t i0,
                                             int64_t Ts) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t idx = i0 + k;
        x[k] = (idx >= 0 && idx < Ts) ? __ldg(sb + idx) : 0.f;
    }
}

// Four source samples x = s[i0 .. i0 + 3] as the words of the two parity
// windows at one word position: w[(2 b + q) * stride] = (part_q(x[b]),
// part_q(x[b + 2])).
__device__ __forceinline__ void store_split4(uint32_t *w, int stride, const float (&x)[4]) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        const float h0 = bf16_round(x[b]), h1 = bf16_round(x[b + 2]);
        w[(2 * b) * stride] = pack_bf16(h0, h1);
        w[(2 * b + 1) * stride] = pack_bf16(x[b] - h0, x[b + 2] - h1);
    }
}

__device__ __forceinline__ void store_decimated(uint32_t *w, int stride, const float *sb,
                                                int64_t i0, int64_t Ts) {
    float x[4];
    load_source4(x, sb, i0, Ts);
    store_split4(w, stride, x);
}

// Per-tile constants shared by the three roles.
struct PTile {
    Tile tl;
    int64_t Lh, Ts, T0, c0;
    int ch_lo, n_live, nm;
};

__device__ __forceinline__ PTile p_tile(const ConvJob *jobs, const Tile *tiles, int idx) {
    PTile t;
    t.tl = tiles[idx];
    const ConvJob &J = jobs[t.tl.job];
    t.Lh = J.rir_len;
    t.Ts = J.src_len;
    t.T0 = t.tl.t0;
    t.c0 = t.T0 - t.Lh + 1;
    t.nm = min(MG, J.n_mics - t.tl.mic0);
    const int n_chunks = (int)((t.Lh + 15 + P_KC - 1) / P_KC);
    // chunk ch reads s[c0 + 64 ch .. c0 + 64 ch + 63 + 16 (NN - 1)]
    int64_t lo_c = -t.c0 - (P_KC - 1 + P_PH * (NN - 1));
    lo_c = lo_c <= 0 ? 0 : (lo_c + P_KC - 1) / P_KC;
    int64_t hi_c = t.Ts - 1 - t.c0;
    hi_c = hi_c < 0 ? -1 : hi_c / P_KC;
    t.ch_lo = (int)lo_c;
    const int ch_hi = (int)min(hi_c, (int64_t)n_chunks - 1);
    t.n_live = ch_hi >= t.ch_lo ? ch_hi - t.ch_lo + 1 : 0;
    return t;
}

// Units (segment windows) of a tile: its live chunks in segments of P_SEG,
// one empty unit if it has none.
__device__ __forceinline__ int p_units(const PTile &t) {
    return t.n_live > 0 ? (t.n_live + P_SEG - 1) / P_SEG : 1;
}
// Words per array of segment sg's window (0 for a tile without live chunks).
__device__ __forceinline__ int p_seg_words(const PTile &t, int sg) {
    if (t.n_live == 0) return 0;
    return p_window_len(min(P_SEG, t.n_live - sg * P_SEG)) / 2;
}
// First source sample of segment sg's window.
__device__ __forceinline__ int64_t p_seg_base(const PTile &t, int sg) {
    return t.c0 + (int64_t)P_KC * (t.ch_lo + sg * P_SEG);
}

// Operand rows of thread (m, p) for one chunk, p of parity PAR, written
// into the thread's TMEM lane.  Element kl (kappa = 32 ch + kl) of operand
// (b, q) is part_q(stg[m][e_b - 2 kl]), e_b = 63 + p - b; word w of k-group
// kg takes kl = 8 kg + 2w, 8 kg + 2w + 1, the same half (high if e_b is odd)
// of cv words I_b - kl and I_b - kl - 1, I_b = e_b >> 1.  For even p, I_0 =
// I_1; for odd p, I_0 = I_1 + 1.  Operand (b, q) takes the 16 columns
// taddr + (2 b + q) 16 + [0, 16): column c holds kl = 2c (low half) and
// 2c + 1, the packing of a K-major A operand in TMEM.
template <int PAR>
__device__ __forceinline__ void p_rows(const uint32_t *cvb, uint32_t taddr, int m, int p, int q) {
    const int I1 = (62 + p) >> 1;  // I_1 (odd p: (61 + p) / 2 = (62 + p) >> 1 too)
    const uint32_t *cv = cvb + q * (P_CVW / 2) + m * 40 + (I1 - 31);
    uint32_t W[33];
#pragma unroll
    for (int k = 0; k < 33; ++k) W[k] = (PAR == 1 || k < 32) ? cv[k] : 0u;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        // window offset of operand b in W, and its half
        const int off = (PAR == 1 && b == 0) ? 1 : 0;
        const uint32_t sel = ((PAR == 0) == (b == 0)) ? 0x7632u : 0x5410u;
        uint32_t v[16];
#pragma unroll
        for (int kg = 0; kg < 4; ++kg)
#pragma unroll
            for (int w = 0; w < 4; ++w)
                v[4 * kg + w] = __byte_perm(W[off + 31 - 8 * kg - 2 * w],
                                            W[off + 30 - 8 * kg - 2 * w], sel);
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
            "%12,%13,%14,%15,%16};" ::"r"(taddr + (uint32_t)((2 * b + q) * 16)),
            "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
            "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]),
            "r"(v[14]), "r"(v[15])
            : "memory");
    }
}

// D (TMEM) (+)= A (TMEM, K-major bf16 pairs) B (shared-memory descriptor), instruction
// descriptor idesc (kIdesc with its N field replaced for narrower MMAs).
__device__ __forceinline__ void mma_f16_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t acc,
                                           uint32_t idesc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar));
}

__global__ void __launch_bounds__(P_NT, 1)
k_conv_tcp(const ConvJob *__restrict__ jobs, const Tile *__restrict__ tiles, int n_tiles,
           int max_lh, const float *__restrict__ h, const float *__restrict__ src,
           float *__restrict__ y, double *__restrict__ part, int h_aligned16,
           const WaitCtl wc) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[P_NS], bar_empty[P_NS], bar_win[2], bar_accf[2],
        bar_acce[2], bar_done, bar_never;
    __shared__ double s_red[2][4];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const PLayout Lay = p_layout(max_lh);
    const int bl = Lay.bl;
    const int n_my = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1
                                               : 0;

    if (tid == 0) {
        for (int s = 0; s < P_NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[s])),
                         "r"(P_NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_empty[s])),
                         "r"(1));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_win[b])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_accf[b])),
                         "r"(1));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_acce[b])),
                         "r"(128));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_done)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_never)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (warp < 8) {
        // ------------------------------------------------------------------
        // producers: warps 0-3 build the hi operands, warps 4-7 the lo ones;
        // in each group warps 0, 1 take the even phases, warps 2, 3 the odd
        // ------------------------------------------------------------------
        const int q = warp >> 2;
        const int par = (warp >> 1) & 1;
        const int i64 = (warp & 1) * 32 + lane;
        // operand row R = 64 par + 8 m + j (the warp's TMEM lane quadrant,
        // warp % 4, times 32, plus its lane) holds phase p = 2 j + par of mic m
        const int m = i64 >> 3, p = 2 * (i64 & 7) + par;
        const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
        float *stg = reinterpret_cast<float *>(smem + Lay.stg);
        const uint32_t stg_u32 = smem_u32(stg);
        uint32_t *cvb0 = reinterpret_cast<uint32_t *>(smem + Lay.cv);
        // this thread's raw staging pairs w = tid + P_NPROD r (elements 2 w,
        // 2 w + 1: mic st_mm, offsets st_ee, st_ee + 1), or, for RIRs whose
        // rows start on 16-byte boundaries, its quad tid < P_STG / 4 (elements
        // 4 tid .. 4 tid + 3: mic qd_mm, offset qd_ee) in one 16-byte copy.  A
        // thread converts exactly the values it staged, so its own cp.async
        // wait covers them.
        constexpr int SR = (P_STG / 2 + P_NPROD - 1) / P_NPROD;
        int st_mm[SR], st_ee[SR];
#pragma unroll
        for (int r = 0; r < SR; ++r) {
            const int w = tid + P_NPROD * r;
            st_mm[r] = w / 40;
            st_ee[r] = 2 * w - 80 * st_mm[r];
        }
        static_assert(P_STG / 4 <= P_NPROD, "one quad per thread");
        const int qd_mm = tid / 20, qd_ee = 4 * tid - 80 * qd_mm;
        int gi = 0;  // chunks produced by this CTA so far
        int gu = 0;  // units (segment windows) of this CTA so far
        // the window of segment sg of tile T into buffer wb, words [w_lo, w_hi)
        // of each array
        auto convert_window = [&](const PTile &T, int sg, int wb, int w_lo, int w_hi) {
            const ConvJob &J = jobs[T.tl.job];
            const float *sb = src + J.src_offset;
            const int64_t base = p_seg_base(T, sg);
            uint32_t *w = reinterpret_cast<uint32_t *>(smem + Lay.win + wb * Lay.win_bytes);
            for (int e2 = w_lo + tid; e2 < w_hi; e2 += P_NPROD)
                store_decimated(w + e2, bl / 2, sb, base + 4 * (int64_t)e2, T.Ts);
        };
        // the window buffer of unit g is free once unit g - 2's MMAs are done
        auto wait_window = [&](int g) {
            if (g >= 2 && !mbar_wait(smem_u32(&bar_win[g & 1]), ((g >> 1) - 1) & 1, wc))
                s_abort = 1;
        };
        if (n_my > 0) {
            const PTile T = p_tile(jobs, tiles, (int)blockIdx.x);
            convert_window(T, 0, 0, 0, p_seg_words(T, 0));
            // the window's stores before the first chunk's arrivals, for the MMAs
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        for (int lt = 0; lt < n_my; ++lt) {
            const PTile T = p_tile(jobs, tiles, (int)blockIdx.x + lt * (int)gridDim.x);
            const ConvJob &J = jobs[T.tl.job];
            const float *hb = h + J.h_offset + (int64_t)T.tl.mic0 * T.Lh;
            // every row start and chunk offset a multiple of 4 elements
            const bool quad = h_aligned16 && (T.Lh & 3) == 0 && (J.h_offset & 3) == 0;
            auto stage_rir = [&](int ch, int buf) {
                // stg[buf][mm][e] = h_mm[Lh - 64 - 64 ch + e], e in [0, 80)
                const int64_t start = T.Lh - 64 - (int64_t)ch * P_KC;
                if (quad) {
                    if (tid < P_STG / 4) {
                        // idx and Lh multiples of 4: the quad is all in or all out
                        const int64_t idx = start + qd_ee;
                        const bool ok = qd_mm < T.nm && idx >= 0 && idx < T.Lh;
                        cp_async16(stg_u32 + 16u * (uint32_t)(buf * (P_STG / 4) + tid),
                                   ok ? hb + (int64_t)qd_mm * T.Lh + idx : hb, ok);
                    }
                    asm volatile("cp.async.commit_group;" ::: "memory");
                    return;
                }
#pragma unroll
                for (int r = 0; r < SR; ++r) {
                    const int w = tid + P_NPROD * r;
                    if (w < P_STG / 2) {
                        const float *row = hb + (int64_t)st_mm[r] * T.Lh;
#pragma unroll
                        for (int c = 0; c < 2; ++c) {
                            const int64_t idx = start + st_ee[r] + c;
                            const bool ok = st_mm[r] < T.nm && idx >= 0 && idx < T.Lh;
                            cp_async4(stg_u32 + 4u * (uint32_t)(buf * P_STG + 2 * w + c),
                                      ok ? row + idx : hb, ok);
                        }
                    }
                }
                asm volatile("cp.async.commit_group;" ::: "memory");
            };
            // one cp.async group per chunk, P_PD chunks ahead (empty groups
            // keep the count when the tile has fewer)
            for (int k = 0; k < P_PD; ++k) {
                if (k < T.n_live) stage_rir(T.ch_lo + k, k);
                else asm volatile("cp.async.commit_group;" ::: "memory");
            }
            bool aborted = false;
            const int nu = p_units(T);
            int i = 0;  // chunk of the tile
            for (int sg = 0; sg < nu; ++sg, ++gu) {
                // the next unit: this tile's next segment, else the next tile's
                // first; its window is converted a slice per chunk of this unit
                const bool same = sg + 1 < nu;
                const bool has_next = same || lt + 1 < n_my;
                const PTile Tn =
                    (!same && has_next)
                        ? p_tile(jobs, tiles, (int)blockIdx.x + (lt + 1) * (int)gridDim.x)
                        : T;
                const int sgn = same ? sg + 1 : 0;
                const int next_words = has_next ? p_seg_words(Tn, sgn) : 0;
                const int64_t nbase = p_seg_base(Tn, sgn);
                int next_pos = 0;
                bool next_waited = false;
                // source samples of this thread's word (next_pos + tid) of the
                // next slice, loaded one chunk before they are stored
                const float *sbn = src + jobs[Tn.tl.job].src_offset;
                uint32_t *wn =
                    reinterpret_cast<uint32_t *>(smem + Lay.win + ((gu + 1) & 1) * Lay.win_bytes);
                float px[4];
                if (tid < next_words) load_source4(px, sbn, nbase + 4 * (int64_t)tid, Tn.Ts);
                if (p_producers_any(s_abort)) {
                    aborted = true;
                    break;
                }
                const int i_end = min(T.n_live, (sg + 1) * P_SEG);
                for (; i < i_end; ++i, ++gi) {
                    const int ch = T.ch_lo + i, s = gi % P_NS, u = gi / P_NS, buf = i % P_PB;
                    const int il = i - sg * P_SEG;  // chunk of the unit
                    asm volatile("cp.async.wait_group %0;" ::"n"(P_PD - 1) : "memory");
                    const bool ok =
                        (u == 0) || mbar_wait(smem_u32(&bar_empty[s]), (u - 1) & 1, wc);
                    // the chunk as bf16 pairs (the pairs this thread staged), into
                    // the converted buffer that chunk gi - 2 read (every producer
                    // passed chunk gi - 1's barrier after its reads)
                    uint32_t *cvb = cvb0 + (gi & 1) * P_CVW;
                    if (quad) {
                        if (tid < P_STG / 4) {
                            const float4 x =
                                reinterpret_cast<const float4 *>(stg + buf * P_STG)[tid];
                            const float h0 = bf16_round(x.x), h1 = bf16_round(x.y);
                            const float h2 = bf16_round(x.z), h3 = bf16_round(x.w);
                            reinterpret_cast<uint2 *>(cvb)[tid] =
                                make_uint2(pack_bf16(h0, h1), pack_bf16(h2, h3));
                            reinterpret_cast<uint2 *>(cvb + P_STG / 2)[tid] = make_uint2(
                                pack_bf16(x.x - h0, x.y - h1), pack_bf16(x.z - h2, x.w - h3));
                        }
                    } else {
                        const float2 *sv2 = reinterpret_cast<const float2 *>(stg + buf * P_STG);
                        for (int w = tid; w < P_STG / 2; w += P_NPROD) {
                            const float2 x = sv2[w];
                            const float h0 = bf16_round(x.x), h1 = bf16_round(x.y);
                            cvb[w] = pack_bf16(h0, h1);
                            cvb[P_STG / 2 + w] = pack_bf16(x.x - h0, x.y - h1);
                        }
                    }
                    // one barrier: conversions visible, stg[buf] free again, and a
                    // uniform abort decision before the stage is written
                    if (p_producers_any(!ok || s_abort)) {
                        s_abort = 1;
                        aborted = true;
                        break;
                    }
                    // buffer (i + P_PD) % P_PB was last read by chunk i - 1's conversion
                    if (i + P_PD < T.n_live) stage_rir(ch + P_PD, (i + P_PD) % P_PB);
                    else asm volatile("cp.async.commit_group;" ::: "memory");
                    // stage s's TMEM columns are free (its MMAs completed)
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t ta = tmem + tlane + (uint32_t)(P_ACOL + s * P_SCOL);
                    if (par) p_rows<1>(cvb, ta, m, p, q);
                    else p_rows<0>(cvb, ta, m, p, q);
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    mbar_arrive(smem_u32(&bar_full[s]));
                    // a slice of the next unit's window, after the chunk is released
                    // (read by the MMAs of the next unit only: the proxy fence at the
                    // end of this unit orders these writes before its arrivals)
                    if (next_pos < next_words && il >= P_NS) {
                        if (!next_waited) {
                            wait_window(gu + 1);
                            next_waited = true;
                        }
                        const int e2 = next_pos + tid;
                        if (e2 < next_words && ISM_IN_RANGE(e2 < bl / 2, kOobTcpWindow))
                            store_split4(wn + e2, bl / 2, px);
                        next_pos += P_NPROD;
                        if (e2 + P_NPROD < next_words)
                            load_source4(px, sbn, nbase + 4 * (int64_t)(e2 + P_NPROD), Tn.Ts);
                    }
                }
                if (aborted) break;
                if (next_pos < next_words) {
                    if (!next_waited) wait_window(gu + 1);
                    const int e2 = next_pos + tid;
                    if (e2 < next_words && ISM_IN_RANGE(e2 < bl / 2, kOobTcpWindow))
                        store_split4(wn + e2, bl / 2, px);
                    convert_window(Tn, sgn, (gu + 1) & 1, next_pos + P_NPROD, next_words);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (aborted) break;
        }
    } else if (warp == 8) {
        // ------------------------------------------------------------------
        // MMA issuer (one lane)
        // ------------------------------------------------------------------
        if (lane == 0) {
            int gi = 0, gu = 0;
            // test aid: a wait that nothing ends, before any MMA is issued
            if (wc.inject && !mbar_wait(smem_u32(&bar_never), 0, wc)) s_abort = 1;
            for (int lt = 0; lt < n_my && !s_abort; ++lt) {
                const PTile T = p_tile(jobs, tiles, (int)blockIdx.x + lt * (int)gridDim.x);
                // one accumulator: the previous tile's epilogue has drained it
                if (lt >= 1 && !mbar_wait(smem_u32(&bar_acce[0]), (lt - 1) & 1, wc)) {
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t d = tmem;
                const uint32_t wstr = (uint32_t)bl * 2u;
                uint32_t acc = 0;
                bool aborted = false;
                const int nu = p_units(T);
                int i = 0;  // chunk of the tile
                for (int sg = 0; sg < nu && !aborted; ++sg, ++gu) {
                    const uint32_t w0 = smem_u32(smem + Lay.win + (gu & 1) * Lay.win_bytes);
                    const int i_end = min(T.n_live, (sg + 1) * P_SEG);
                    for (; i < i_end; ++i, ++gi) {
                        const int ch = T.ch_lo + i, s = gi % P_NS, u = gi / P_NS;
                        const int cw = i - sg * P_SEG;  // chunk of the unit's window
                        if (!mbar_wait(smem_u32(&bar_full[s]), u & 1, wc)) {
                            s_abort = 1;
                            aborted = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t a0 = tmem + (uint32_t)(P_ACOL + s * P_SCOL);
                        // live columns: column n of chunk ch reads source samples
                        // base + 16 n + [0, 64); the others only multiply zero
                        // padding and are left out (the tile's first chunk takes
                        // all 256 columns, which initialises the accumulator).
                        // Rounded to 32 columns, the TMEM allocation granularity.
                        int n0 = 0, nw = NN;
                        if (i > 0) {
                            const int64_t base = T.c0 + (int64_t)P_KC * ch;
                            const int64_t lo = -((63 + base) >> 4);     // ceil((-63 - base) / 16)
                            const int64_t hi = (T.Ts - 1 - base) >> 4;  // floor
                            const int nl = lo > 0 ? (int)lo : 0,
                                      nh = hi < NN - 1 ? (int)hi : NN - 1;
                            if (nl <= nh) {
                                n0 = nl & ~31;
                                nw = ((nh | 31) + 1) - n0;
                            }
                        }
                        const uint32_t idesc =
                            (kIdesc & ~(0x3Fu << 17)) | ((uint32_t)(nw >> 3) << 17);
                        const uint32_t dn = d + (uint32_t)n0;
                        // the last window element the chunk's MMAs read (per parity array)
                        if (!ISM_IN_RANGE(32 * cw + 16 + 15 + 8 * (n0 + nw - 1) < bl,
                                          kOobTcpOperand)) {
                            mma_commit(smem_u32(&bar_empty[s]));
                            continue;
                        }
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                            for (int b = 0; b < 2; ++b) {
                                // A (hi, lo) of parity b, k-slice kk: 8 TMEM columns each
                                const uint32_t ahi = a0 + (uint32_t)((2 * b) * 16 + 8 * kk);
                                const uint32_t alo = ahi + 16u;
                                const uint32_t bb = w0 + 64u * (uint32_t)cw + 32u * (uint32_t)kk +
                                                    16u * (uint32_t)n0;
                                const uint64_t bhi = make_desc(bb + (2 * b) * wstr, 16, 128);
                                const uint64_t blo = make_desc(bb + (2 * b + 1) * wstr, 16, 128);
                                mma_f16_ts(dn, ahi, bhi, acc, idesc);
                                acc = 1;
                                mma_f16_ts(dn, alo, bhi, 1, idesc);
                                mma_f16_ts(dn, ahi, blo, 1, idesc);
                            }
                        }
                        mma_commit(smem_u32(&bar_empty[s]));
                    }
                    mma_commit(smem_u32(&bar_win[gu & 1]));  // the unit's window buffer free
                }
                mma_commit(smem_u32(&bar_accf[0]));  // the tile's MMAs done
                if (aborted) break;
            }
            mma_commit(smem_u32(&bar_done));
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------------
        // epilogue (warps 9-12): TMEM lane quadrant warp % 4 = rows 32 qd ..
        // 32 qd + 31 = (par = R / 64, m = (R / 8) % 8, p = 2 (R % 8) + par);
        // column n is output T0 + 16 n + p
        // ------------------------------------------------------------------
        const int qd = warp & 3;
        const int R = 32 * qd + lane, m = (R >> 3) & 7, p = 2 * (R & 7) + (R >> 6);
        const int et = tid - 288;  // 0..127
        for (int lt = 0; lt < n_my; ++lt) {
            const PTile T = p_tile(jobs, tiles, (int)blockIdx.x + lt * (int)gridDim.x);
            const ConvJob &J = jobs[T.tl.job];
            const int ab = lt & 1;  // s_red buffer
            // after an abort the remaining tiles are written as zeros at once;
            // a wait of its own that runs out aborts the CTA (its later
            // accumulator phases would no longer match)
            bool ok = !s_abort;
            if (ok && !mbar_wait(smem_u32(&bar_accf[0]), lt & 1, wc)) {
                s_abort = 1;
                ok = false;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            ok = ok && !s_abort && T.n_live > 0;
            const int64_t ylen = J.y_len;
            float *ym = y + J.y_offset + (int64_t)(T.tl.mic0 + m) * ylen;
            float ss = 0.f, se = 0.f;
            for (int cb = 0; cb < NN; cb += 32) {
                uint32_t r[32];
                if (ok) {
                    const uint32_t addr =
                        tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)cb;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                        "%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,"
                        "%29,%30,%31}, [%32];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                          "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]),
                          "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                          "=r"(r[31])
                        : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) r[j] = 0u;
                }
                if (m < T.nm) {
                    // outputs t0 + 16 j of this row: one base address and
                    // immediate offsets; the bounds test only on the block
                    // that the signal's end cuts.  The block's squares are
                    // summed in FP32 (four chains of eight positive terms,
                    // within 5e-7), then added to the float-float sum.
                    const int64_t t0 = T.T0 + P_PH * cb + p;
                    float *yo = ym + t0;
                    float q[4] = {0.f, 0.f, 0.f, 0.f};
                    if (t0 + P_PH * 31 < ylen) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float v = __uint_as_float(r[j]);
                            yo[P_PH * j] = v;
                            q[j & 3] = __fmaf_rn(v, v, q[j & 3]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float v = __uint_as_float(r[j]);
                            if (t0 + P_PH * j < ylen) {
                                yo[P_PH * j] = v;
                                q[j & 3] = __fmaf_rn(v, v, q[j & 3]);
                            }
                        }
                    }
                    // (ss, se) += the block's sum: two-sum, error into se
                    const float x = __fadd_rn(__fadd_rn(q[0], q[1]), __fadd_rn(q[2], q[3]));
                    const float t = __fadd_rn(ss, x);
                    const float bb = __fsub_rn(t, ss);
                    se = __fadd_rn(se, __fadd_rn(__fsub_rn(ss, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
                    ss = t;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(smem_u32(&bar_acce[0]));  // the accumulator may be refilled
            const double rs = warp_sum_f64((double)ss + (double)se);
            if (lane == 0) s_red[ab][qd] = rs;
            asm volatile("bar.sync 2, 128;" ::: "memory");
            if (et == 0 && part) {
                // the tile spans two slots of the noise-partial grid: its sum
                // in the first, zero in the second
                const int np = conv_partials_per_job(J.n_mics, ylen);
                const int s0 = conv_partial_slot(T.tl.mic0, T.T0, ylen);
                if (ISM_IN_RANGE(s0 >= 0 && s0 < np, kOobTcpPartial))
                    part[J.part_offset + s0] =
                        (s_red[ab][0] + s_red[ab][1]) + (s_red[ab][2] + s_red[ab][3]);
                if (T.T0 + kConvTT < ylen) {
                    const int s1 = conv_partial_slot(T.tl.mic0, T.T0 + kConvTT, ylen);
                    if (ISM_IN_RANGE(s1 >= 0 && s1 < np, kOobTcpPartial))
                        part[J.part_offset + s1] = 0.0;
                }
            }
        }
    }
    __syncthreads();
    if (warp == 8) {
        // every issued MMA has completed before the columns are freed
        mbar_wait(smem_u32(&bar_done), 0, wc);
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// Raises a kernel's dynamic shared memory limit to smem once per device
// (the attribute call is not repeated for calls of the same or smaller size).
template <class K>
cudaError_t ensure_smem(K kern, int (&set)[64], std::mutex &mu, size_t smem) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d < 0 || d >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if ((size_t)set[d] >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) set[d] = (int)smem;
    return e;
}

std::mutex g_smem_mu;
int g_smem_persistent[64];

}  // namespace

ISM_OOB_READER(conv_tc)

int64_t conv_bf16x3_persistent_tiles(int n_mics, int64_t rir_len, int64_t y_len) {
    if (p_layout(rir_len).total > kMaxDynSmem) return -1;
    return (int64_t)((n_mics + MG - 1) / MG) * ((y_len + P_TT - 1) / P_TT);
}

int conv_bf16x3_plan(const ConvLaunch &L, ConvPlan *P) {
    // every RIR on the persistent three-product kernel (long RIRs in segment
    // windows), batch and served calls alike: a job's tiles depend on the
    // job alone, so its result is the same in any batch.  The tiles go to
    // the CTAs longest RIR first: the CTAs take them in rounds, and a round
    // lasts as long as its longest tile.
    std::vector<Tile> ptiles;
    int64_t p_max_lh = 0;
    for (int j = 0; j < L.n_jobs; ++j) {
        const ConvJob &J = L.jobs_host[j];
        p_max_lh = std::max(p_max_lh, J.rir_len);
        for (int m0 = 0; m0 < J.n_mics; m0 += MG)
            for (int64_t t0 = 0; t0 < J.y_len; t0 += P_TT) ptiles.push_back(Tile{j, m0, t0});
    }
    if (ptiles.size() > 0x7fffffffULL) return fail(ISM_ERR_INVALID_ARG, "too many tiles");
    std::stable_sort(ptiles.begin(), ptiles.end(), [&](const Tile &a, const Tile &b) {
        return L.jobs_host[a.job].rir_len > L.jobs_host[b.job].rir_len;
    });
    P->precision = ISM_BF16X3;
    P->tiles = std::move(ptiles);
    P->p_max_lh = p_max_lh;
    return ISM_OK;
}

int conv_bf16x3_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                        cudaStream_t stream) {
    WaitCtl wc{L.err_dev, kWaitNs, 0};
    if (L.inject) {
        wc.inject = 1;
        wc.limit_ns = 20000000ull;  // 20 ms: the injected wait and the aborts it causes
    }
    if (P.tiles.empty()) return ISM_OK;
    const size_t smem = p_layout(P.p_max_lh).total;
    cudaError_t e = ensure_smem(k_conv_tcp, g_smem_persistent, g_smem_mu, smem);
    const int grid = (int)std::min<size_t>(P.tiles.size(), (size_t)device_sm_count());
    if (e == cudaSuccess)
        k_conv_tcp<<<grid, P_NT, smem, stream>>>(
            L.jobs_dev, d_tiles, (int)P.tiles.size(), (int)P.p_max_lh, L.h_dev, L.src_dev,
            L.y_dev, L.noise_partials_dev, (int)(((uintptr_t)L.h_dev & 15) == 0), wc);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_conv_tcp");
    return ISM_OK;
}

int launch_conv_bf16x3(const ConvLaunch &L, cudaStream_t stream) {
    ConvPlan P;
    if (int st = conv_bf16x3_plan(L, &P)) return st;
    if (P.tiles.empty()) return ISM_OK;
    void *d_tiles = nullptr;
    int st = scratch_alloc(&d_tiles, P.tiles.size() * sizeof(Tile), stream);
    if (st) return st;
    st = upload_async(d_tiles, P.tiles.data(), P.tiles.size() * sizeof(Tile), stream);
    if (!st) st = conv_bf16x3_enqueue(L, P, (const Tile *)d_tiles, stream);
    scratch_free(d_tiles, stream);
    return st;
}

}  // namespace ism
