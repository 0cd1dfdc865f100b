// ism_conv_tc.cu -- K2: the convolution y_m = s * h_m on the tcgen05 tensor
// cores, in split BF16 (each FP32 operand as bf16 hi + lo, FP32 accumulate).
//
// Convolution (arXiv 2104.13347, Sec. II.A: the dataset is built by batch
// convolution of the RIRs with source signals), for every mic m of a room:
//   y_m[t] = sum_k h_m[k] s[t - k],  t in [0, Ts + Lh - 1).
//
// Block-Toeplitz GEMM.  A tile of 2048 outputs t = T0 + 8n + p (n < 256
// columns, p < 8 phases) of 8 mics is one GEMM D (128 x 256) = A (128 x K) B
// (K x 256) over the RIR taps:
//   B[k][n] = s[c + k + 8n],  c = T0 - Lh + 1      (source, forward)
//   A[(q,m,p)][k] = part_q(h_m[Lh - 1 + p - k])    (RIR, reversed, phase p)
// so that D[(q,m,p)][n] = sum_k A B accumulates, over q in {hi, lo},
// y_m[T0 + 8n + p] (each row's j = Lh-1+p-k runs over the whole RIR).
// B is a Toeplitz matrix whose rows shift by 8 elements = 16 bytes, so it is
// read straight from a linear copy of the source in shared memory through a
// no-swizzle K-major descriptor with leading-dimension offset 16 B and
// stride offset 128 B (core matrices overlap); A is materialised per chunk
// of 64 taps (8 phases x 8 mics x hi/lo = 128 rows, 16 KB).  Per chunk the
// MMA issuer runs 4 K-steps x {B_hi, B_lo} = 8 MMAs of 128 x 256 x 16 into
// one TMEM accumulator, so the result holds all four products hi/lo x hi/lo.
// Chunks whose source window is all zero padding are skipped.
//
// The tile's whole source window is converted to bf16 hi/lo once at the
// start when it fits in shared memory (RIRs up to ~9k samples); longer RIRs
// convert each chunk's 2112-sample window into its pipeline stage instead.
// The raw RIR values of each chunk are staged with cp.async (double
// buffered, zero-filled outside the RIR) and each producer thread builds one
// 16-byte row (one row group, one phase) per k-group, so a warp's 128-bit
// stores cover 512 contiguous bytes.
//
// Warp roles (160 threads): warps 0-3 produce the pipeline stages and run
// the epilogue; warp 4 allocates TMEM and one of its lanes issues the MMAs.  Stages hand over through mbarriers
// (full: 128 producer arrivals; empty: tcgen05.commit).  Every wait is
// bounded: on timeout the kernel records an error, stops issuing, waits
// (bounded) for its own MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "ism_internal.h"

namespace ism {

__device__ int g_conv_tc_error;  // set to 1 by a timed-out wait

namespace {

constexpr int KC = 64;                 // RIR taps per chunk
constexpr int NN = 256;                // GEMM N: time groups of 8
constexpr int TT = 8 * NN;             // outputs per tile (2048)
constexpr int MG = 8;                  // mics per tile
static_assert(TT == kConvTT && MG == kConvMG, "tile shape of the noise partials");
constexpr int NS = 4;                  // pipeline stages
constexpr int BW = 2112;               // source window per chunk (>= KC + 8 (NN-1), x8)
constexpr int A_BYTES = 8 * 16 * 128;  // 8 k-groups x 16 row groups x 8 rows x 16 B
constexpr int STAGE = A_BYTES + 2 * BW * 2;
constexpr int NPROD = 128;             // producer threads (warps 0-3)
constexpr int NTHR = 160;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s bound on any mbarrier wait

struct Tile {
    int job;
    int mic0;
    int64_t t0;
};

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

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the given phase parity of an mbarrier, at most kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
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
        if (global_ns() - t0 > kWaitNs) break;
    }
    atomicExch(&g_conv_tc_error, 1);
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

constexpr int STG_FLOATS = 8 * 72;     // raw RIR staging per chunk: 8 mics x 72 values
constexpr int CV_WORDS = 2 * 8 * 36;   // one chunk's RIR as bf16 pairs: [hi/lo][mic][36 words]
constexpr int CV_BYTES = CV_WORDS * 4;

__device__ __forceinline__ void cp_async4(uint32_t dst, const float *src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
                 "r"(ok ? 4 : 0)
                 : "memory");
}

// OR of pred over the 128 producer threads (named barrier 1); also a barrier.
__device__ __forceinline__ bool producers_any(bool pred) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, 128, p;\n"
        "selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void producers_sync() {
    asm volatile("bar.sync 1, 128;" ::: "memory");
}

// Shared-memory layout.  whole_b: NS A stages (16 KB each), RIR staging
// (two raw chunks), the converted RIR (one chunk of bf16 hi / lo: the
// barrier that opens each chunk orders every read of it before the next
// conversion), then the tile's source window (bf16 hi, bf16 lo; bl elements
// each).  Otherwise NS stages of (A, window hi, window lo), then the RIR
// staging and conversion.
struct TcLayout {
    size_t a_stride, stg, cv, bhi, blo, total;
    int bl;
};

__host__ __device__ inline TcLayout tc_layout(bool whole_b, int n_chunks) {
    TcLayout L;
    if (whole_b) {
        L.bl = (n_chunks * KC + 8 * (NN - 1) + 8 + 7) & ~7;
        L.a_stride = A_BYTES;
        L.stg = (size_t)NS * A_BYTES;
        L.cv = L.stg + STG_FLOATS * 2 * 4;
        L.bhi = L.cv + CV_BYTES;
        L.blo = L.bhi + (size_t)L.bl * 2;
        L.total = L.blo + (size_t)L.bl * 2;
    } else {
        L.bl = BW;
        L.a_stride = STAGE;
        L.stg = (size_t)NS * STAGE;
        L.cv = L.stg + STG_FLOATS * 2 * 4;
        L.bhi = L.blo = 0;  // per stage, after A
        L.total = L.cv + CV_BYTES;
    }
    return L;
}

template <bool WHOLE_B>
__global__ void __launch_bounds__(NTHR, 1)
k_conv_tc(const ConvJob *__restrict__ jobs, const Tile *__restrict__ tiles,
          const float *__restrict__ h, const float *__restrict__ src, float *__restrict__ y,
          double *__restrict__ part) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[NS], bar_empty[NS], bar_done;
    __shared__ double s_red[2];
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Tile tl = tiles[blockIdx.x];
    const ConvJob J = jobs[tl.job];
    const int64_t Lh = J.rir_len, Ts = J.src_len, T0 = tl.t0;
    const int nm = min(MG, J.n_mics - tl.mic0);
    const float *hb = h + J.h_offset + (int64_t)tl.mic0 * Lh;
    const float *sb = src + J.src_offset;
    const int64_t c0 = T0 - Lh + 1;                    // source index of B[0][0] at k = 0
    const int n_chunks = (int)((Lh + 7 + KC - 1) / KC);
    const TcLayout Lay = tc_layout(WHOLE_B, n_chunks);
    // live chunks (source window not all zero padding) form one range
    int64_t lo_c = -c0 - (KC - 1 + 8 * (NN - 1));
    lo_c = lo_c <= 0 ? 0 : (lo_c + KC - 1) / KC;
    int64_t hi_c = Ts - 1 - c0;
    hi_c = hi_c < 0 ? -1 : hi_c / KC;
    const int ch_lo = (int)lo_c, ch_hi = (int)min(hi_c, (int64_t)n_chunks - 1);
    const int n_live = ch_hi >= ch_lo ? ch_hi - ch_lo + 1 : 0;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_full[s])),
                         "r"(NPROD));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_empty[s])),
                         "r"(1));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar_done)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    if (WHOLE_B && n_live > 0) {
        // the tile's source window s[c0 + e], e in [0, bl), as bf16 hi / lo
        uint32_t *bh = reinterpret_cast<uint32_t *>(smem + Lay.bhi);
        uint32_t *bl = reinterpret_cast<uint32_t *>(smem + Lay.blo);
        for (int e2 = tid; e2 < Lay.bl / 2; e2 += NTHR) {
            const int64_t i0 = c0 + 2 * e2;
            const float x0 = (i0 >= 0 && i0 < Ts) ? __ldg(sb + i0) : 0.f;
            const float x1 = (i0 + 1 >= 0 && i0 + 1 < Ts) ? __ldg(sb + i0 + 1) : 0.f;
            const float h0 = bf16_round(x0), h1 = bf16_round(x1);
            bh[e2] = pack_bf16(h0, h1);
            bl[e2] = pack_bf16(x0 - h0, x1 - h1);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = s_tmem;

    if (warp < 4) {
        // ------------------------------------------------------------------
        // producers: thread = (row group g = (q, m), phase p)
        // ------------------------------------------------------------------
        const int g = tid >> 3, q = g >> 3, m = g & 7, p = tid & 7;
        float *stg = reinterpret_cast<float *>(smem + Lay.stg);
        const uint32_t stg_u32 = smem_u32(stg);
        auto stage_rir = [&](int ch, int buf) {
            // stg[buf][mm][e] = h_mm[Lh - 64 - 64 ch + e], e in [0, 72)
            const int64_t start = Lh - 64 - (int64_t)ch * KC;
            for (int e = tid; e < STG_FLOATS; e += NPROD) {
                const int mm = e / 72, ee = e - mm * 72;
                const int64_t idx = start + ee;
                const bool ok = mm < nm && idx >= 0 && idx < Lh;
                cp_async4(stg_u32 + 4u * (uint32_t)(buf * STG_FLOATS + e),
                          ok ? hb + (int64_t)mm * Lh + idx : hb, ok);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        if (n_live > 0) stage_rir(ch_lo, 0);
        if (n_live > 1) stage_rir(ch_lo + 1, 1);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        uint32_t *cvb = reinterpret_cast<uint32_t *>(smem + Lay.cv);
        const uint32_t sel = (p & 1) ? 0x3254u : 0x1032u;  // see the row build below
        for (int i = 0; i < n_live; ++i) {
            const int ch = ch_lo + i, s = i % NS, u = i / NS, buf = i & 1;
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            const bool ok = (u == 0) || mbar_wait(smem_u32(&bar_empty[s]), (u - 1) & 1);
            if (producers_any(!ok || s_abort)) {  // uniform decision, also a barrier
                s_abort = 1;
                break;
            }
            // (1) the staged chunk as bf16 pairs, once per value:
            // cv[q][mm][w] = (part_q(stg[mm][2w]), part_q(stg[mm][2w + 1]))
            {
                const float2 *sv2 = reinterpret_cast<const float2 *>(stg + buf * STG_FLOATS);
                uint32_t *cv = cvb;
                for (int w = tid; w < STG_FLOATS / 2; w += NPROD) {
                    const float2 x = sv2[w];
                    const float h0 = bf16_round(x.x), h1 = bf16_round(x.y);
                    cv[w] = pack_bf16(h0, h1);
                    cv[STG_FLOATS / 2 + w] = pack_bf16(x.x - h0, x.y - h1);
                }
            }
            producers_sync();  // conversions visible; stg[buf] free again
            if (i + 2 < n_live) stage_rir(ch + 2, buf);
            else asm volatile("cp.async.commit_group;" ::: "memory");
            // (2) A rows (q, m, p) for each k-group kg: element kr is
            // part_q(h_m[Lh - 1 + p - 64 ch - 8 kg - kr]) = part_q(stg[m][63 + p - 8 kg - kr]).
            // With p = 2a + o and V[i] = cv[q][m][a + i], word j of row kg
            // (elements kr = 2j, 2j + 1) is, for o = 1, the low half of
            // V[32 - 4 kg - j] and the high half of V[31 - 4 kg - j]
            // (byte_perm selector 0x3254); for o = 0, the two halves of
            // V[31 - 4 kg - j] swapped (0x1032).
            {
                const uint32_t *cv = cvb + q * (STG_FLOATS / 2) + m * 36 + (p >> 1);
                uint32_t V[33];
#pragma unroll
                for (int k = 0; k < 33; ++k) V[k] = cv[k];
                unsigned char *st = smem + (size_t)s * Lay.a_stride;
#pragma unroll
                for (int kg = 0; kg < 8; ++kg) {
                    uint4 row;
                    row.x = __byte_perm(V[31 - 4 * kg], V[32 - 4 * kg], sel);
                    row.y = __byte_perm(V[30 - 4 * kg], V[31 - 4 * kg], sel);
                    row.z = __byte_perm(V[29 - 4 * kg], V[30 - 4 * kg], sel);
                    row.w = __byte_perm(V[28 - 4 * kg], V[29 - 4 * kg], sel);
                    *reinterpret_cast<uint4 *>(st + kg * 2048 + g * 128 + p * 16) = row;
                }
            }
            if (!WHOLE_B) {
                // the chunk's source window, s[c0 + 64 ch + e], split hi / lo
                unsigned char *st = smem + (size_t)s * Lay.a_stride;
                uint32_t *bh = reinterpret_cast<uint32_t *>(st + A_BYTES);
                uint32_t *bl = reinterpret_cast<uint32_t *>(st + A_BYTES + BW * 2);
                const int64_t sbase = c0 + (int64_t)ch * KC;
                for (int e2 = tid; e2 < BW / 2; e2 += NPROD) {
                    const int64_t i0 = sbase + 2 * e2;
                    const float x0 = (i0 >= 0 && i0 < Ts) ? __ldg(sb + i0) : 0.f;
                    const float x1 = (i0 + 1 >= 0 && i0 + 1 < Ts) ? __ldg(sb + i0 + 1) : 0.f;
                    const float h0 = bf16_round(x0), h1 = bf16_round(x1);
                    bh[e2] = pack_bf16(h0, h1);
                    bl[e2] = pack_bf16(x0 - h0, x1 - h1);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(smem_u32(&bar_full[s]));
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (lane == 0) {
        // ------------------------------------------------------------------
        // MMA issuer
        // ------------------------------------------------------------------
        uint32_t acc = 0;
        for (int i = 0; i < n_live; ++i) {
            const int ch = ch_lo + i, s = i % NS, u = i / NS;
            if (!mbar_wait(smem_u32(&bar_full[s]), u & 1)) {
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(smem + (size_t)s * Lay.a_stride);
            uint32_t bh0, bl0;
            if (WHOLE_B) {
                bh0 = smem_u32(smem + Lay.bhi) + 2u * (uint32_t)(ch * KC);
                bl0 = smem_u32(smem + Lay.blo) + 2u * (uint32_t)(ch * KC);
            } else {
                bh0 = a0 + A_BYTES;
                bl0 = bh0 + BW * 2;
            }
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
                const uint64_t ad = make_desc(a0 + kk * 2 * 2048, 2048, 128);
                const uint64_t bhd = make_desc(bh0 + kk * 32, 16, 128);
                const uint64_t bld = make_desc(bl0 + kk * 32, 16, 128);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bhd), "r"(kIdesc), "r"(acc));
                acc = 1;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bld), "r"(kIdesc), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&bar_empty[s])));
        }
        // all issued MMAs done -> bar_done
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar_done)));
    }

    // ----------------------------------------------------------------------
    // epilogue (warps 0-3): TMEM lane quadrant w = rows 32w .. 32w+31 =
    // (q = w/2, m = 4 (w%2) + lane/8, p = lane%8).  The lo half (warps 2, 3)
    // goes through shared memory (the stage buffers are idle by then).
    // ----------------------------------------------------------------------
    bool ok = true;
    if (warp < 4) ok = mbar_wait(smem_u32(&bar_done), 0);
    asm volatile("tcgen05.fence::after_thread_sync;");
    __syncthreads();
    ok = ok && !s_abort && n_live > 0;
    // [64 rows][257]: the odd row stride puts a warp's 32 rows (one column)
    // in 32 different banks
    constexpr int LOS = NN + 1;
    static_assert(64 * LOS * 4 <= NS * A_BYTES + STG_FLOATS * 2 * 4, "lo rows fit the idle stages");
    float *lo_buf = reinterpret_cast<float *>(smem);
    if (warp >= 2 && warp < 4 && ok) {
        const int row = (warp - 2) * 32 + lane;
        for (int cb = 0; cb < NN; cb += 32) {
            uint32_t r[32];
            const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                  "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                  "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                  "=r"(r[30]), "=r"(r[31])
                : "r"(addr));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 32; ++j) lo_buf[row * LOS + cb + j] = __uint_as_float(r[j]);
        }
    }
    __syncthreads();
    if (warp < 2) {
        const int row = warp * 32 + lane;           // (m, p) within the hi half
        const int m = row >> 3, p = row & 7;
        const int64_t ylen = J.y_len;
        float *ym = y + J.y_offset + (int64_t)(tl.mic0 + m) * ylen;
        float ss = 0.f, se = 0.f;
        for (int cb = 0; cb < NN; cb += 32) {
            uint32_t r[32];
            if (ok) {
                const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                    "%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,"
                    "%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                      "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                      "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
                      "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
                      "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(addr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = 0u;
            }
            if (m < nm) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t t = T0 + 8 * (cb + j) + p;
                    const float v = __uint_as_float(r[j]) + (ok ? lo_buf[row * LOS + cb + j] : 0.f);
                    if (t < ylen) {
                        ym[t] = v;
                        ff_accumulate_sq(v, ss, se);
                    }
                }
            }
        }
        // noise partial: the tile's sum of y^2 (float-float per row, FP64
        // across rows, fixed order)
        const double r = warp_sum_f64((double)ss + (double)se);
        if (lane == 0) s_red[warp] = r;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (part && tid == 0)
        part[J.part_offset + conv_partial_slot(tl.mic0, T0, J.y_len)] = s_red[0] + s_red[1];
    if (warp == 4) {
        __syncwarp();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
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
int g_smem_whole[64], g_smem_chunked[64];

}  // namespace

int launch_conv_bf16x3(const ConvLaunch &L, cudaStream_t stream) {
    // one launch per layout: tiles whose whole source window fits in shared
    // memory, and the rest (long RIRs) with per-chunk windows
    std::vector<Tile> tiles[2];
    int max_chunks = 0;
    for (int j = 0; j < L.n_jobs; ++j) {
        const ConvJob &J = L.jobs_host[j];
        const int n_chunks = (int)((J.rir_len + 7 + KC - 1) / KC);
        const bool whole = tc_layout(true, n_chunks).total <= 227 * 1024;
        if (whole) max_chunks = std::max(max_chunks, n_chunks);
        for (int m0 = 0; m0 < J.n_mics; m0 += MG)
            for (int64_t t0 = 0; t0 < J.y_len; t0 += TT) tiles[whole].push_back(Tile{j, m0, t0});
    }
    const size_t n_tiles = tiles[0].size() + tiles[1].size();
    if (n_tiles == 0) return ISM_OK;
    if (n_tiles > 0x7fffffffULL) return fail(ISM_ERR_INVALID_ARG, "too many tiles");
    void *d_tiles = nullptr;
    int st = scratch_alloc(&d_tiles, n_tiles * sizeof(Tile), stream);
    if (st) return st;
    std::vector<Tile> all(tiles[1]);
    all.insert(all.end(), tiles[0].begin(), tiles[0].end());
    st = upload_async(d_tiles, all.data(), n_tiles * sizeof(Tile), stream);
    if (st) { scratch_free(d_tiles, stream); return st; }
    cudaError_t e = cudaSuccess;
    if (!tiles[1].empty()) {
        const size_t smem = tc_layout(true, max_chunks).total;
        e = ensure_smem(k_conv_tc<true>, g_smem_whole, g_smem_mu, smem);
        if (e == cudaSuccess)
            k_conv_tc<true><<<(unsigned)tiles[1].size(), NTHR, smem, stream>>>(
                L.jobs_dev, (const Tile *)d_tiles, L.h_dev, L.src_dev, L.y_dev,
                L.noise_partials_dev);
    }
    if (e == cudaSuccess && !tiles[0].empty()) {
        const size_t smem = tc_layout(false, 0).total;
        e = ensure_smem(k_conv_tc<false>, g_smem_chunked, g_smem_mu, smem);
        if (e == cudaSuccess)
            k_conv_tc<false><<<(unsigned)tiles[0].size(), NTHR, smem, stream>>>(
                L.jobs_dev, (const Tile *)d_tiles + tiles[1].size(), L.h_dev, L.src_dev, L.y_dev,
                L.noise_partials_dev);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    scratch_free(d_tiles, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch k_conv_tc");
    return ISM_OK;
}

}  // namespace ism
