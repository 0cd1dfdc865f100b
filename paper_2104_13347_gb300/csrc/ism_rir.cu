// ism_rir.cu -- K1: image-source room impulse responses on sm_103a.
//
// Computes, for every (room, microphone) RIR, the sum over the image lattice
// of arXiv 2104.13347, Sec. II.A: each image (u,v,w,l,m,n) at distance d
// contributes a fractional-delay tap group at tau = d fs / c with gain
// prod(beta^hits) / (4 pi d).
//
// Work decomposition (GB300-first, no global atomics on h):
//  * A work item is one output window [w0, w0+W) of one RIR.  A persistent
//    grid pulls items from one atomic counter, later windows (more images)
//    first.
//  * The CTA enumerates only the images whose taps reach its window: per
//    lattice column (u,l,v,m,w) the admissible n are the integers with
//    zmin <= |Delta_z(n)| <= zmax, solved in FP32 with a safety margin; each
//    candidate is then tested exactly on its delay.
//  * Delays: image-to-mic squared offsets per axis are tabled in FP64 with
//    the definition's rounding (once per RIR by k_ism_tables for the sparse
//    kernel, once per item for the direct one), d^2 and sqrt are done in
//    float-float (FP32 pipe; GB300's FP64 rate is a small fraction of FP32),
//    and the integer split is redone in FP64 with the definition's exact
//    operation order whenever the float-float delay lies within 1e-6 samples
//    of a rounding boundary or of an integer (so exact integer delays give
//    exact Kronecker deltas).  The integer part therefore equals the
//    definition's bit for bit, and the fractional part to ~1e-9 samples.
//
// Two ways to lay the taps down:
//  * k_ism_sparse (default): the tap function of the filter, g_j(f), is
//    expanded in Chebyshev polynomials of the fraction, g_j(f) ~ sum_p
//    B[p][j] T_p(x(f)) (FP64 table, truncated where the remaining terms sum
//    below 1e-6 of the peak tap for the Hann sinc -- 8 terms for 81 taps --
//    and exact for the 8-tap Lagrange filter, whose taps are degree-7
//    polynomials in the delay).  Each image then adds a T_p(x) to P sparse integer-delay
//    arrays c_p[kb] -- the paper's representation of the integer delays as a
//    sparse array -- held in 32-bit fixed point (native u32 shared-memory
//    atomics, order-independent sums: bitwise reproducible), and one FIR per
//    window gives h[n] = sum_p sum_j B[p][j] c_p[n - j].  Per image: P
//    terms instead of one reciprocal and ~7 operations per tap.  The
//    lattice columns of each RIR are sorted once by rho^2 = x^2 + y^2
//    (k_ism_tables); a window sweeps the contiguous range of that order
//    that can reach it, one column per lane, each lane walking its own
//    column's candidates (neighbouring columns have nearly equal counts).
//  * k_ism_taps (direct): one warp per image, one lane per tap (81 taps -> 3
//    rows of 32).  sin(pi (j-f)) = -(-1)^j sin(pi f), and the Hann window,
//    written cos^2(pi (j-f) / (2(H+1))), is expanded in cos/sin of
//    pi j/(2(H+1)) (per-lane constants) and of pi f/(2(H+1)) (per image),
//    leaving one reciprocal per tap.  Each warp
//    accumulates into its own shared-memory copy of the window (no atomics,
//    fixed order, bitwise reproducible).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>

#include "ism_internal.h"

namespace ism {
namespace {

constexpr int NT = 256;           // threads per CTA
constexpr int NW = NT / 32;       // warps per CTA
constexpr int CAP = 2048;         // candidate buffer (images)
constexpr float kEps = 0.2f;      // metres of margin in the column solve
constexpr int PADL = 8;           // left padding of the sparse arrays (floats)

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exclusive block-wide scan of v over NT threads; total returned by ref.
__device__ __forceinline__ int block_scan(int v, int *s_w, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = lane < NW ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NW) s_w[lane] = t;
    }
    __syncthreads();
    int off = (warp ? s_w[warp - 1] : 0) + x - v;
    total = s_w[NW - 1];
    __syncthreads();
    return off;
}

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int round64(int x) { return (x + 63) & ~63; }

// Storage order of the sparse arrays: word x is kept at x ^ (bit 5 of x ->
// bit 2), i.e. the 16-byte groups of every odd 32-word line are swapped in
// pairs.  The FIR reads 128-bit words at a stride of 8 words per lane, which
// in plain order hits only 4 of the 8 16-byte bank groups per 8-lane phase
// (2-way conflicts); swizzled, any 8 consecutive lanes cover all 8, for every
// alignment.  The map permutes each 32-word line in place, keeps 16-byte
// groups whole and, with the row length a multiple of 64 words, commutes
// with the row offsets.
__device__ __forceinline__ int swz(int x) { return x ^ ((x >> 3) & 4); }

struct Tables {
    const double *sq;  // [3][TE] squared axis offsets (FP64, definition rounding)
    float4 *hlg;  // [3][TE] (hi, lo, g, -): float-float split of sq and the
                  // wall damping product along the axis, one 128-bit load
    float *dl;    // [3][TE] axis offset, FP32
};

// Shared-memory carve-up.  Common part: the per-axis tables.  The direct
// kernel adds the axis lists, the candidate buffer and one private window
// row per warp; the sparse kernel the FIR partial sums (in the candidate
// slot), the P sparse arrays and the integer-delay (delta) array.
struct Layout {
    int TE, RL, CL;
    size_t off_sq, off_hlg, off_dl, off_lx, off_ly, off_cand, off_rows, off_c,
        off_delta, off_part, total;
};

__host__ __device__ inline Layout make_layout(bool sparse, int window, int max_order,
                                              int max_taps, int max_cheb) {
    Layout L;
    L.TE = 2 * (2 * max_order + 1);
    L.RL = round4(window + 2 * (max_taps - 1));
    L.CL = sparse ? round64(window + max_taps + 12 + PADL) : round4(window + max_taps + 12 + PADL);
    size_t o = 0;
    // the sparse kernel reads the FP64 squares (exact path only) from the
    // per-RIR tables in global memory
    L.off_sq = o;   o = align16(o + (sparse ? 0 : sizeof(double) * 3 * L.TE));
    L.off_hlg = o;  o = align16(o + sizeof(float4) * 3 * L.TE);
    L.off_dl = o;   o = align16(o + sizeof(float) * 3 * L.TE);
    // axis lists and the candidate buffer: direct kernel only; the sparse
    // kernel keeps the FIR partial sums (W floats) in the candidate slot
    L.off_lx = o;   o = align16(o + (sparse ? 0 : sizeof(int) * L.TE));
    L.off_ly = o;   o = align16(o + (sparse ? 0 : sizeof(int) * L.TE));
    const size_t cand_words = sparse ? (size_t)window : (size_t)CAP;
    L.off_cand = o; o = align16(o + sizeof(uint32_t) * cand_words);
    L.off_rows = L.off_c = L.off_delta = o;
    L.off_part = L.off_cand;
    if (!sparse) {
        L.off_rows = o; o = align16(o + sizeof(float) * (size_t)NW * L.RL);
    } else {
        L.off_c = o;     o = align16(o + sizeof(float) * (size_t)max_cheb * L.CL);
        L.off_delta = o; o = align16(o + sizeof(float) * (size_t)L.CL);
    }
    L.total = o;
    return L;
}

// Float-float sum (ah + al) + (bh + bl): two-sum of the high parts, the
// low parts added to the error, renormalised.
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float &sh,
                                       float &sl) {
    const float s = __fadd_rn(ah, bh);
    const float bb = __fsub_rn(s, ah);
    float e = __fadd_rn(__fsub_rn(ah, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    e = __fadd_rn(e, __fadd_rn(al, bl));
    sh = __fadd_rn(s, e);
    sl = __fsub_rn(e, __fsub_rn(sh, s));
}

// Delay split of one image (Sec. II.A: the delay of every image must keep
// its sub-sample precision) from tau^2 = Th + Tl in float-float (the tables
// hold the axis offsets in samples, q = fs / c folded in).  Returns the
// integer part k (rint, ties to even, for Hann; floor for Lagrange) and the
// fraction in FP32, plus tau.  sqx, sqy, sqz: the FP64 squared axis offsets
// in metres, read only on the exact path.
template <int KIND>
__device__ __forceinline__ void split_tau2(float Th, float Tl, const double *sqx,
                                           const double *sqy, const double *sqz, double q,
                                           int &k_out, float &f_out, float &tau_out) {
    // sqrt: FP32 estimate plus one Newton correction in float-float.
    const float r = rsqrtf(Th);
    const float s0 = __fmul_rn(Th, r);
    const float res = __fadd_rn(__fmaf_rn(-s0, s0, Th), Tl);
    float th = s0;
    float tl = __fmul_rn(res, __fmul_rn(0.5f, r));
    const float tt = __fadd_rn(th, tl);
    tl = __fsub_rn(tl, __fsub_rn(tt, th));
    th = tt;
    // The low part can carry f just past the rounding boundary (|tl| is at
    // most half an ulp of th); every such f lies within 1e-6 of it and takes
    // the exact path below, so no correction is made here.
    float k, f;
    bool near;
    if (KIND == ISM_FD_HANN_SINC) {
        k = rintf(th);
        f = __fadd_rn(__fsub_rn(th, k), tl);
        near = fabsf(f) > 0.5f - 1e-6f || fabsf(f) < 1e-6f;  // ties and integers
    } else {
        k = floorf(th);
        f = __fadd_rn(__fsub_rn(th, k), tl);
        near = f < 1e-6f || f > 1.f - 1e-6f;
    }
    if (near) {
        // Exact path: the definition's FP64 operations in its order.
        const double d2 = __dadd_rn(__dadd_rn(*sqx, *sqy), *sqz);
        const double d = __dsqrt_rn(d2);
        const double tau = __dmul_rn(d, q);
        const double kd = (KIND == ISM_FD_HANN_SINC) ? rint(tau) : floor(tau);
        k = (float)kd;
        f = (float)(tau - kd);
    }
    k_out = (int)k;
    f_out = f;
    tau_out = th;
}

// Delay split of image (ix, iy, iz) from the tables; also returns the wall
// damping product g.
template <int KIND>
__device__ __forceinline__ void delay_split(const Tables &T, int TE, int ix, int iy, int iz,
                                            double q, int &k_out, float &f_out, float &tau_out,
                                            float &g_out) {
    const float4 X = T.hlg[ix], Y = T.hlg[TE + iy], Z = T.hlg[2 * TE + iz];
    g_out = X.z * Y.z * Z.z;
    float s1, e1, Th, Tl;
    ff_add(X.x, X.y, Y.x, Y.y, s1, e1);
    ff_add(s1, e1, Z.x, Z.y, Th, Tl);
    split_tau2<KIND>(Th, Tl, &T.sq[ix], &T.sq[TE + iy], &T.sq[2 * TE + iz], q, k_out, f_out,
                     tau_out);
}

// Per-item constants (identical in every thread of the CTA).
struct Item {
    int N, TEj, n_taps, H, P;   // order, table entries, taps, Hann half-width, Lagrange order
    int w0, W;
    long long Lh, kb_lo, kb_hi; // window's first-tap range
    int kb_lo32, kb_hi32, Lh32, wend;  // 32-bit copies; wend = min(w0 + W, Lh)
    double q;
    float qh, ql, dlo2, dhi2, dhe2, dhe, eps, inv2Lz;
};

// Per-RIR FP32 constants of the sparse kernel's window setup (computed once
// in FP64, so that no window needs the FP64 pipe for them).
struct JobConst {
    float d_dir;   // |source - mic|: no image is closer (points inside the box)
    float inv_q;   // c / fs, metres per sample
    float qh, ql;  // fs / c split into two floats
    float inv2Lz;  // 1 / (2 Lz)
    float pad[3];
};

template <int KIND>
__device__ __forceinline__ void item_setup(const RirJob &J, int W, int wi, Item &it) {
    it.N = J.order;
    it.TEj = 2 * (2 * it.N + 1);
    it.n_taps = J.n_taps;
    it.H = (it.n_taps - 1) / 2;
    it.P = it.n_taps - 1;
    it.Lh = J.rir_len;
    it.W = W;
    it.w0 = wi * W;
    it.q = J.q;
    it.qh = (float)it.q;
    it.ql = (float)(it.q - (double)it.qh);
    it.kb_lo = (long long)it.w0 - it.n_taps + 1;
    it.kb_hi = min((long long)it.w0 + W - 1, it.Lh - 1);
    it.kb_lo32 = (int)it.kb_lo;
    it.kb_hi32 = (int)it.kb_hi;
    it.Lh32 = (int)it.Lh;
    it.wend = (int)min((long long)it.w0 + W, it.Lh);
    double tau_lo, tau_hi;
    if (KIND == ISM_FD_HANN_SINC) {
        tau_lo = (double)(it.kb_lo + it.H) - 0.5;
        tau_hi = (double)(it.kb_hi + it.H) + 0.5;
    } else {
        tau_lo = (double)(it.kb_lo + (it.P - 1) / 2);
        tau_hi = (double)(it.kb_hi + (it.P + 1) / 2);
    }
    const float d_lo = (float)fmax(tau_lo / it.q, 0.0);
    const float d_hi = (float)(tau_hi / it.q);
    it.eps = kEps + 1e-6f * d_hi;
    it.dlo2 = d_lo * d_lo;
    it.dhi2 = d_hi * d_hi;
    it.dhe = d_hi + it.eps;
    it.dhe2 = it.dhe * it.dhe;
    it.inv2Lz = 1.f / (2.f * (float)J.dims[2]);
}

// One per-axis table entry: axis a, entry ei = p (2N+1) + (qq + N) of a
// job.  Offset in FP64 with the definition's rounding,
// ((1-2p) s + (2q) L) - r, its square (FP64, and split into two floats),
// and the wall damping product along the axis.
__device__ __forceinline__ void table_entry(const RirJob &J, int N, int a, int ei, double &sq,
                                            float4 &hlg, float &dl) {
    const int p = ei / (2 * N + 1), qq = ei - p * (2 * N + 1) - N;
    const double s = J.src[a], Ld = J.dims[a], r = J.mic[a];
    const double img = __dadd_rn(p ? -s : s, __dmul_rn((double)(2 * qq), Ld));
    const double dlt = __dsub_rn(img, r);
    sq = __dmul_rn(dlt, dlt);
    // float-float square of the offset in samples: (q dlt)^2, q = fs / c
    const double t2 = sq * (J.q * J.q);
    const float sh = __double2float_rn(t2);
    dl = __double2float_rn(dlt);
    const float b0 = J.beta[2 * a], b1 = J.beta[2 * a + 1];
    hlg = make_float4(sh, __double2float_rn(t2 - (double)sh),
                      powf(b0, (float)abs(qq - p)) * powf(b1, (float)abs(qq)), 0.f);
}

// The sparse kernel's per-window constants in FP32 from the per-RIR
// constants: the same fields as item_setup (bounds in metres carry the
// column solve's 0.2 m margin, far above FP32 rounding).
template <int KIND>
__device__ __forceinline__ void item_setup_f32(const RirJob &J, const JobConst &jc, int W, int wi,
                                               Item &it, float &tau_lo, float &tau_hi) {
    it.N = J.order;
    it.TEj = 2 * (2 * it.N + 1);
    it.n_taps = J.n_taps;
    it.H = (it.n_taps - 1) / 2;
    it.P = it.n_taps - 1;
    it.Lh = J.rir_len;
    it.W = W;
    it.w0 = wi * W;
    it.q = J.q;
    it.qh = jc.qh;
    it.ql = jc.ql;
    it.kb_lo = (long long)it.w0 - it.n_taps + 1;
    it.kb_hi = min((long long)it.w0 + W - 1, it.Lh - 1);
    it.kb_lo32 = (int)it.kb_lo;
    it.kb_hi32 = (int)it.kb_hi;
    it.Lh32 = (int)it.Lh;
    it.wend = (int)min((long long)it.w0 + W, it.Lh);
    if (KIND == ISM_FD_HANN_SINC) {
        tau_lo = (float)(it.kb_lo32 + it.H) - 0.5f;
        tau_hi = (float)(it.kb_hi32 + it.H) + 0.5f;
    } else {
        tau_lo = (float)(it.kb_lo32 + (it.P - 1) / 2);
        tau_hi = (float)(it.kb_hi32 + (it.P + 1) / 2);
    }
    const float d_lo = fmaxf(tau_lo * jc.inv_q, 0.f);
    const float d_hi = tau_hi * jc.inv_q;
    it.eps = kEps + 1e-6f * d_hi;
    it.dlo2 = d_lo * d_lo;
    it.dhi2 = d_hi * d_hi;
    it.dhe = d_hi + it.eps;
    it.dhe2 = it.dhe * it.dhe;
    it.inv2Lz = jc.inv2Lz;
}

// Per-axis tables of one job (all NT threads of the direct kernel).
__device__ __forceinline__ void build_tables(const RirJob &J, const Tables &T, double *sq_out,
                                             int TE, const Item &it) {
    const int N = it.N, TEj = it.TEj;
    for (int e = threadIdx.x; e < 3 * TEj; e += NT) {
        const int a = e / TEj, ei = e - a * TEj;
        double sq;
        float4 hlg;
        float dl;
        table_entry(J, N, a, ei, sq, hlg, dl);
        sq_out[a * TE + ei] = sq;
        T.dl[a * TE + ei] = dl;
        T.hlg[a * TE + ei] = hlg;
    }
}

// Per-RIR tables in global memory for the sparse kernel, computed once per
// RIR instead of once per window (GB300's FP64 pipe is narrow): RIR j's
// entry (a, ei) at j * 3 TE + a TE + ei.
//
// The same kernel sorts the RIR's lattice columns (x entry, y entry) by
// rho^2 = x^2 + y^2 for the sparse kernel's sweep: a counting sort into KB
// bins of equal width over [0, R^2], R the largest distance any window of
// the RIR reaches (columns beyond it hold no image of any window), written
// to g_cols + offs[2 j] as ix | iy << 16.  For every window w it records in
// g_wr[offs[2 j + 1] + w] the rank range [c_lo, c_hi) of the bins that can
// hold a column with candidates in w: columns closer than
// rho^2 = d_lo^2 - (Z + eps)^2 (Z: the largest |z offset| of the lattice)
// have every image nearer than the window, columns farther than d_hi + eps
// none that near; one bin of margin on either side.  The order inside a bin
// is whatever the atomics give: it changes only how the sweep's lanes are
// loaded, never which images are summed (and the sums are exact integers).
constexpr int KB = 2048;          // rho^2 bins of the column sort
constexpr int TNT = 256;          // threads of k_ism_tables
constexpr int kMaxTE = 2 * (2 * 200 + 1);

// rho^2 of a column and its bin, with explicit roundings: the histogram and
// the scatter must place every column in the same bin.
__device__ __forceinline__ float col_rho2(float x, float y) {
    return __fmaf_rn(x, x, __fmul_rn(y, y));
}
__device__ __forceinline__ int rho2_bin(float r2, float sc) {
    return (int)fminf(__fmul_rn(r2, sc), (float)(KB - 1));
}

template <int KIND>
__global__ void __launch_bounds__(TNT)
k_ism_tables(const RirJob *__restrict__ jobs, int n_rirs, int TE, int W,
             double *__restrict__ g_sq, float4 *__restrict__ g_hlg, float *__restrict__ g_dl,
             JobConst *__restrict__ g_jc, uint32_t *__restrict__ g_cols, int2 *__restrict__ g_wr,
             const long long *__restrict__ g_offs) {
    __shared__ float s_x[kMaxTE], s_y[kMaxTE];
    __shared__ unsigned s_bin[KB + 1];
    __shared__ unsigned s_zmax;  // float bits of max |z offset| (>= 0)
    __shared__ JobConst s_jc;
    __shared__ unsigned s_wsum[TNT / 32];
    const int tid = threadIdx.x;
    for (int j = blockIdx.x; j < n_rirs; j += gridDim.x) {
        const RirJob &J = jobs[j];
        const int N = J.order, TEj = 2 * (2 * N + 1);
        const size_t base = (size_t)j * 3 * TE;
        if (tid == 0) {
            const double dx = J.src[0] - J.mic[0], dy = J.src[1] - J.mic[1],
                         dz = J.src[2] - J.mic[2];
            JobConst c;
            c.d_dir = (float)sqrt(dx * dx + dy * dy + dz * dz);
            c.inv_q = (float)(1.0 / J.q);
            c.qh = (float)J.q;
            c.ql = (float)(J.q - (double)c.qh);
            c.inv2Lz = (float)(0.5 / J.dims[2]);
            c.pad[0] = c.pad[1] = c.pad[2] = 0.f;
            g_jc[j] = c;
            s_jc = c;
            s_zmax = 0u;
        }
        for (int i = tid; i <= KB; i += TNT) s_bin[i] = 0u;
        __syncthreads();
        for (int e = tid; e < 3 * TEj; e += TNT) {
            const int a = e / TEj, ei = e - a * TEj;
            double sq;
            float4 hlg;
            float dl;
            table_entry(J, N, a, ei, sq, hlg, dl);
            g_sq[base + a * TE + ei] = sq;
            g_hlg[base + a * TE + ei] = hlg;
            g_dl[base + a * TE + ei] = dl;
            if (a == 0) s_x[ei] = dl;
            else if (a == 1) s_y[ei] = dl;
            else atomicMax(&s_zmax, __float_as_uint(fabsf(dl)));
        }
        __syncthreads();
        const JobConst jc = s_jc;
        Item it;
        float tau_lo, tau_hi;
        item_setup_f32<KIND>(J, jc, W, J.n_windows - 1, it, tau_lo, tau_hi);
        const float R2 = fmaxf(it.dhe2, 1e-30f);
        const float sc = (float)KB / R2;
        const int n_cols = TEj * TEj;
        // histogram of the columns within R
        for (int c = tid; c < n_cols; c += TNT) {
            const int ix = c / TEj, iy = c - ix * TEj;
            const float r2 = col_rho2(s_x[ix], s_y[iy]);
            if (r2 <= R2) atomicAdd(&s_bin[rho2_bin(r2, sc)], 1u);
        }
        __syncthreads();
        // exclusive scan of the KB bins: each thread scans KB / TNT
        // consecutive bins, the warps' totals go through shared memory
        {
            constexpr int PER = KB / TNT;
            unsigned loc[PER], run = 0u;
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                loc[k] = run;
                run += s_bin[tid * PER + k];
            }
            const int lane = tid & 31, warp = tid >> 5;
            unsigned x = run;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            unsigned off = x - run;
            for (int w = 0; w < warp; ++w) off += s_wsum[w];
#pragma unroll
            for (int k = 0; k < PER; ++k) s_bin[tid * PER + k] = off + loc[k];
            if (tid == TNT - 1) s_bin[KB] = off + run;
        }
        __syncthreads();
        // per-window rank ranges
        const float zr = __uint_as_float(s_zmax);
        for (int w = tid; w < J.n_windows; w += TNT) {
            Item iw;
            float tl, th;
            item_setup_f32<KIND>(J, jc, W, w, iw, tl, th);
            const float zz = zr + iw.eps;
            const float r2lo = fmaxf(iw.dlo2 - zz * zz, 0.f);
            const int b_lo = max(rho2_bin(r2lo, sc) - 1, 0);
            const int b_hi = min(rho2_bin(iw.dhe2, sc) + 1, KB - 1);
            g_wr[g_offs[2 * j + 1] + w] = make_int2((int)s_bin[b_lo], (int)s_bin[b_hi + 1]);
        }
        __syncthreads();
        // scatter (the bin starts become cursors)
        uint32_t *out = g_cols + g_offs[2 * j];
        for (int c = tid; c < n_cols; c += TNT) {
            const int ix = c / TEj, iy = c - ix * TEj;
            const float r2 = col_rho2(s_x[ix], s_y[iy]);
            if (r2 <= R2) {
                const unsigned pos = atomicAdd(&s_bin[rho2_bin(r2, sc)], 1u);
                if (ISM_IN_RANGE(pos < (unsigned)n_cols, kOobColumnSlot))
                    out[pos] = (uint32_t)ix | ((uint32_t)iy << 16);
            }
        }
        __syncthreads();
    }
}

// Axis lists (warps 0 and 1): table entries whose offset alone is in reach.
__device__ __forceinline__ void build_lists(const Tables &T, int TE, const Item &it, int *s_lx,
                                            int *s_ly, int *s_nl) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 2) {
        const float *dd = T.dl + warp * TE;
        int *lst = warp ? s_ly : s_lx;
        int cnt = 0;
        for (int base = 0; base < it.TEj; base += 32) {
            const int e = base + lane;
            const bool ok = e < it.TEj && fabsf(dd[e]) <= it.dhe;
            const unsigned b = __ballot_sync(0xffffffffu, ok);
            if (ok) lst[cnt + __popc(b & ((1u << lane) - 1u))] = e;
            cnt += __popc(b);
        }
        if (lane == 0) s_nl[warp] = cnt;
    }
}

// Column solve: for column c = ((u,l), (v,m), w) of the axis lists, the
// admissible n (|Delta_z(n)| in [zmin, zmax]) as up to two intervals
// [lo_a, hi_a], [lo_b, hi_b]; empty intervals have lo > hi.
struct Col {
    int lo_a, hi_a, lo_b, hi_b, ix, iy, wz;
    __device__ __forceinline__ int count() const {
        return max(hi_a - lo_a + 1, 0) + max(hi_b - lo_b + 1, 0);
    }
};

// sqrt(x) for x >= 0 from the approximate reciprocal square root (2 ulp);
// the column bounds carry a margin of eps >= 0.2 m, far above its error.
__device__ __forceinline__ float sqrt_bound(float x) {
    return x * rsqrtf(fmaxf(x, 1e-30f));
}

// The admissible n of column (ix, iy, wz): the z runs whose image distance
// can fall in the item's delay range [d_lo, d_hi] (widened by eps).
__device__ __forceinline__ Col column_solve_xy(const Tables &T, int TE, const Item &it, int ix,
                                               int iy, int wz) {
    const int N = it.N;
    Col r{1, 0, 1, 0, ix, iy, wz};
    const float dx = T.dl[ix], dy = T.dl[TE + iy];
    const float rho2 = dx * dx + dy * dy;
    if (rho2 > it.dhe2) return r;
    // Delta_z(n) = cz + 2 Lz n must satisfy zmin <= |Delta_z| <= zmax:
    // the full range [-zmax, zmax] minus the open hole (-zmin, zmin).
    const float zmax = sqrt_bound(fmaxf(it.dhi2 - rho2, 0.f)) + it.eps;
    const float zmin2 = it.dlo2 - rho2;
    const float zmin = zmin2 > 0.f ? sqrt_bound(zmin2) - it.eps : 0.f;
    const float cz = T.dl[2 * TE + wz * (2 * N + 1) + N];
    const float lim = (float)N + 1.f;
    const float u_lo = fminf(fmaxf((-zmax - cz) * it.inv2Lz, -lim), lim);
    const float u_hi = fminf(fmaxf((zmax - cz) * it.inv2Lz, -lim), lim);
    int n_lo = (int)ceilf(u_lo);
    int n_hi = (int)floorf(u_hi);
    if (n_lo < -N) n_lo = -N;
    if (n_hi > N) n_hi = N;
    int h_lo = 1, h_hi = 0;  // hole (excluded n), empty by default
    if (zmin > 0.f) {
        const float v_lo = fminf(fmaxf((-zmin - cz) * it.inv2Lz, -lim), lim);
        const float v_hi = fminf(fmaxf((zmin - cz) * it.inv2Lz, -lim), lim);
        h_lo = (int)floorf(v_lo) + 1;
        h_hi = (int)ceilf(v_hi) - 1;
    }
    if (h_lo <= h_hi) {
        r.lo_a = n_lo;
        r.hi_a = n_hi < h_lo - 1 ? n_hi : h_lo - 1;
        r.lo_b = n_lo > h_hi + 1 ? n_lo : h_hi + 1;
        r.hi_b = n_hi;
    } else {
        r.lo_a = n_lo;
        r.hi_a = n_hi;
    }
    return r;
}

// Column c = ((u,l), (v,m), w) of the axis lists (direct kernel's sweep).
// rnly: an FP32 reciprocal of nLY (any rounding: the quotient is corrected).
__device__ __forceinline__ Col column_solve(const Tables &T, int TE, const Item &it,
                                            const int *s_lx, const int *s_ly, int nLY,
                                            float rnly, int c, int n_cols) {
    if (c >= n_cols) return Col{1, 0, 1, 0, 0, 0, 0};
    // (x, y) list positions of column pair t = c / 2 (t < 2^20): quotient
    // by an FP32 reciprocal, corrected to the exact integer division
    const int t = c >> 1;
    int xi = (int)((float)t * rnly);
    int yi = t - xi * nLY;
    if (yi < 0) { --xi; yi += nLY; }
    else if (yi >= nLY) { ++xi; yi -= nLY; }
    return column_solve_xy(T, TE, it, s_lx[xi], s_ly[yi], c & 1);
}

// Writes the candidates of column col whose warp- or block-level index
// (first index off) lies in [g_lo, g_hi), candidate index i going to
// dst[(base + i) & mask].
__device__ __forceinline__ void column_emit(const Col &col, int N, int off, int g_lo, int g_hi,
                                            uint32_t *dst, int base, int mask) {
    const int zb = col.wz * (2 * N + 1) + N;
    const uint32_t code = (uint32_t)col.ix | ((uint32_t)col.iy << 10);
    int gi = off;
    for (int n = col.lo_a; n <= col.hi_a; ++n, ++gi)
        if (gi >= g_lo && gi < g_hi) dst[(base + gi) & mask] = code | ((uint32_t)(zb + n) << 20);
    for (int n = col.lo_b; n <= col.hi_b; ++n, ++gi)
        if (gi >= g_lo && gi < g_hi) dst[(base + gi) & mask] = code | ((uint32_t)(zb + n) << 20);
}

// Column sweep: candidates per (u,l,v,m,w) column, handed to flush(nc) in
// batches of at most CAP.  All threads call it; block-uniform control flow.
template <class Flush>
__device__ __forceinline__ void column_sweep(const Tables &T, int TE, const Item &it,
                                             const int *s_lx, const int *s_ly, int nLX, int nLY,
                                             int *s_scan, uint32_t *s_cand, Flush &flush) {
    const int N = it.N, tid = threadIdx.x;
    const int n_cols = nLX * nLY * 2;
    const float rnly = __frcp_rn((float)nLY);
    int n_cand = 0;  // block-uniform
    for (int cb = 0; cb < n_cols; cb += NT) {
        const int c = cb + tid;
        const Col col = column_solve(T, TE, it, s_lx, s_ly, nLY, rnly, c, n_cols);
        int total;
        const int off = block_scan(col.count(), s_scan, total);
        if (total == 0) continue;
        if (n_cand + total > CAP && n_cand > 0) {
            flush(n_cand);
            n_cand = 0;
        }
        if (total <= CAP) {
            column_emit(col, N, off, 0, total, s_cand, n_cand, 0x7fffffff);
            n_cand += total;
        } else {
            for (int pb = 0; pb < total; pb += CAP) {
                column_emit(col, N, off, pb, pb + CAP, s_cand, -pb, 0x7fffffff);
                flush(min(CAP, total - pb));
            }
        }
    }
    if (n_cand > 0) flush(n_cand);
}

// Sorted column sweep of the sparse kernel.  The item's columns are the
// ranks [c_lo, c_hi) of the RIR's column list, sorted by rho^2 = x^2 + y^2
// (k_ism_tables), each (x, y) entry standing for two columns (z parity
// w = 0, 1).  Warp w takes column batches w, w + NW, ... of 32 columns, one
// per lane; each lane solves its column and walks the column's candidates
// itself.  Neighbouring ranks have nearly the same rho and hence nearly the
// same candidate count, so the lanes of a batch finish close together.
// proc(rho_h, rho_l, g_xy, iz, ix, iy) is called once per candidate (iz:
// absolute index of the z table entry; ix, iy: the column's entries).  No
// block-wide barrier is involved.
template <class Proc>
__device__ __forceinline__ void sorted_sweep(const Tables &T, int TE, const Item &it,
                                             const uint32_t *__restrict__ cols, int c_lo,
                                             int c_hi, Proc &proc) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_cols = 2 * (c_hi - c_lo);
    const int N = it.N;
    for (int cb = warp * 32; cb < n_cols; cb += NT) {
        const int c = cb + lane;
        int na = 0, nb = 0, iz_a = 0, iz_b = 0, ix = 0, iy = 0;
        float Rh = 0.f, Rl = 0.f, gxy = 0.f;
        if (c < n_cols) {
            const uint32_t e = __ldg(cols + c_lo + (c >> 1));
            ix = (int)(e & 0xffffu);
            iy = (int)(e >> 16);
            // (entries are < TEj by construction; the guard keeps a bad
            // entry from indexing past the tables)
            const bool ok_e = ISM_IN_RANGE(ix < it.TEj && iy < it.TEj, kOobColumnEntry);
            const Col col = ok_e ? column_solve_xy(T, TE, it, ix, iy, c & 1)
                                 : Col{1, 0, 1, 0, 0, 0, 0};
            na = max(col.hi_a - col.lo_a + 1, 0);
            nb = max(col.hi_b - col.lo_b + 1, 0);
            if (na + nb > 0) {
                const float4 X = T.hlg[ix], Y = T.hlg[TE + iy];
                ff_add(X.x, X.y, Y.x, Y.y, Rh, Rl);
                gxy = X.z * Y.z;
                // candidate i is z entry iz_a + i (i < na) or iz_b + i
                const int iz0 = 2 * TE + col.wz * (2 * N + 1) + N;
                iz_a = iz0 + col.lo_a;
                iz_b = iz0 + col.lo_b - na;
            }
        }
        const int cnt = na + nb;
        for (int i = 0; i < cnt; ++i) proc(Rh, Rl, gxy, (i < na ? iz_a : iz_b) + i, ix, iy);
    }
}

// Evaluates one candidate: delay split, window test, gain, statistics.
// Returns false if the image's taps miss the window.
template <int KIND>
__device__ __forceinline__ bool eval_candidate(const Tables &T, int TE, const Item &it,
                                               uint32_t cd, int &kb, float &f, float &a,
                                               unsigned long long &my_taps,
                                               unsigned long long &my_contrib) {
    const int ix = cd & 1023, iy = (cd >> 10) & 1023, iz = cd >> 20;
    int k;
    float tau, g;
    delay_split<KIND>(T, TE, ix, iy, iz, it.q, k, f, tau, g);
    kb = (KIND == ISM_FD_HANN_SINC) ? k - it.H : k - (it.P - 1) / 2;
    if (kb < it.kb_lo32 || kb > it.kb_hi32) return false;
    // g / (4 pi d) = g q / (4 pi tau)
    a = g * (it.qh * __frcp_rn(12.566370614359172f * tau));
    // statistics: taps in [w0, w0+W) n [0, Lh); an image counts as
    // contributing in the window of its first in-range tap.  All indices
    // here fit in 32 bits (Lh <= 2^30).
    const int lo = max(kb, max(it.w0, 0));
    const int hi = min(kb + it.n_taps, it.wend);
    if (hi > lo) my_taps += (unsigned)(hi - lo);
    const int first = max(kb, 0);
    if (first < min(kb + it.n_taps, it.Lh32) && first >= it.w0 && first < it.w0 + it.W)
        ++my_contrib;
    return true;
}

// Evaluates one column-expanded candidate: delay split from the column's
// (q rho)^2 (Rh + Rl) and the z table entry iz (absolute index), window
// test, gain, statistics.  ix, iy: the column's x and y entries (exact path
// only).  Returns false if the image's taps miss the window.
// a is returned as g / tau: the caller folds q / (4 pi) into its scale.
template <int KIND, bool STATS>
__device__ __forceinline__ bool eval_expanded(const Tables &T, int TE, const Item &it, float Rh,
                                              float Rl, float gxy, int iz, int ix, int iy, int &kb,
                                              float &f, float &a, unsigned &my_taps,
                                              unsigned &my_contrib) {
    if (!ISM_IN_RANGE(iz >= 2 * TE && iz < 2 * TE + it.TEj, kOobTableIndex)) return false;
    const float4 Z = T.hlg[iz];
    float Th, Tl;
    ff_add(Rh, Rl, Z.x, Z.y, Th, Tl);
    int k;
    float tau;
    split_tau2<KIND>(Th, Tl, &T.sq[ix], &T.sq[TE + iy], &T.sq[iz], it.q, k, f, tau);
    kb = (KIND == ISM_FD_HANN_SINC) ? k - it.H : k - (it.P - 1) / 2;
    // kb in [kb_lo, kb_hi], one unsigned comparison
    if ((unsigned)(kb - it.kb_lo32) > (unsigned)(it.kb_hi32 - it.kb_lo32)) return false;
    // approximate reciprocal (about 1 ulp, below the FP32 accumulation)
    a = (gxy * Z.z) * rcp_approx(tau);
    if (STATS) {
        const int lo = max(kb, max(it.w0, 0));
        const int hi = min(kb + it.n_taps, it.wend);
        if (hi > lo) my_taps += (unsigned)(hi - lo);
        const int first = max(kb, 0);
        if (first < min(kb + it.n_taps, it.Lh32) && first >= it.w0 && first < it.w0 + it.W)
            ++my_contrib;
    }
    return true;
}

__device__ __forceinline__ void flush_stats(long long *stats, const RirJob &J,
                                            unsigned long long *s_stat,
                                            unsigned long long my_contrib,
                                            unsigned long long my_taps) {
    if (!stats) return;
    atomicAdd(&s_stat[0], my_contrib);
    atomicAdd(&s_stat[1], my_taps);
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long si = J.stat_index;
        atomicAdd((unsigned long long *)&stats[2 * si], s_stat[0]);
        atomicAdd((unsigned long long *)&stats[2 * si + 1], s_stat[1]);
    }
}

// ===========================================================================
// k_ism_taps: direct per-tap kernel
// ===========================================================================
// Three CTAs per SM (at most 85 registers; 80 are used, without spills):
// bounded at two, the compiler took 114-124 registers and the kernel stayed
// latency-bound at four warps per scheduler.
template <int R, int KIND>
__global__ void __launch_bounds__(NT, 3)
k_ism_taps(const RirJob *__restrict__ jobs, int n_rirs, int wmax, int W, int max_order,
           int max_taps, float *__restrict__ h, long long *__restrict__ stats,
           unsigned int *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Layout Lay = make_layout(false, W, max_order, max_taps, 0);
    const int TE = Lay.TE;
    Tables T;
    double *s_sq = (double *)(smem + Lay.off_sq);
    T.sq = s_sq;
    T.hlg = (float4 *)(smem + Lay.off_hlg);
    T.dl = (float *)(smem + Lay.off_dl);
    int *s_lx = (int *)(smem + Lay.off_lx);
    int *s_ly = (int *)(smem + Lay.off_ly);
    uint32_t *s_cand = (uint32_t *)(smem + Lay.off_cand);
    float *s_rows = (float *)(smem + Lay.off_rows);
    __shared__ int s_scan[NW];
    __shared__ int s_item, s_nl[2];
    __shared__ unsigned long long s_stat[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HALO = max_taps - 1;
    const int RL = Lay.RL;

    for (int i = tid; i < NW * RL; i += NT) s_rows[i] = 0.f;

    const long long n_items = (long long)n_rirs * wmax;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= n_items) break;
        const int wi = wmax - 1 - (int)(item / n_rirs);
        const RirJob &J = jobs[(int)(item % n_rirs)];
        if (wi >= J.n_windows) { __syncthreads(); continue; }
        Item it;
        item_setup<KIND>(J, W, wi, it);
        build_tables(J, T, s_sq, TE, it);
        if (tid < 2) s_stat[tid] = 0ull;
        __syncthreads();
        build_lists(T, TE, it, s_lx, s_ly, s_nl);
        const int H = it.H, P = it.P, w0 = it.w0;
        // per-lane tap constants
        float cC[R], cS[R], cQ[R], cSJ[R], cMS[R];
        bool cOK[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (KIND == ISM_FD_HANN_SINC) {
                const int j = lane - H + 32 * r;
                cOK[r] = j <= H;
                const float sg = (j & 1) ? -1.f : 1.f;
                cSJ[r] = sg * (float)j;
                cMS[r] = -sg;
                // ch, sh = cos, sin(pi j / (2 (H + 1))) from the
                // complementary angle pi (H + 1 - |j|) / (2 (H + 1)), whose
                // exact integer numerator keeps the small cosines of the
                // outer taps at full relative precision
                const int aj = j < 0 ? -j : j;
                float sx, cx;
                sincospif((float)(H + 1 - aj) / (float)(2 * (H + 1)), &sx, &cx);
                const float ch = sx, sh = j < 0 ? -cx : cx;
                cC[r] = ch * ch;
                cS[r] = ch * sh;
                cQ[r] = sh * sh;
            } else {
                const int j = lane + 32 * r;
                cOK[r] = j <= P;
                float den = 1.f;
                for (int i = 0; i <= P; ++i)
                    if (i != j) den *= (float)(j - i);
                cC[r] = cOK[r] ? 1.f / den : 0.f;
                cS[r] = cQ[r] = cSJ[r] = cMS[r] = 0.f;
            }
        }
        __syncthreads();
        const int nLX = s_nl[0], nLY = s_nl[1];
        unsigned long long my_contrib = 0, my_taps = 0;

        // flush: for each candidate, one warp lays its taps into that warp's
        // private row.  Candidates are handed out round-robin to warps in
        // candidate order; each thread evaluates its warp's candidates
        // lane-parallel first, then the warp walks them one by one.
        auto flush = [&](int nc) {
            __syncthreads();
            float *rowp = s_rows + warp * RL + lane;
            for (int base = warp * 32; base < nc; base += NW * 32) {
                const int ci = base + lane;
                int kb = INT32_MIN;
                float f = 0.f, a = 0.f;
                if (ci < nc) {
                    if (!eval_candidate<KIND>(T, TE, it, s_cand[ci], kb, f, a, my_taps,
                                              my_contrib))
                        kb = INT32_MIN;
                }
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (kb != INT32_MIN) {
                    if (KIND == ISM_FD_HANN_SINC) {
                        if (fabsf(f) < 1e-30f) {
                            v = make_float4(a, 0.f, 0.f, 0.f);
                        } else {
                            float sp, cp, sw, cw;
                            sincospif(f, &sp, &cp);
                            sincospif(f / (float)(2 * (H + 1)), &sw, &cw);
                            // a sinc(j - f) = A (-1)^j / (j - f), A = -a sin(pi f) / pi
                            const float A = -a * sp * 0.3183098861837907f;
                            v = make_float4(A * (cw * cw), A * (2.f * cw * sw), A * (sw * sw), f);
                        }
                    } else {
                        v = make_float4(a, f + (float)((P - 1) / 2), 0.f, 0.f);
                    }
                }
                unsigned vm = __ballot_sync(0xffffffffu, kb != INT32_MIN);
                while (vm) {
                    const int src = __ffs(vm) - 1;
                    vm &= vm - 1;
                    const int kbs = __shfl_sync(0xffffffffu, kb, src);
                    const float vx = __shfl_sync(0xffffffffu, v.x, src);
                    const float vy = __shfl_sync(0xffffffffu, v.y, src);
                    const float vz = __shfl_sync(0xffffffffu, v.z, src);
                    const float vw = __shfl_sync(0xffffffffu, v.w, src);
                    // row index of tap index n is n - w0 + HALO, in [0, RL)
                    const int ri = kbs - w0 + HALO;
                    if (!ISM_IN_RANGE(ri >= 0 && ri + it.n_taps - 1 < RL, kOobDirectRow))
                        continue;
                    float *p = rowp + ri;
                    if (KIND == ISM_FD_HANN_SINC) {
                        if (vw == 0.f) {
                            if (lane == 0) p[H] += vx;
                            continue;
                        }
                        // Hann window w(t) = (1 + cos(pi t / (H + 1))) / 2 as
                        // cos^2(pi t / (2 (H + 1))), t = j - f, the square of
                        // ch cos(b) + sh sin(b) (b = pi f / (2 (H + 1)))
                        // expanded over per-lane and per-image products: its
                        // terms cancel at most a few-fold, where 1 + cos
                        // would lose most bits at the outer taps
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if (cOK[r]) {
                                const float xs = fmaf(cMS[r], vw, cSJ[r]);
                                const float rcp = rcp_approx(xs);
                                const float nn = fmaf(cC[r], vx, fmaf(cS[r], vy, cQ[r] * vz));
                                p[32 * r] = fmaf(nn, rcp, p[32 * r]);
                            }
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            if (cOK[r]) {
                                const int j = lane + 32 * r;
                                float prod = cC[r];
                                for (int i2 = 0; i2 <= P; ++i2)
                                    if (i2 != j) prod *= (vy - (float)i2);
                                p[32 * r] = fmaf(vx, prod, p[32 * r]);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        };
        column_sweep(T, TE, it, s_lx, s_ly, nLX, nLY, s_scan, s_cand, flush);

        // window output: fixed-order sum of the private rows
        __syncthreads();
        float *hout = h + J.h_offset;
        for (int i = tid; i < W; i += NT) {
            const long long n = (long long)w0 + i;
            float acc = 0.f;
#pragma unroll
            for (int wv = 0; wv < NW; ++wv) acc += s_rows[wv * RL + HALO + i];
            if (n < it.Lh) hout[n] = acc;
        }
        __syncthreads();
        for (int i = tid; i < NW * RL; i += NT) s_rows[i] = 0.f;
        flush_stats(stats, J, s_stat, my_contrib, my_taps);
        __syncthreads();
    }
}

// ===========================================================================
// k_ism_sparse: sparse integer-delay arrays + Chebyshev FIR
// ===========================================================================
// Fixed-point sparse arrays.  Per window, gains are scaled so that the
// largest gain an image reaching the window can have, a_max = 1/(4 pi
// d_floor) (d_floor: the window's first delay, or the direct path, which no
// image undercuts for points inside the box; beta <= 1), maps to kFix0 =
// 2^24.  Term p of an image is rounded to an int32 and added with a native
// u32 shared-memory atomic: an FP32 shared atomic costs a load and a
// compare-and-swap on this GPU, and shared-memory wavefronts bound this
// kernel.  c_0 = sum of a >= |c_p| for every p (|T_p| <= 1), so while no c_0
// entry (nor an integer-delay entry, also a sum of gains) passes kFixLimit
// = 2^31 - 2^25, every array ends at its exact integer sum in int32 range
// (wrap-around of intermediate sums cancels modulo 2^32).  The c_0 update
// returns the old value; a sum past the limit flags the window, which is
// redone at a 2^7 coarser scale (so the quantum stays near 2^-24 of the
// largest sum).  The fourth attempt takes the scale at which n_bound images
// at a_max stay below the limit: one delay bucket (one sample) holds at most
// n_bound = 4 C (l / (2 Lz) + 1) images, C = (2 (2N+1))^2 lattice columns,
// each meeting the bucket's spherical shell in at most two z-intervals of
// length l <= sqrt(2 d t + t^2) per z-parity (t: the bucket's width in
// metres, d: the window's largest distance).  Integer sums do not depend on
// the order of the additions: the sparse path is bitwise reproducible.
// Sets n4 16-byte words of shared memory to zero (all threads of the CTA).
__device__ __forceinline__ void zero_words4(void *p, int n4) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    for (int i = threadIdx.x; i < n4; i += NT) q[i] = make_uint4(0u, 0u, 0u, 0u);
}

// Fixed point -> float in place over n4 16-byte words: v * inv_s, the words
// read as int32 (SIGNED) or uint32.
template <bool SIGNED>
__device__ __forceinline__ void fix_to_float4(void *p, int n4, float inv_s) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
    float4 *f = reinterpret_cast<float4 *>(p);
    for (int i = threadIdx.x; i < n4; i += NT) {
        const uint4 v = q[i];
        float4 o;
        if (SIGNED) {
            o.x = (float)(int)v.x * inv_s; o.y = (float)(int)v.y * inv_s;
            o.z = (float)(int)v.z * inv_s; o.w = (float)(int)v.w * inv_s;
        } else {
            o.x = (float)v.x * inv_s; o.y = (float)v.y * inv_s;
            o.z = (float)v.z * inv_s; o.w = (float)v.w * inv_s;
        }
        f[i] = o;
    }
}

constexpr double kFix0 = 16777216.0;           // 2^24
constexpr uint32_t kFixLimit = 0x7e000000u;    // 2^31 - 2^25

// PFIX > 0: every job of the launch has PFIX Chebyshev terms (the term loop
// is unrolled); 0: per-job count.  SPEC > 0: the launch's window is kSpecW
// and every job has SPEC taps (the dataset's 81-tap Hann sinc, or the
// paper's 8-tap Lagrange filter), so the sparse arrays' stride, the FIR's
// tap loop and the window loop are compile-time constants (the term atomics
// address their arrays with immediate offsets).
constexpr int kSpecW = 1024;

template <int KIND, bool STATS, int PFIX, int SPEC>
__global__ void __launch_bounds__(NT, 4)
k_ism_sparse(const RirJob *__restrict__ jobs, int n_rirs, int wmax, int W_arg, int max_order,
             int max_taps_arg, int max_cheb, const float *__restrict__ tabs, float *__restrict__ h,
             long long *__restrict__ stats, unsigned int *__restrict__ counter,
             const double *__restrict__ g_sq, const float4 *__restrict__ g_hlg,
             const float *__restrict__ g_dl, const JobConst *__restrict__ g_jc,
             const uint32_t *__restrict__ g_cols, const int2 *__restrict__ g_wr,
             const long long *__restrict__ g_offs) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int W = SPEC ? kSpecW : W_arg;
    const int max_taps = SPEC ? SPEC : max_taps_arg;
    const Layout Lay = make_layout(true, W, max_order, max_taps, max_cheb);
    const int TE = Lay.TE;
    const int CL = SPEC ? round64(kSpecW + SPEC + 12 + PADL) : Lay.CL;
    Tables T;
    T.sq = nullptr;  // per item: the RIR's FP64 table in global memory (exact path only)
    T.hlg = (float4 *)(smem + Lay.off_hlg);
    T.dl = (float *)(smem + Lay.off_dl);
    float *s_c = (float *)(smem + Lay.off_c);
    float *s_delta = (float *)(smem + Lay.off_delta);
    float *s_part = (float *)(smem + Lay.off_part);
    __shared__ int s_item, s_ovf;
    __shared__ unsigned long long s_stat[2];

    const int tid = threadIdx.x;
    uint32_t *s_cq = (uint32_t *)s_c;      // the same words before conversion
    uint32_t *s_dq = (uint32_t *)s_delta;
    // CL is a multiple of 64 and both arrays start on 16-byte boundaries
    zero_words4(s_cq, max_cheb * CL / 4);
    zero_words4(s_dq, CL / 4);
    if (tid == 0) s_ovf = 0;

    const long long n_items = (long long)n_rirs * wmax;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= n_items) break;
        const int wi = wmax - 1 - (int)(item / n_rirs);
        const int jr = (int)(item % n_rirs);
        const RirJob &J = jobs[jr];
        if (wi >= J.n_windows) { __syncthreads(); continue; }
        {
            // the RIR's tables, computed once per RIR by k_ism_tables
            const int TEj = 2 * (2 * J.order + 1);
            const size_t base = (size_t)jr * 3 * TE;
            for (int e = tid; e < 3 * TEj; e += NT) {
                const int a = e / TEj, ei = e - a * TEj;
                T.hlg[a * TE + ei] = g_hlg[base + a * TE + ei];
                T.dl[a * TE + ei] = g_dl[base + a * TE + ei];
            }
            T.sq = g_sq + base;
        }
        if (tid == 0) {
            s_stat[0] = s_stat[1] = 0ull;
            s_ovf = 0;
        }
        __syncthreads();
        // per-window constants, FP32 (see item_setup_f32)
        Item it;
        float tau_lo, tau_hi;
        const JobConst jc = g_jc[jr];
        item_setup_f32<KIND>(J, jc, W, wi, it, tau_lo, tau_hi);
        if (SPEC) {  // the same values, known to the compiler
            it.n_taps = SPEC;
            it.H = (SPEC - 1) / 2;
            it.P = SPEC - 1;
            it.W = kSpecW;
        }
        // fixed-point scales (see kFix0): d_floor bounds from below the
        // distance of every image whose taps reach this window; one delay
        // bucket holds at most n_bound images
        const float d_floor = fmaxf(jc.d_dir, tau_lo * jc.inv_q) * (1.f - 1e-5f);
        const float tb = (1.f + 1e-5f) * jc.inv_q, dmax = tau_hi * jc.inv_q + tb;
        const float ncol = 4.f * (float)(2 * it.N + 1) * (float)(2 * it.N + 1);
        const float n_bound = 4.f * ncol * (sqrtf(2.f * dmax * tb + tb * tb) * jc.inv2Lz + 1.f);
        const float S0 = (float)kFix0 * 12.566370614359172f * d_floor;
        auto scale_of = [&](int at) {
            // a_max = 1 / (4 pi d_floor) maps to kFix0, then 2^7 less per
            // retry; the fourth attempt takes the scale at which n_bound
            // images at a_max cannot exceed the limit
            if (at < 3) return ldexpf(S0, -7 * at);
            return fminf(ldexpf(S0, -21),
                         0.5f * (float)kFixLimit * 12.566370614359172f * d_floor / n_bound);
        };
        const int Pc = J.n_cheb;
        const int n_taps = SPEC ? SPEC : it.n_taps;
        // this window's ranks in the RIR's sorted column list
        const int2 wr = g_wr[g_offs[2 * jr + 1] + wi];
        const uint32_t *cols = g_cols + g_offs[2 * jr];
        // position of first-tap index kb in the sparse arrays; chosen so that
        // the FIR's 128-bit loads are aligned
        const int OFF = (4 - (n_taps - 1) % 4) % 4;
        const int POS0 = OFF + PADL - (int)it.kb_lo;
        const int jdelta = (KIND == ISM_FD_HANN_SINC) ? it.H : (it.P - 1) / 2;
        unsigned my_contrib = 0, my_taps = 0;
        float S = 0.f, S4 = 0.f;
        auto proc = [&](float Rh, float Rl, float gxy, int iz, int ix, int iy) {
            int kb;
            float f, a;
            if (!eval_expanded<KIND, STATS>(T, TE, it, Rh, Rl, gxy, iz, ix, iy, kb, f, a, my_taps,
                                            my_contrib))
                return;
            const int pos = kb + POS0;
            if (!ISM_IN_RANGE(pos >= 0 && pos < CL, kOobSparsePos)) return;
            const int sp = swz(pos);
            const float as = a * S4;  // a S, with a = prod(beta^hits) / (4 pi d)
                                      // (a = g / tau here, S4 = S q / (4 pi))
            const uint32_t q0 = __float2uint_rn(as);
            uint32_t *c0 = (f == 0.f) ? s_dq : s_cq;  // integer delay: exact Kronecker delta
            const uint32_t old = atomicAdd(&c0[sp], q0);
            if (f != 0.f) {
                // u_p = a S T_p(x) by the Chebyshev recurrence on the scaled
                // values, u_{p+1} = 2 x u_p - u_{p-1}: one FMA, one conversion
                // and one atomic per term
                const float x = (KIND == ISM_FD_HANN_SINC) ? 2.f * f : 2.f * f - 1.f;
                const float x2 = 2.f * x;
                uint32_t *cp = s_cq + sp;
                float u0 = as, u1 = as * x;
                if (PFIX > 0) {
                    atomicAdd(cp + CL, (uint32_t)__float2int_rn(u1));
#pragma unroll
                    for (int p = 2; p < PFIX; ++p) {
                        const float u2 = fmaf(x2, u1, -u0);
                        atomicAdd(cp + p * CL, (uint32_t)__float2int_rn(u2));
                        u0 = u1;
                        u1 = u2;
                    }
                } else {
                    if (Pc > 1) atomicAdd(cp + CL, (uint32_t)__float2int_rn(u1));
                    for (int p = 2; p < Pc; ++p) {
                        const float u2 = fmaf(x2, u1, -u0);
                        atomicAdd(cp + p * CL, (uint32_t)__float2int_rn(u2));
                        u0 = u1;
                        u1 = u2;
                    }
                }
            }
            if (old + q0 > kFixLimit) s_ovf = 1;  // this window is redone at a coarser scale
        };
        float invS = 0.f;
        for (int attempt = 0;; ++attempt) {
            S = scale_of(attempt);
            S4 = S * (0.07957747154594767f * it.qh);  // S q / (4 pi): a = g / tau
            invS = 1.f / S;
            my_contrib = 0;
            my_taps = 0;
            sorted_sweep(T, TE, it, cols, wr.x, wr.y, proc);
            __syncthreads();
            const int ovf = s_ovf;
            if (!ovf || attempt >= 3) break;
            __syncthreads();
            if (tid == 0) s_ovf = 0;
            zero_words4(s_cq, Pc * CL / 4);
            zero_words4(s_dq, CL / 4);
            __syncthreads();
        }
        // fixed point -> float, in place (the integer-delay sums are >= 0)
        fix_to_float4<true>(s_c, Pc * CL / 4, invS);
        fix_to_float4<false>(s_delta, CL / 4, invS);
        __syncthreads();

        // FIR: h[w0+i] = sum_p sum_j B[p][j] c_p[kb = w0+i-j] + delta.  Threads
        // 0..127 take p in [0, ceil(P/2)), threads 128..255 the rest; each owns
        // 8 consecutive outputs and walks the taps 4 at a time with a sliding
        // 12-value window of c in registers (128-bit shared loads).  The
        // table B (rows padded to a multiple of 4 taps with zeros) is read
        // through the read-only cache; all lanes load the same words.
        {
            const int half = tid >> 7, gt = tid & 127;
            const int ph = (Pc + 1) / 2;
            const int p_lo = half ? ph : 0, p_hi = half ? Pc : ph;
            const int TPj = round4(n_taps);
            const float *Bj = tabs + J.tab_offset;
            for (int g0 = 0; g0 < W / 8; g0 += 128) {
                const int g = g0 + gt;
                float acc[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = 0.f;
                if (g < W / 8) {
                    const int base = 8 * g + n_taps - 1 + OFF + PADL;  // multiple of 4
                    for (int p = p_lo; p < p_hi; ++p) {
                        const float *cp = s_c + p * CL;
                        const float4 *bp = reinterpret_cast<const float4 *>(Bj + p * TPj);
                        // 12-register window: at sub-step s (taps jb + 4s ..
                        // jb + 4s + 3) logical value L = c[base - jb - 4s - 4 + L]
                        // sits in R[(L - 4s) mod 12], so three sub-steps rotate it
                        // in place without register moves
                        float R[12];
#pragma unroll
                        for (int v = 0; v < 3; ++v) {
                            const int fi = base - 4 + 4 * v;
                            const float4 w4 =
                                ISM_IN_RANGE(fi >= 0 && fi + 3 < CL, kOobFirRead)
                                    ? *reinterpret_cast<const float4 *>(cp + swz(fi))
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
                            R[4 * v] = w4.x; R[4 * v + 1] = w4.y;
                            R[4 * v + 2] = w4.z; R[4 * v + 3] = w4.w;
                        }
                        auto step = [&](int jb, auto sc) {
                            constexpr int S = decltype(sc)::value;
                            const float4 b4 = __ldg(bp + (jb >> 2) + S);
                            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                                for (int q = 0; q < 8; ++q)
                                    acc[q] = fmaf(bv[jj], R[(4 + q - jj - 4 * S + 12) % 12], acc[q]);
                            if (jb + 4 * S + 4 < TPj) {
                                const int fi = base - jb - 4 * S - 8;
                                const float4 w4 =
                                    ISM_IN_RANGE(fi >= 0 && fi + 3 < CL, kOobFirRead)
                                        ? *reinterpret_cast<const float4 *>(cp + swz(fi))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                                constexpr int d = (12 - 4 * (S + 1) % 12) % 12;
                                R[d] = w4.x; R[d + 1] = w4.y; R[d + 2] = w4.z; R[d + 3] = w4.w;
                            }
                        };
                        int jb = 0;
                        for (; jb + 12 <= TPj; jb += 12) {
                            step(jb, std::integral_constant<int, 0>{});
                            step(jb, std::integral_constant<int, 1>{});
                            step(jb, std::integral_constant<int, 2>{});
                        }
                        if (jb < TPj) step(jb, std::integral_constant<int, 0>{});
                        if (jb + 4 < TPj) step(jb, std::integral_constant<int, 1>{});
                    }
                    if (half) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) s_part[8 * g + q] = acc[q];
                    }
                }
                __syncthreads();
                if (!half && g < W / 8) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) s_part[8 * g + q] += acc[q];
                }
            }
        }
        __syncthreads();
        float *hout = h + J.h_offset;
        for (int i = tid; i < W; i += NT) {
            const long long n = (long long)it.w0 + i;
            const int di = i + n_taps - 1 - jdelta + OFF + PADL;
            const float v =
                s_part[i] + (ISM_IN_RANGE(di >= 0 && di < CL, kOobDeltaRead) ? s_delta[swz(di)] : 0.f);
            if (n < it.Lh) hout[n] = v;
        }
        __syncthreads();
        zero_words4(s_c, Pc * CL / 4);
        zero_words4(s_delta, CL / 4);
        flush_stats(stats, J, s_stat, my_contrib, my_taps);
        __syncthreads();
    }
}

// Per kernel and device: the dynamic shared memory limit set so far and the
// occupancy measured for the last size asked, so that a call of the same
// shape makes neither query again.
struct KernelCache {
    std::mutex mu;
    int smem_set[64] = {};
    size_t occ_smem[64] = {};
    int occ[64] = {};
};

// Raises the kernel's dynamic shared memory limit to smem if needed and
// returns its persistent grid (SMs x resident CTAs per SM).
template <class K>
int prepare_launch(K kern, KernelCache &c, size_t smem, const char *name, int *grid) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (d < 0 || d >= 64) return fail(ISM_ERR_INTERNAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(c.mu);
    if ((size_t)c.smem_set[d] < smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, (std::string("cudaFuncSetAttribute(") + name + ")").c_str());
        c.smem_set[d] = (int)smem;
        c.occ_smem[d] = 0;
    }
    if (c.occ_smem[d] != smem || c.occ[d] <= 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
        if (e != cudaSuccess) return cuda_fail(e, (std::string("occupancy(") + name + ")").c_str());
        c.occ[d] = per_sm > 0 ? per_sm : 1;
        c.occ_smem[d] = smem;
    }
    *grid = device_sm_count() * c.occ[d];
    return ISM_OK;
}

template <int R, int KIND>
int launch_direct_t(const RirLaunch &L, cudaStream_t stream) {
    const Layout Lay = make_layout(false, L.window, L.max_order, L.max_taps, 0);
    auto kern = k_ism_taps<R, KIND>;
    static KernelCache cache;
    int grid = 0;
    if (int st = prepare_launch(kern, cache, Lay.total, "k_ism_taps", &grid)) return st;
    if (L.grid > 0) grid = L.grid;
    cudaError_t e = cudaSuccess;
    const long long items = (long long)L.n_rirs * L.wmax;
    if ((long long)grid > items) grid = (int)items;
    if (grid < 1) return ISM_OK;
    kern<<<grid, NT, Lay.total, stream>>>(L.jobs_dev, L.n_rirs, L.wmax, L.window, L.max_order,
                                          L.max_taps, L.h_dev, L.stats_dev, L.counter_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_ism_taps");
    return ISM_OK;
}

template <int KIND, bool STATS, int PFIX, int SPEC = 0>
int launch_sparse_t(const RirLaunch &L, cudaStream_t stream) {
    const Layout Lay = make_layout(true, L.window, L.max_order, L.max_taps, L.max_cheb);
    auto kern = k_ism_sparse<KIND, STATS, PFIX, SPEC>;
    static KernelCache cache;
    int grid = 0;
    if (int st = prepare_launch(kern, cache, Lay.total, "k_ism_sparse", &grid)) return st;
    if (L.grid > 0) grid = L.grid;
    const long long items = (long long)L.n_rirs * L.wmax;
    if ((long long)grid > items) grid = (int)items;
    if (grid < 1) return ISM_OK;
    // per-RIR tables: FP64 squares, (hi, lo, damping) and offsets, in the
    // caller's scratch when it gave some
    const size_t n_ent = (size_t)L.n_rirs * 3 * Lay.TE;  // even: TE = 2 (2N + 1)
    void *tab = L.tables_dev;
    if (!tab) {
        if (int st = scratch_alloc(&tab, rir_tables_bytes(L.n_rirs, L.max_order), stream))
            return st;
    }
    double *g_sq = (double *)tab;
    float4 *g_hlg = (float4 *)(g_sq + n_ent);
    JobConst *g_jc = (JobConst *)(g_hlg + n_ent);
    float *g_dl = (float *)(g_jc + L.n_rirs);
    const int tgrid = (int)std::min<long long>(L.n_rirs, (long long)device_sm_count() * 8);
    k_ism_tables<KIND><<<tgrid, TNT, 0, stream>>>(L.jobs_dev, L.n_rirs, Lay.TE, L.window, g_sq,
                                                  g_hlg, g_dl, g_jc, L.cols_dev, L.wr_dev,
                                                  L.offs_dev);
    kern<<<grid, NT, Lay.total, stream>>>(L.jobs_dev, L.n_rirs, L.wmax, L.window, L.max_order,
                                          L.max_taps, L.max_cheb, L.tabs_dev, L.h_dev,
                                          L.stats_dev, L.counter_dev, g_sq, g_hlg, g_dl, g_jc,
                                          L.cols_dev, L.wr_dev, L.offs_dev);
    const cudaError_t e = cudaGetLastError();
    if (!L.tables_dev) scratch_free(tab, stream);
    if (e != cudaSuccess) return cuda_fail(e, "launch k_ism_sparse");
    return ISM_OK;
}

}  // namespace

ISM_OOB_READER(rir)

size_t rir_smem_bytes(int window, int max_order, int max_taps) {
    return make_layout(false, window, max_order, max_taps, 0).total;
}

size_t rir_sparse_smem_bytes(int window, int max_order, int max_taps, int max_cheb) {
    return make_layout(true, window, max_order, max_taps, max_cheb).total;
}

size_t rir_tables_bytes(long long n_rirs, int max_order) {
    const size_t n_ent = (size_t)n_rirs * 3 * (size_t)(2 * (2 * max_order + 1));
    return n_ent * (sizeof(double) + sizeof(float4) + sizeof(float)) +
           (size_t)n_rirs * sizeof(JobConst);
}

int launch_rir(const RirLaunch &L, cudaStream_t stream) {
    if (L.fd_kind == ISM_FD_LAGRANGE) return launch_direct_t<1, ISM_FD_LAGRANGE>(L, stream);
    const int rows = (L.max_taps + 31) / 32;
    switch (rows) {
        case 1: return launch_direct_t<1, ISM_FD_HANN_SINC>(L, stream);
        case 2: return launch_direct_t<2, ISM_FD_HANN_SINC>(L, stream);
        case 3: return launch_direct_t<3, ISM_FD_HANN_SINC>(L, stream);
        case 4: return launch_direct_t<4, ISM_FD_HANN_SINC>(L, stream);
        case 5: return launch_direct_t<5, ISM_FD_HANN_SINC>(L, stream);
        case 6: return launch_direct_t<6, ISM_FD_HANN_SINC>(L, stream);
        case 7: return launch_direct_t<7, ISM_FD_HANN_SINC>(L, stream);
        case 8: return launch_direct_t<8, ISM_FD_HANN_SINC>(L, stream);
        default: return fail(ISM_ERR_INVALID_ARG, "n_taps above 255 is not supported");
    }
}

int launch_rir_sparse(const RirLaunch &L, cudaStream_t stream) {
    if (L.window % 8 != 0) return fail(ISM_ERR_INVALID_ARG, "window must be a multiple of 8");
    if (L.max_cheb < 1 || L.max_cheb > kMaxCheb)
        return fail(ISM_ERR_INVALID_ARG, "Chebyshev term count out of range");
    if (!L.cols_dev || !L.wr_dev || !L.offs_dev)
        return fail(ISM_ERR_INTERNAL, "sparse launch without column-list scratch");
    if (L.max_order > 200) return fail(ISM_ERR_INVALID_ARG, "order above 200");
    const bool st = L.stats_dev != nullptr;  // statistics compiled out when not asked for
    const int pf = L.min_cheb == L.max_cheb ? L.max_cheb : 0;
    if (L.fd_kind == ISM_FD_LAGRANGE) {
        if (pf == 8 && L.window == kSpecW && L.max_taps == 8 && L.min_taps == 8)
            return st ? launch_sparse_t<ISM_FD_LAGRANGE, true, 8, 8>(L, stream)
                      : launch_sparse_t<ISM_FD_LAGRANGE, false, 8, 8>(L, stream);
        if (pf == 8)
            return st ? launch_sparse_t<ISM_FD_LAGRANGE, true, 8>(L, stream)
                      : launch_sparse_t<ISM_FD_LAGRANGE, false, 8>(L, stream);
        return st ? launch_sparse_t<ISM_FD_LAGRANGE, true, 0>(L, stream)
                  : launch_sparse_t<ISM_FD_LAGRANGE, false, 0>(L, stream);
    }
    if (pf == 9)
        return st ? launch_sparse_t<ISM_FD_HANN_SINC, true, 9>(L, stream)
                  : launch_sparse_t<ISM_FD_HANN_SINC, false, 9>(L, stream);
    if (pf == 8 && L.window == kSpecW && L.max_taps == 81 && L.min_taps == 81)
        return st ? launch_sparse_t<ISM_FD_HANN_SINC, true, 8, 81>(L, stream)
                  : launch_sparse_t<ISM_FD_HANN_SINC, false, 8, 81>(L, stream);
    if (pf == 8)
        return st ? launch_sparse_t<ISM_FD_HANN_SINC, true, 8>(L, stream)
                  : launch_sparse_t<ISM_FD_HANN_SINC, false, 8>(L, stream);
    return st ? launch_sparse_t<ISM_FD_HANN_SINC, true, 0>(L, stream)
              : launch_sparse_t<ISM_FD_HANN_SINC, false, 0>(L, stream);
}

}  // namespace ism
