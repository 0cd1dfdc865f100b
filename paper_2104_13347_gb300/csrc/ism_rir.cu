// ism_rir.cu -- K1: image-source room impulse responses on sm_103a.
//
// Computes, for every (room, microphone) RIR, the sum over the image lattice
// of arXiv 2104.13347, Sec. II.A: each image (u,v,w,l,m,n) at distance d
// contributes a fractional-delay tap group at tau = d fs / c with gain
// prod(beta^hits) / (4 pi d).
//
// Work decomposition (GB300-first, no global atomics on h):
//  * A work item is one output window [w0, w0+W) of one RIR.  A persistent
//    grid (SMs x 2 CTAs) pulls items from one atomic counter, later windows
//    (more images) first.
//  * The CTA enumerates only the images whose taps reach its window: per
//    lattice column (u,l,v,m,w) the admissible n form at most two intervals
//    (a quadratic in n), solved in FP32 with a safety margin; each candidate
//    is then tested exactly on its delay.
//  * Delays: image-to-mic squared offsets per axis are tabled once per item in
//    FP64 with the definition's rounding, d^2 and sqrt are done in
//    float-float (FP32 pipe; GB300's FP64 rate is a small fraction of FP32),
//    and the integer split is redone in FP64 with the definition's exact
//    operation order whenever the float-float delay lies within 1e-6 samples
//    of a rounding boundary or of an integer (so exact integer delays give
//    exact Kronecker deltas).  The integer part therefore equals the
//    definition's bit for bit, and the fractional part to ~1e-9 samples.
//  * Taps: one warp per image, one lane per tap (81 taps -> 3 rows of 32).
//    sin(pi (j-f)) = -(-1)^j sin(pi f) and the Hann term is expanded in
//    cos/sin of pi j/(H+1) (per-lane constants) and of pi f/(H+1) (per
//    image), leaving one reciprocal per tap.  Each warp accumulates into its
//    own shared-memory copy of the window (no atomics, fixed order), and the
//    copies are summed in a fixed order into coalesced stores of h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ism_internal.h"

namespace ism {
namespace {

constexpr int NT = 256;           // threads per CTA
constexpr int NW = NT / 32;       // warps per CTA
constexpr int CAP = 2048;         // candidate / record buffer (images)
constexpr int CPT = CAP / NT;     // candidates per thread in the record phase
constexpr float kEps = 0.2f;      // metres of margin in the column solve

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

struct Tables {
    double *sq;   // [3][TE] squared axis offsets (FP64, definition rounding)
    float *hi;    // [3][TE] float-float split of sq
    float *lo;
    float *dl;    // [3][TE] axis offset, FP32
    float *g;     // [3][TE] wall damping product along the axis
};

// Shared-memory carve-up (sizes from the launch's max order / taps).
struct Layout {
    int TE;       // table entries per axis: 2 (2 Nmax + 1)
    int RL;       // private row length in floats
    size_t off_sq, off_hi, off_lo, off_dl, off_g, off_lx, off_ly, off_cand, off_rec4,
        off_reck, off_idx, off_rows, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline Layout make_layout(int window, int max_order, int max_taps) {
    Layout L;
    L.TE = 2 * (2 * max_order + 1);
    L.RL = (window + 2 * (max_taps - 1) + 3) & ~3;
    size_t o = 0;
    L.off_sq = o;   o = align16(o + sizeof(double) * 3 * L.TE);
    L.off_hi = o;   o = align16(o + sizeof(float) * 3 * L.TE);
    L.off_lo = o;   o = align16(o + sizeof(float) * 3 * L.TE);
    L.off_dl = o;   o = align16(o + sizeof(float) * 3 * L.TE);
    L.off_g = o;    o = align16(o + sizeof(float) * 3 * L.TE);
    L.off_lx = o;   o = align16(o + sizeof(int) * L.TE);
    L.off_ly = o;   o = align16(o + sizeof(int) * L.TE);
    L.off_cand = o; o = align16(o + sizeof(uint32_t) * CAP);
    L.off_rec4 = o; o = align16(o + sizeof(float4) * CAP);
    L.off_reck = o; o = align16(o + sizeof(int) * CAP);
    L.off_idx = o;  o = align16(o + sizeof(uint16_t) * CAP);
    L.off_rows = o; o = align16(o + sizeof(float) * (size_t)NW * L.RL);
    L.total = o;
    return L;
}

// Image record of one candidate (shared memory, at the candidate's slot):
// first tap index kb, and v = (A, A cos(pi f/(H+1)), A sin(pi f/(H+1)), f)
// with A = -a sin(pi f) / (2 pi) for the Hann-sinc filter, or v = (a, D)
// for the Lagrange filter.

// Delay split of one image (Sec. II.A: the delay of every image must keep
// its sub-sample precision).  Returns the integer part k (rint, ties to even, for Hann;
// floor for Lagrange) and the fraction in FP32, plus d (FP32).
template <int KIND>
__device__ __forceinline__ void delay_split(const Tables &T, int TE, int ix, int iy, int iz,
                                            float qh, float ql, double q, int &k_out,
                                            float &f_out, float &d_out) {
    const float xh = T.hi[ix], xl = T.lo[ix];
    const float yh = T.hi[TE + iy], yl = T.lo[TE + iy];
    const float zh = T.hi[2 * TE + iz], zl = T.lo[2 * TE + iz];
    // d^2 = x + y + z in float-float (two-sum with renormalisation).
    float s1 = __fadd_rn(xh, yh);
    float bb = __fsub_rn(s1, xh);
    float e1 = __fadd_rn(__fsub_rn(xh, __fsub_rn(s1, bb)), __fsub_rn(yh, bb));
    e1 = __fadd_rn(e1, __fadd_rn(xl, yl));
    float t1 = __fadd_rn(s1, e1);
    e1 = __fsub_rn(e1, __fsub_rn(t1, s1));
    s1 = t1;
    float s2 = __fadd_rn(s1, zh);
    bb = __fsub_rn(s2, s1);
    float e2 = __fadd_rn(__fsub_rn(s1, __fsub_rn(s2, bb)), __fsub_rn(zh, bb));
    e2 = __fadd_rn(e2, __fadd_rn(e1, zl));
    const float Dh = __fadd_rn(s2, e2);
    const float Dl = __fsub_rn(e2, __fsub_rn(Dh, s2));
    // sqrt: FP32 estimate plus one Newton correction in float-float.
    const float r = rsqrtf(Dh);
    const float s0 = __fmul_rn(Dh, r);
    const float res = __fadd_rn(__fmaf_rn(-s0, s0, Dh), Dl);
    float dh = s0;
    float dl = __fmul_rn(res, __fmul_rn(0.5f, r));
    float tt = __fadd_rn(dh, dl);
    dl = __fsub_rn(dl, __fsub_rn(tt, dh));
    dh = tt;
    // tau = d * q in float-float.
    const float th = __fmul_rn(dh, qh);
    const float terr = __fmaf_rn(dh, qh, -th);
    const float tl = __fadd_rn(terr, __fmaf_rn(dh, ql, __fmul_rn(dl, qh)));
    float k, f;
    bool near;
    if (KIND == ISM_FD_HANN_SINC) {
        k = rintf(th);
        f = __fadd_rn(__fsub_rn(th, k), tl);
        if (f > 0.5f) { k += 1.f; f -= 1.f; }
        else if (f < -0.5f) { k -= 1.f; f += 1.f; }
        near = fabsf(f) > 0.5f - 1e-6f || fabsf(f) < 1e-6f;  // ties and integers
    } else {
        k = floorf(th);
        f = __fadd_rn(__fsub_rn(th, k), tl);
        if (f >= 1.f) { k += 1.f; f -= 1.f; }
        else if (f < 0.f) { k -= 1.f; f += 1.f; }
        near = f < 1e-6f || f > 1.f - 1e-6f;
    }
    if (near) {
        // Exact path: the definition's FP64 operations in its order.
        const double d2 = __dadd_rn(__dadd_rn(T.sq[ix], T.sq[TE + iy]), T.sq[2 * TE + iz]);
        const double d = __dsqrt_rn(d2);
        const double tau = __dmul_rn(d, q);
        const double kd = (KIND == ISM_FD_HANN_SINC) ? rint(tau) : floor(tau);
        k = (float)kd;
        f = (float)(tau - kd);
    }
    k_out = (int)k;
    f_out = f;
    d_out = dh;
}

template <int R, int KIND>
__global__ void __launch_bounds__(NT, 2)
k_ism_taps(const RirJob *__restrict__ jobs, int n_rirs, int wmax, int W, int max_order,
           int max_taps, float *__restrict__ h, long long *__restrict__ stats,
           unsigned int *__restrict__ counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Layout Lay = make_layout(W, max_order, max_taps);
    const int TE = Lay.TE;
    Tables T;
    T.sq = (double *)(smem + Lay.off_sq);
    T.hi = (float *)(smem + Lay.off_hi);
    T.lo = (float *)(smem + Lay.off_lo);
    T.dl = (float *)(smem + Lay.off_dl);
    T.g = (float *)(smem + Lay.off_g);
    int *s_lx = (int *)(smem + Lay.off_lx);
    int *s_ly = (int *)(smem + Lay.off_ly);
    uint32_t *s_cand = (uint32_t *)(smem + Lay.off_cand);
    float4 *s_rec4 = (float4 *)(smem + Lay.off_rec4);
    int *s_reck = (int *)(smem + Lay.off_reck);
    uint16_t *s_idx = (uint16_t *)(smem + Lay.off_idx);
    float *s_rows = (float *)(smem + Lay.off_rows);
    __shared__ int s_scan[NW];
    __shared__ int s_item, s_nl[2];
    __shared__ unsigned long long s_stat[2];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int HALO = max_taps - 1;
    const int RL = Lay.RL;

    // Private rows start zeroed; each item leaves them zeroed.
    for (int i = tid; i < NW * RL; i += NT) s_rows[i] = 0.f;

    const long long n_items = (long long)n_rirs * wmax;
    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const long long item = s_item;
        if (item >= n_items) break;
        const int wi = wmax - 1 - (int)(item / n_rirs);
        const int ji = (int)(item % n_rirs);
        const RirJob &J = jobs[ji];
        if (wi >= J.n_windows) { __syncthreads(); continue; }

        const int N = J.order;
        const int TEj = 2 * (2 * N + 1);
        const int n_taps = J.n_taps;
        const int H = (n_taps - 1) / 2;            // Hann half-width
        const int P = n_taps - 1;                   // Lagrange order
        const long long Lh = J.rir_len;
        const int w0 = wi * W;
        const double q = J.q;
        const float qh = (float)q;
        const float ql = (float)(q - (double)qh);

        // ---- per-axis tables (FP64 offsets with the definition's rounding)
        for (int e = tid; e < 3 * TEj; e += NT) {
            const int a = e / TEj, ei = e - a * TEj;
            const int p = ei / (2 * N + 1), qq = ei - p * (2 * N + 1) - N;
            const double s = J.src[a], Ld = J.dims[a], r = J.mic[a];
            const double img = __dadd_rn(p ? -s : s, __dmul_rn((double)(2 * qq), Ld));
            const double dlt = __dsub_rn(img, r);
            const double sq = __dmul_rn(dlt, dlt);
            const float sh = __double2float_rn(sq);
            T.sq[a * TE + ei] = sq;
            T.hi[a * TE + ei] = sh;
            T.lo[a * TE + ei] = __double2float_rn(sq - (double)sh);
            T.dl[a * TE + ei] = __double2float_rn(dlt);
            const float b0 = J.beta[2 * a], b1 = J.beta[2 * a + 1];
            T.g[a * TE + ei] = powf(b0, (float)abs(qq - p)) * powf(b1, (float)abs(qq));
        }
        if (tid < 2) s_stat[tid] = 0ull;

        // ---- window bounds: first-tap index kb in [kb_lo, kb_hi]
        const long long kb_lo = (long long)w0 - n_taps + 1;
        const long long kb_hi = min((long long)w0 + W - 1, Lh - 1);
        double tau_lo, tau_hi;
        if (KIND == ISM_FD_HANN_SINC) {
            tau_lo = (double)(kb_lo + H) - 0.5;
            tau_hi = (double)(kb_hi + H) + 0.5;
        } else {
            tau_lo = (double)(kb_lo + (P - 1) / 2);
            tau_hi = (double)(kb_hi + (P + 1) / 2);
        }
        const float d_lo = (float)fmax(tau_lo / q, 0.0);
        const float d_hi = (float)(tau_hi / q);
        const float eps = kEps + 1e-6f * d_hi;
        const float dlo2 = d_lo * d_lo, dhi2 = d_hi * d_hi;
        const float dhe = d_hi + eps, dhe2 = dhe * dhe;
        __syncthreads();

        // ---- axis lists: entries whose offset alone is within reach
        if (warp < 2) {
            const float *dd = T.dl + warp * TE;
            int *lst = warp ? s_ly : s_lx;
            int cnt = 0;
            for (int base = 0; base < TEj; base += 32) {
                const int e = base + lane;
                const bool ok = e < TEj && fabsf(dd[e]) <= dhe;
                const unsigned b = __ballot_sync(0xffffffffu, ok);
                if (ok) lst[cnt + __popc(b & ((1u << lane) - 1u))] = e;
                cnt += __popc(b);
            }
            if (lane == 0) s_nl[warp] = cnt;
        }
        // per-lane tap constants
        float cC[R], cS[R], cSJ[R], cMS[R];
        bool cOK[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (KIND == ISM_FD_HANN_SINC) {
                const int j = lane - H + 32 * r;
                cOK[r] = j <= H;
                const float sg = (j & 1) ? -1.f : 1.f;
                cSJ[r] = sg * (float)j;
                cMS[r] = -sg;
                sincospif((float)j / (float)(H + 1), &cS[r], &cC[r]);
            } else {
                const int j = lane + 32 * r;
                cOK[r] = j <= P;
                float den = 1.f;
                for (int i = 0; i <= P; ++i)
                    if (i != j) den *= (float)(j - i);
                cC[r] = cOK[r] ? 1.f / den : 0.f;
                cS[r] = cSJ[r] = cMS[r] = 0.f;
            }
        }
        __syncthreads();
        const int nLX = s_nl[0], nLY = s_nl[1];
        const long long n_cols = (long long)nLX * nLY * 2;
        const float Lz = (float)J.dims[2];
        const float inv2Lz = 1.f / (2.f * Lz);
        unsigned long long my_contrib = 0, my_taps = 0;

        // ---- flush: records for s_cand[0..nc), then taps
        auto flush = [&](int nc) {
            __syncthreads();
            // records are written at their candidate slot; only the indices
            // of the valid ones are compacted (block scan, fixed order)
            unsigned vmask = 0;
            const int c0 = tid * CPT;
#pragma unroll 1
            for (int t = 0; t < CPT; ++t) {
                const int ci = c0 + t;
                if (ci >= nc) break;
                const uint32_t cd = s_cand[ci];
                const int ix = cd & 1023, iy = (cd >> 10) & 1023, iz = cd >> 20;
                int k;
                float f, d;
                delay_split<KIND>(T, TE, ix, iy, iz, qh, ql, q, k, f, d);
                const int kb = (KIND == ISM_FD_HANN_SINC) ? k - H : k - (P - 1) / 2;
                if (kb < kb_lo || kb > kb_hi) continue;
                const float a = T.g[ix] * T.g[TE + iy] * T.g[2 * TE + iz] *
                                __frcp_rn(12.566370614359172f * d);
                float4 v;
                if (KIND == ISM_FD_HANN_SINC) {
                    if (fabsf(f) < 1e-30f) {
                        v = make_float4(a, 0.f, 0.f, 0.f);
                    } else {
                        float sp, cp, sw, cw;
                        sincospif(f, &sp, &cp);
                        sincospif(f / (float)(H + 1), &sw, &cw);
                        const float A = -a * sp * 0.15915494309189535f;
                        v = make_float4(A, A * cw, A * sw, f);
                    }
                } else {
                    v = make_float4(a, f + (float)((P - 1) / 2), 0.f, 0.f);
                }
                s_reck[ci] = kb;
                s_rec4[ci] = v;
                vmask |= 1u << t;
                // statistics: taps in [w0, w0+W) n [0, Lh); an image counts
                // as contributing in the window of its first in-range tap.
                const long long lo = max((long long)kb, max((long long)w0, 0ll));
                const long long hi = min((long long)kb + n_taps, min((long long)w0 + W, Lh));
                if (hi > lo) my_taps += (unsigned long long)(hi - lo);
                const long long first = max((long long)kb, 0ll);
                if (first < min((long long)kb + n_taps, Lh) && first >= w0 &&
                    first < (long long)w0 + W)
                    ++my_contrib;
            }
            int nrec;
            int o = block_scan(__popc(vmask), s_scan, nrec);
            while (vmask) {
                const int t = __ffs(vmask) - 1;
                vmask &= vmask - 1;
                s_idx[o++] = (uint16_t)(c0 + t);
            }
            __syncthreads();
            // taps: warp per image, lane per tap, private row per warp
            float *rowp = s_rows + warp * RL + lane;
            for (int i = warp; i < nrec; i += NW) {
                const int ri = s_idx[i];
                const int kb = s_reck[ri];
                const float4 v = s_rec4[ri];
                // row index of tap index n is n - w0 + HALO, in [0, RL)
                float *p = rowp + (kb - w0 + HALO);
                if (KIND == ISM_FD_HANN_SINC) {
                    if (v.w == 0.f) {
                        if (lane == 0) p[H] += v.x;
                        continue;
                    }
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (cOK[r]) {
                            const float xs = fmaf(cMS[r], v.w, cSJ[r]);
                            const float rcp = rcp_approx(xs);
                            const float nn = fmaf(cC[r], v.y, fmaf(cS[r], v.z, v.x));
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
                                if (i2 != j) prod *= (v.y - (float)i2);
                            p[32 * r] = fmaf(v.x, prod, p[32 * r]);
                        }
                    }
                }
            }
            __syncthreads();
        };

        // ---- column sweep: candidates per (u,l,v,m,w) column
        int n_cand = 0;  // block-uniform
        for (long long cb = 0; cb < n_cols; cb += NT) {
            const long long c = cb + tid;
            int lo_a = 1, hi_a = 0, lo_b = 1, hi_b = 0, ix = 0, iy = 0, wz = 0;
            if (c < n_cols) {
                wz = (int)(c & 1);
                const long long t = c >> 1;
                ix = s_lx[(int)(t / nLY)];
                iy = s_ly[(int)(t % nLY)];
                const float dx = T.dl[ix], dy = T.dl[TE + iy];
                const float rho2 = dx * dx + dy * dy;
                if (rho2 <= dhe2) {
                    // Delta_z(n) = cz + 2 Lz n must satisfy zmin <= |Delta_z| <= zmax:
                    // the full range [-zmax, zmax] minus the open hole (-zmin, zmin).
                    const float zmax = sqrtf(fmaxf(dhi2 - rho2, 0.f)) + eps;
                    const float zmin2 = dlo2 - rho2;
                    const float zmin = zmin2 > 0.f ? sqrtf(zmin2) - eps : 0.f;
                    const float cz = T.dl[2 * TE + wz * (2 * N + 1) + N];
                    const float lim = (float)N + 1.f;
                    const float u_lo = fminf(fmaxf((-zmax - cz) * inv2Lz, -lim), lim);
                    const float u_hi = fminf(fmaxf((zmax - cz) * inv2Lz, -lim), lim);
                    int n_lo = (int)ceilf(u_lo);
                    int n_hi = (int)floorf(u_hi);
                    if (n_lo < -N) n_lo = -N;
                    if (n_hi > N) n_hi = N;
                    int h_lo = 1, h_hi = 0;  // hole (excluded n), empty by default
                    if (zmin > 0.f) {
                        const float v_lo = fminf(fmaxf((-zmin - cz) * inv2Lz, -lim), lim);
                        const float v_hi = fminf(fmaxf((zmin - cz) * inv2Lz, -lim), lim);
                        h_lo = (int)floorf(v_lo) + 1;
                        h_hi = (int)ceilf(v_hi) - 1;
                    }
                    if (h_lo <= h_hi) {
                        lo_a = n_lo;
                        hi_a = n_hi < h_lo - 1 ? n_hi : h_lo - 1;
                        lo_b = n_lo > h_hi + 1 ? n_lo : h_hi + 1;
                        hi_b = n_hi;
                    } else {
                        lo_a = n_lo;
                        hi_a = n_hi;
                    }
                }
            }
            const int cnt = max(hi_a - lo_a + 1, 0) + max(hi_b - lo_b + 1, 0);
            int total;
            const int off = block_scan(cnt, s_scan, total);
            if (total == 0) continue;
            if (n_cand + total > CAP && n_cand > 0) {
                flush(n_cand);
                n_cand = 0;
            }
            const int zb = wz * (2 * N + 1) + N;
            const uint32_t base_code = (uint32_t)ix | ((uint32_t)iy << 10);
            // write candidates with global index in [g_lo, g_hi) at dst + idx
            auto emit = [&](int g_lo, int g_hi, int dst) {
                int gi = off;
                for (int n = lo_a; n <= hi_a; ++n, ++gi)
                    if (gi >= g_lo && gi < g_hi)
                        s_cand[dst + gi] = base_code | ((uint32_t)(zb + n) << 20);
                for (int n = lo_b; n <= hi_b; ++n, ++gi)
                    if (gi >= g_lo && gi < g_hi)
                        s_cand[dst + gi] = base_code | ((uint32_t)(zb + n) << 20);
            };
            if (total <= CAP) {
                emit(0, total, n_cand);
                n_cand += total;
            } else {
                for (int pb = 0; pb < total; pb += CAP) {
                    emit(pb, pb + CAP, -pb);
                    flush(min(CAP, total - pb));
                }
            }
        }
        if (n_cand > 0) flush(n_cand);

        // ---- window output: fixed-order sum of the private rows
        __syncthreads();
        float *hout = h + J.h_offset;
        for (int i = tid; i < W; i += NT) {
            const long long n = (long long)w0 + i;
            float acc = 0.f;
#pragma unroll
            for (int wv = 0; wv < NW; ++wv) acc += s_rows[wv * RL + HALO + i];
            if (n < Lh) hout[n] = acc;
        }
        __syncthreads();
        for (int i = tid; i < NW * RL; i += NT) s_rows[i] = 0.f;
        if (stats) {
            atomicAdd(&s_stat[0], my_contrib);
            atomicAdd(&s_stat[1], my_taps);
            __syncthreads();
            if (tid == 0) {
                const long long si = J.stat_index;
                atomicAdd((unsigned long long *)&stats[2 * si], s_stat[0]);
                atomicAdd((unsigned long long *)&stats[2 * si + 1], s_stat[1]);
            }
        }
        __syncthreads();
    }
}

template <int R, int KIND>
int launch_t(const RirLaunch &L, cudaStream_t stream) {
    const Layout Lay = make_layout(L.window, L.max_order, L.max_taps);
    auto kern = k_ism_taps<R, KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Lay.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_ism_taps)");
    int grid = L.grid;
    if (grid <= 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, Lay.total);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy(k_ism_taps)");
        grid = device_sm_count() * (per_sm > 0 ? per_sm : 1);
    }
    const long long items = (long long)L.n_rirs * L.wmax;
    if ((long long)grid > items) grid = (int)items;
    if (grid < 1) return ISM_OK;
    kern<<<grid, NT, Lay.total, stream>>>(L.jobs_dev, L.n_rirs, L.wmax, L.window, L.max_order,
                                          L.max_taps, L.h_dev, L.stats_dev, L.counter_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_ism_taps");
    return ISM_OK;
}

}  // namespace

size_t rir_smem_bytes(int window, int max_order, int max_taps) {
    return make_layout(window, max_order, max_taps).total;
}

int launch_rir(const RirLaunch &L, cudaStream_t stream) {
    if (L.fd_kind == ISM_FD_LAGRANGE) return launch_t<1, ISM_FD_LAGRANGE>(L, stream);
    const int rows = (L.max_taps + 31) / 32;
    switch (rows) {
        case 1: return launch_t<1, ISM_FD_HANN_SINC>(L, stream);
        case 2: return launch_t<2, ISM_FD_HANN_SINC>(L, stream);
        case 3: return launch_t<3, ISM_FD_HANN_SINC>(L, stream);
        case 4: return launch_t<4, ISM_FD_HANN_SINC>(L, stream);
        case 5: return launch_t<5, ISM_FD_HANN_SINC>(L, stream);
        case 6: return launch_t<6, ISM_FD_HANN_SINC>(L, stream);
        case 7: return launch_t<7, ISM_FD_HANN_SINC>(L, stream);
        case 8: return launch_t<8, ISM_FD_HANN_SINC>(L, stream);
        default: return fail(ISM_ERR_INVALID_ARG, "n_taps above 255 is not supported");
    }
}

}  // namespace ism
