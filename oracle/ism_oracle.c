/*
 * ism_oracle.c -- plain FP64 CPU oracle for the shoebox image-source RIR path
 * and the multichannel convolution that follows it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only tests/, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it computes (arXiv 2104.13347, Sec. II.A, "Synthetic and experimental
 * datasets generation"): room impulse responses built from every image source
 * of a shoebox room (Allen--Berkley image method), each image contributing a
 * fractionally delayed tap group whose gain is the product of the wall
 * reflection factors it met and the spherical spreading 1/(4 pi d); then the
 * batch convolution of source signals with those RIRs, plus the additive
 * Gaussian noise at a drawn SNR used as data augmentation (Sec. III.A).
 *
 * Everything is written as the plain definition, in FP64, in the order the
 * definition states it, with no blocking, tables or algebraic shortcuts:
 *
 *   image (u,v,w,l,m,n), u,v,w in {0,1}, l,m,n in [-N, N]      (Sec. II.A)
 *     dx = ((1-2u) xs + (2l) Lx) - xr      (same for y, z)
 *     d  = sqrt((dx*dx + dy*dy) + dz*dz)   (left to right, no FMA)
 *     tau = d * (fs / c),  k0 = rint(tau) (ties to even),  f = tau - k0
 *     a  = bx0^|l-u| bx1^|l| by0^|m-v| by1^|m| bz0^|n-w| bz1^|n| / (4 pi d)
 *   Hann-windowed sinc taps, j = -H..H, t = j - f:
 *     h[k0+j] += a * sinc(t) * 0.5 (1 + cos(pi t / (H+1))),  sinc(0) = 1
 *   Lagrange taps (the paper's own 7th-order filter, 8 coefficients):
 *     P = n_taps - 1 (odd), k1 = floor(tau) - (P-1)/2, D = tau - k1,
 *     h[k1+j] += a * prod_{i != j} (D - i) / (j - i),  j = 0..P
 *   convolution: y[t] = sum_k h[k] s[t-k],  t in [0, Ts + Lh - 1)
 *   noise: y += sigma z, sigma^2 = mean(y^2 over the room's mics and
 *     samples) / 10^(snr/10); z from SplitMix64 counters and Box--Muller
 *     (one counter output per pair of samples, both branches).
 *
 * Readings of what the paper leaves open (Hann window width and centring, the
 * rounding rule of the delay split, the wall-coefficient convention, the SNR
 * definition) are the ones listed in the project's design notes.  This file
 * must be compiled with -ffp-contract=off so that the FP64 distance and delay
 * arithmetic rounds exactly as written above.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

enum { ORACLE_FD_HANN_SINC = 0, ORACLE_FD_LAGRANGE = 1 };

/* ------------------------------------------------------------------------ */
/* Per-image quantities (Sec. II.A: image positions, delay, wall dampings).  */
/* ------------------------------------------------------------------------ */

/* Offset between image and microphone along one axis:
 * image coordinate (1-2p) s + 2 q L, minus the microphone coordinate. */
static double axis_offset(int p, int q, double s, double L, double r)
{
    double img = (p ? -s : s) + (double)(2 * q) * L;
    return img - r;
}

/* Wall damping along one axis: beta0^|q-p| * beta1^|q| (0^0 = 1). */
static double axis_damping(int p, int q, double beta0, double beta1)
{
    return pow(beta0, (double)abs(q - p)) * pow(beta1, (double)abs(q));
}

typedef struct {
    double d, tau, f, amp;
    int64_t k0;
} image_t;

static image_t image_eval(const double *dims, const double *beta, const double *src,
                          const double *mic, double q, int u, int v, int w, int l, int m, int n)
{
    image_t im;
    double dx = axis_offset(u, l, src[0], dims[0], mic[0]);
    double dy = axis_offset(v, m, src[1], dims[1], mic[1]);
    double dz = axis_offset(w, n, src[2], dims[2], mic[2]);
    double d2 = dx * dx + dy * dy;
    d2 = d2 + dz * dz;
    im.d = sqrt(d2);
    im.tau = im.d * q;
    double k = rint(im.tau);
    im.k0 = (int64_t)k;
    im.f = im.tau - k;
    double g = axis_damping(u, l, beta[0], beta[1]) * axis_damping(v, m, beta[2], beta[3]) *
               axis_damping(w, n, beta[4], beta[5]);
    im.amp = g / (4.0 * ORACLE_PI * im.d);
    return im;
}

/* ------------------------------------------------------------------------ */
/* Fractional-delay filters.                                                 */
/* ------------------------------------------------------------------------ */

/* sin(pi t) through the identity sin(pi t) = (-1)^k sin(pi (t - k)),
 * k = rint(t), which is exactly zero at integer t. */
static double sin_pi(double t)
{
    double k = rint(t);
    double s = sin(ORACLE_PI * (t - k));
    return fmod(k, 2.0) == 0.0 ? s : -s;
}

/* Hann-windowed sinc tap for the continuous offset t = j - f. */
static double hann_sinc(double t, int H)
{
    double s = (t == 0.0) ? 1.0 : sin_pi(t) / (ORACLE_PI * t);
    double win = 0.5 * (1.0 + cos(ORACLE_PI * t / (double)(H + 1)));
    return s * win;
}

/* Lagrange interpolation coefficient j of order P at delay D. */
static double lagrange_coef(int j, int P, double D)
{
    double c = 1.0;
    for (int i = 0; i <= P; ++i) {
        if (i == j) continue;
        c *= (D - (double)i) / (double)(j - i);
    }
    return c;
}

/* Taps of one fractional delay (exported for the filter pins). */
void oracle_hann_sinc_taps(double f, int n_taps, double *out)
{
    int H = (n_taps - 1) / 2;
    for (int j = -H; j <= H; ++j) out[j + H] = hann_sinc((double)j - f, H);
}

void oracle_lagrange_taps(double D, int n_taps, double *out)
{
    int P = n_taps - 1;
    for (int j = 0; j <= P; ++j) out[j] = lagrange_coef(j, P, D);
}

/* ------------------------------------------------------------------------ */
/* One RIR: direct sum over every image of the (2N+1)^3 x 8 lattice.        */
/* ------------------------------------------------------------------------ */

/* Lattice order of the delay-limited image set (Sec. II.A keeps every
 * reflection that arrives within the reverberation time, i.e. within the
 * response): the smallest N whose cubic lattice holds every image able to
 * put a tap into [0, Lh).  The first tap of an image with delay tau lies at
 * or after tau - n_taps, so no image farther than
 * d_reach = (Lh + n_taps) c / fs reaches the response; along axis a the
 * image offset (1-2p) s + 2 q L - r is within d_reach only for
 * |q| <= (d_reach + |(1-2p) s - r|) / (2 L). */
int oracle_auto_order(const double *dims, const double *src, const double *mic, double fs,
                      double c, int n_taps, int64_t rir_len)
{
    const double d_reach = ((double)rir_len + (double)n_taps) * c / fs;
    int N = 0;
    for (int a = 0; a < 3; ++a)
        for (int p = 0; p <= 1; ++p) {
            const double cp = (p ? -src[a] : src[a]) - mic[a];
            const int na = (int)floor((d_reach + fabs(cp)) / (2.0 * dims[a]));
            if (na > N) N = na;
        }
    return N;
}

/* stats[0] = images enumerated, stats[1] = images with at least one tap in
 * [0, Lh), stats[2] = taps that landed in [0, Lh).  order < 0: the
 * delay-limited lattice of oracle_auto_order. */
int oracle_rir(const double *dims, const double *beta, const double *src, const double *mic,
               double fs, double c, int order, int n_taps, int fd_kind, int64_t rir_len,
               double *h, int64_t *stats)
{
    const double q = fs / c;
    const int N = order < 0 ? oracle_auto_order(dims, src, mic, fs, c, n_taps, rir_len) : order;
    int64_t n_img = 0, n_contrib = 0, n_in = 0;
    for (int64_t i = 0; i < rir_len; ++i) h[i] = 0.0;

    for (int u = 0; u <= 1; ++u)
    for (int v = 0; v <= 1; ++v)
    for (int w = 0; w <= 1; ++w)
    for (int l = -N; l <= N; ++l)
    for (int m = -N; m <= N; ++m)
    for (int n = -N; n <= N; ++n) {
        image_t im = image_eval(dims, beta, src, mic, q, u, v, w, l, m, n);
        ++n_img;
        int64_t taps_here = 0;
        if (fd_kind == ORACLE_FD_HANN_SINC) {
            int H = (n_taps - 1) / 2;
            for (int j = -H; j <= H; ++j) {
                int64_t idx = im.k0 + j;
                if (idx < 0 || idx >= rir_len) continue;
                h[idx] += im.amp * hann_sinc((double)j - im.f, H);
                ++taps_here;
            }
        } else {
            int P = n_taps - 1;
            double fl = floor(im.tau);
            int64_t k1 = (int64_t)fl - (P - 1) / 2;
            double D = im.tau - (double)k1;
            for (int j = 0; j <= P; ++j) {
                int64_t idx = k1 + j;
                if (idx < 0 || idx >= rir_len) continue;
                h[idx] += im.amp * lagrange_coef(j, P, D);
                ++taps_here;
            }
        }
        if (taps_here) ++n_contrib;
        n_in += taps_here;
    }
    if (stats) {
        stats[0] = n_img;
        stats[1] = n_contrib;
        stats[2] = n_in;
    }
    return 0;
}

/* Every image of the lattice, in (u,v,w,l,m,n) lexicographic order.
 * idx6: 6 ints per image (u,v,w,l,m,n); dtf: d, tau, f, amp per image;
 * k0: the integer part of the delay split.  Returns the image count. */
int64_t oracle_images(const double *dims, const double *beta, const double *src, const double *mic,
                      double fs, double c, int order, int32_t *idx6, double *dtfa, int64_t *k0)
{
    const double q = fs / c;
    const int N = order;
    int64_t i = 0;
    for (int u = 0; u <= 1; ++u)
    for (int v = 0; v <= 1; ++v)
    for (int w = 0; w <= 1; ++w)
    for (int l = -N; l <= N; ++l)
    for (int m = -N; m <= N; ++m)
    for (int n = -N; n <= N; ++n) {
        image_t im = image_eval(dims, beta, src, mic, q, u, v, w, l, m, n);
        if (idx6) {
            int32_t *p = idx6 + 6 * i;
            p[0] = u; p[1] = v; p[2] = w; p[3] = l; p[4] = m; p[5] = n;
        }
        if (dtfa) {
            double *p = dtfa + 4 * i;
            p[0] = im.d; p[1] = im.tau; p[2] = im.f; p[3] = im.amp;
        }
        if (k0) k0[i] = im.k0;
        ++i;
    }
    return i;
}

/* Batch of RIRs: rir j belongs to room room_of[j] and uses mic mics[3j..].
 * Room parameters are packed 15 doubles per room:
 *   dims[3], beta[6], src[3], fs, c, (unused)
 * and 4 ints per room: order, n_taps, fd_kind, (unused); rir_len per room.
 * Output j starts at h + h_off[j].  OpenMP over RIRs. */
int oracle_rir_batch(int64_t n_rirs, const int32_t *room_of, const double *room_f,
                     const int32_t *room_i, const int64_t *room_len, const double *mics,
                     double *h, const int64_t *h_off, int64_t *stats, int n_threads)
{
#ifdef _OPENMP
    /* a num_threads clause, not omp_set_num_threads: a one-thread call must
     * not lower the thread count of later calls in the process */
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
    for (int64_t j = 0; j < n_rirs; ++j) {
        int r = room_of[j];
        const double *rf = room_f + 15 * (int64_t)r;
        const int32_t *ri = room_i + 4 * (int64_t)r;
        oracle_rir(rf, rf + 3, rf + 9, mics + 3 * j, rf[12], rf[13], ri[0], ri[1], ri[2],
                   room_len[r], h + h_off[j], stats ? stats + 3 * j : NULL);
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Convolution (Sec. II.A: batch convolution of RIRs with source signals).   */
/* ------------------------------------------------------------------------ */

/* Full linear convolution, y has Ts + Lh - 1 samples. */
void oracle_convolve(const double *h, int64_t Lh, const double *s, int64_t Ts, double *y)
{
    int64_t Ty = Ts + Lh - 1;
    for (int64_t t = 0; t < Ty; ++t) {
        int64_t k_lo = t - (Ts - 1);
        if (k_lo < 0) k_lo = 0;
        int64_t k_hi = t < Lh - 1 ? t : Lh - 1;
        double acc = 0.0;
        for (int64_t k = k_lo; k <= k_hi; ++k) acc += h[k] * s[t - k];
        y[t] = acc;
    }
}

/* Selected outputs y[ts[i]] of the same convolution. */
void oracle_convolve_at(const double *h, int64_t Lh, const double *s, int64_t Ts,
                        const int64_t *ts, int64_t n, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t t = ts[i];
        int64_t k_lo = t - (Ts - 1);
        if (k_lo < 0) k_lo = 0;
        int64_t k_hi = t < Lh - 1 ? t : Lh - 1;
        double acc = 0.0;
        for (int64_t k = k_lo; k <= k_hi; ++k) acc += h[k] * s[t - k];
        y[i] = acc;
    }
}

/* Batch: convolution j uses h + h_off[j] (length h_len[j]) and the source of
 * its room, s + s_off[room_of[j]] (length s_len[room_of[j]]). */
void oracle_convolve_batch(int64_t n_conv, const int32_t *room_of, const double *h,
                           const int64_t *h_off, const int64_t *h_len, const double *s,
                           const int64_t *s_off, const int64_t *s_len, double *y,
                           const int64_t *y_off, int n_threads)
{
#ifdef _OPENMP
    const int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
#endif
    for (int64_t j = 0; j < n_conv; ++j) {
        int r = room_of[j];
        oracle_convolve(h + h_off[j], h_len[j], s + s_off[r], s_len[r], y + y_off[j]);
    }
}

/* ------------------------------------------------------------------------ */
/* Noise (Sec. III.A: Gaussian noise at a drawn SNR).                        */
/* SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): the i-th output of the    */
/* stream with state x is mix(x + (i+1) * gamma).                            */
/* ------------------------------------------------------------------------ */

static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t state, uint64_t i)
{
    return sm_mix(state + (i + 1) * SM_GAMMA);
}

/* Key of the (room, mic) noise stream: output number room*65536 + mic of the
 * stream seeded with `seed`. */
static uint64_t noise_key(uint64_t seed, uint64_t room, uint64_t mic)
{
    return oracle_splitmix64(seed, room * 65536ULL + mic);
}

/* Standard normal number t of stream (room, mic).  Samples come in pairs
 * (2k, 2k+1) sharing output k of the stream: u1 = (bits 63..40 + 1/2) / 2^24,
 * u2 = (bits 39..16) / 2^24, and Box--Muller gives the pair's two
 * independent normals, r cos(2 pi u2) for the even sample and r sin(2 pi u2)
 * for the odd one, r = sqrt(-2 ln u1). */
double oracle_gauss(uint64_t seed, uint64_t room, uint64_t mic, uint64_t t)
{
    uint64_t key = noise_key(seed, room, mic);
    uint64_t b = oracle_splitmix64(key, t >> 1);
    double u1 = ((double)(b >> 40) + 0.5) * (1.0 / 16777216.0);
    double u2 = (double)((b >> 16) & 0xFFFFFFULL) * (1.0 / 16777216.0);
    double r = sqrt(-2.0 * log(u1));
    return (t & 1) ? r * sin(2.0 * ORACLE_PI * u2) : r * cos(2.0 * ORACLE_PI * u2);
}

/* The uniforms of pairs k0 .. k0+n-1 of stream (room, mic). */
void oracle_uniforms(uint64_t seed, uint64_t room, uint64_t mic, uint64_t k0, int64_t n,
                     double *u1, double *u2)
{
    uint64_t key = noise_key(seed, room, mic);
    for (int64_t i = 0; i < n; ++i) {
        uint64_t b = oracle_splitmix64(key, k0 + (uint64_t)i);
        u1[i] = ((double)(b >> 40) + 0.5) * (1.0 / 16777216.0);
        u2[i] = (double)((b >> 16) & 0xFFFFFFULL) * (1.0 / 16777216.0);
    }
}

/* One training frame (Sec. II.B: the network reads multichannel windows of
 * the convolved signals; Sec. III.A: measurement noise at a drawn SNR):
 *   x[m][i] = y[m][t0 + i], 0 outside [0, y_len),  i < frame_len,
 *   sigma^2 = mean of x^2 over the frame / 10^(snr/10),
 *   out[m][i] = x[m][i] + sigma z, z = oracle_gauss(seed, id, m, i).
 * snr_db NaN or +inf: a clean copy.  y: n_mics rows of y_len; out: n_mics
 * rows of frame_len.  Returns sigma (0 for a clean copy). */
double oracle_frame(const double *y, int n_mics, int64_t y_len, int64_t t0, int frame_len,
                    double snr_db, uint64_t seed, uint64_t id, double *out)
{
    for (int m = 0; m < n_mics; ++m)
        for (int i = 0; i < frame_len; ++i) {
            int64_t t = t0 + i;
            out[(int64_t)m * frame_len + i] = (t >= 0 && t < y_len) ? y[(int64_t)m * y_len + t] : 0.0;
        }
    if (isnan(snr_db) || isinf(snr_db)) return 0.0;
    double p = 0.0;
    for (int64_t e = 0; e < (int64_t)n_mics * frame_len; ++e) p += out[e] * out[e];
    p /= (double)n_mics * (double)frame_len;
    double sigma = sqrt(p / pow(10.0, snr_db / 10.0));
    for (int m = 0; m < n_mics; ++m)
        for (int i = 0; i < frame_len; ++i)
            out[(int64_t)m * frame_len + i] += sigma * oracle_gauss(seed, id, (uint64_t)m, (uint64_t)i);
    return sigma;
}

/* Adds noise in place to one room's signals y[mic][0..T) (mic-major,
 * stride T).  Returns sigma. */
double oracle_add_noise(double *y, int n_mics, int64_t T, double snr_db, uint64_t seed,
                        uint64_t room)
{
    double p = 0.0;
    for (int m = 0; m < n_mics; ++m)
        for (int64_t t = 0; t < T; ++t) p += y[m * T + t] * y[m * T + t];
    p /= (double)n_mics * (double)T;
    double sigma = sqrt(p / pow(10.0, snr_db / 10.0));
    for (int m = 0; m < n_mics; ++m)
        for (int64_t t = 0; t < T; ++t)
            y[m * T + t] += sigma * oracle_gauss(seed, room, (uint64_t)m, (uint64_t)t);
    return sigma;
}
