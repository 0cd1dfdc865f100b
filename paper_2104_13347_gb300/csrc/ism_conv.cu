// ism_conv.cu -- K2b (FP32 direct convolution) and the noise epilogue.
//
// Convolution (arXiv 2104.13347, Sec. II.A: the dataset is built by batch
// convolutions of the RIRs with source signals): for every mic m of a room,
//   y_m[t] = sum_k h_m[k] s[t - k],  t in [0, Ts + Lh - 1).
// Noise (Sec. III.A: Gaussian noise at a drawn SNR):
//   y_m[t] += sigma z,  sigma^2 = mean(y^2 over the room's mics and samples)
//   / 10^(snr/10), z from SplitMix64 counters and Box--Muller (one counter
//   output per pair of samples, both branches).  The sums of
//   y^2 come from the convolution kernels' epilogues, one partial per tile
//   (float-float per thread, FP64 across threads, fixed order).
//
// K2b layout: one CTA per (room, group of 8 mics, tile of 2048 outputs);
// each thread owns 8 consecutive outputs of all 8 mics (64 accumulators),
// the source window and 8 RIR chunks are staged in shared memory, and the
// tap loop runs 8 taps at a time from 16 source values held in registers,
// so the inner loop is FFMAs fed by broadcast / 128-bit shared loads.  RIR
// chunks whose products all hit zero source samples are skipped.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ism_internal.h"

namespace ism {
namespace {

constexpr int CT = 256;          // threads per CTA
constexpr int OPT = 8;           // outputs per thread
constexpr int TT = CT * OPT;     // outputs per tile (2048)
constexpr int MG = 8;            // mics per CTA
constexpr int KC = 256;          // taps per shared-memory chunk
static_assert(TT == kConvTT && MG == kConvMG, "tile shape of the noise partials");

using Tile = ConvTile;

__global__ void __launch_bounds__(CT, 2)
k_conv_f32(const ConvJob *__restrict__ jobs, const Tile *__restrict__ tiles,
           const float *__restrict__ h, const float *__restrict__ src, float *__restrict__ y,
           double *__restrict__ part) {
    __shared__ __align__(16) float s_src[TT + KC + 16];
    __shared__ __align__(16) float s_h[MG][KC];
    const Tile tl = tiles[blockIdx.x];
    const ConvJob J = jobs[tl.job];
    const int tid = threadIdx.x;
    const int64_t t0 = tl.t0;
    const int64_t Lh = J.rir_len, Ts = J.src_len;
    const int nm = min(MG, J.n_mics - tl.mic0);
    const float *hb = h + J.h_offset + (int64_t)tl.mic0 * Lh;
    const float *sb = src + J.src_offset;

    float acc[MG][OPT];
#pragma unroll
    for (int m = 0; m < MG; ++m)
#pragma unroll
        for (int i = 0; i < OPT; ++i) acc[m][i] = 0.f;

    for (int64_t k0 = 0; k0 < Lh; k0 += KC) {
        // source indices used by this chunk: t - k for t in [t0, t0+TT),
        // k in [k0, k0+KC)
        const int64_t lo = t0 - k0 - KC + 1, hi = t0 + TT - 1 - k0;
        if (hi < 0 || lo >= Ts) continue;  // all products vanish
        __syncthreads();
        // s_src[i] = s[t0 - k0 - KC + i - 8 + 8] for i in [0, TT + KC + 16):
        // index i holds s[t0 - k0 - KC - 8 + i]
        for (int i = tid; i < TT + KC + 16; i += CT) {
            const int64_t g = t0 - k0 - KC - 8 + i;
            s_src[i] = (g >= 0 && g < Ts) ? sb[g] : 0.f;
        }
        for (int i = tid; i < MG * KC; i += CT) {
            const int m = i / KC, kk = i - m * KC;
            const int64_t k = k0 + kk;
            s_h[m][kk] = (m < nm && k < Lh) ? hb[(int64_t)m * Lh + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 1
        for (int kk = 0; kk < KC; kk += 8) {
            // output t0 + 8 tid + i, tap k0 + kk + jj needs
            // s[t0 + 8 tid + i - k0 - kk - jj] = s_src[8 tid + i - kk - jj + KC + 8]
            const int base = 8 * tid - kk + KC + 8;  // multiple of 8
            float sv[16];
            const float4 *p4 = reinterpret_cast<const float4 *>(s_src + base - 8);
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float4 q = p4[v];
                sv[4 * v] = q.x; sv[4 * v + 1] = q.y; sv[4 * v + 2] = q.z; sv[4 * v + 3] = q.w;
            }
            // sv[x] = s_src[base - 8 + x]; value for (i, jj) is sv[8 + i - jj]
#pragma unroll
            for (int m = 0; m < MG; ++m) {
                const float4 ha = *reinterpret_cast<const float4 *>(&s_h[m][kk]);
                const float4 hb4 = *reinterpret_cast<const float4 *>(&s_h[m][kk + 4]);
                const float hv[8] = {ha.x, ha.y, ha.z, ha.w, hb4.x, hb4.y, hb4.z, hb4.w};
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
#pragma unroll
                    for (int i = 0; i < OPT; ++i) acc[m][i] = fmaf(hv[jj], sv[8 + i - jj], acc[m][i]);
            }
        }
    }
    const int64_t ylen = J.y_len;
    float *yb = y + J.y_offset + (int64_t)tl.mic0 * ylen;
    float ss = 0.f, se = 0.f;  // float-float sum of y^2 (noise partial)
#pragma unroll
    for (int m = 0; m < MG; ++m) {
        if (m < nm) {
#pragma unroll
            for (int i = 0; i < OPT; ++i) {
                const int64_t t = t0 + 8 * tid + i;
                if (t < ylen) {
                    const float v = acc[m][i];
                    yb[(int64_t)m * ylen + t] = v;
                    ff_accumulate_sq(v, ss, se);
                }
            }
        }
    }
    if (part) {  // uniform: noise partial of this tile, fixed order
        __shared__ double s_red[CT / 32];
        const double r = warp_sum_f64((double)ss + (double)se);
        if ((tid & 31) == 0) s_red[tid >> 5] = r;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < CT / 32; ++w) t += s_red[w];
            const int s0 = conv_partial_slot(tl.mic0, t0, ylen);
            if (ISM_IN_RANGE(s0 >= 0 && s0 < conv_partials_per_job(J.n_mics, ylen), kOobConvF32))
                part[J.part_offset + s0] = t;
        }
    }
}

// Noise: sigma from the job's tile partials (fixed order), then
// y += sigma * z.  The samples of a (room, mic) stream come in pairs
// (2k, 2k+1) that share SplitMix64 output k: u1 = (bits 63..40 + 1/2) / 2^24,
// u2 = (bits 39..16) / 2^24, r = sqrt(-2 ln u1), and the pair gets
// r cos(2 pi u2) and r sin(2 pi u2) (both Box--Muller branches).  Block x of
// job y covers pair indices [x NCH, (x+1) NCH) of the job's (mic, pair)
// sequence; each thread walks its pairs with stride 256, carrying (mic, k)
// and the pair's SplitMix64 input.  The pair math is box_muller().
constexpr int NCH = 32768;  // pairs per block
__global__ void __launch_bounds__(256)
k_noise(const ConvJob *__restrict__ jobs, float *__restrict__ y, const double *__restrict__ part,
        uint64_t seed) {
    const ConvJob J = jobs[blockIdx.y];
    if (isnan(J.snr_db)) return;
    const int64_t ylen = J.y_len;
    const int64_t npr = (ylen + 1) >> 1;              // pairs per mic
    const int64_t n = (int64_t)J.n_mics * npr;
    const int64_t b = (int64_t)blockIdx.x * NCH;
    if (b >= n) return;
    __shared__ float s_sigma;
    if (threadIdx.x == 0) {
        const int np = conv_partials_per_job(J.n_mics, ylen);
        double p = 0.0;
        for (int i = 0; i < np; ++i) p += part[J.part_offset + i];
        p /= (double)J.n_mics * (double)ylen;
        s_sigma = (float)sqrt(p / pow(10.0, (double)J.snr_db / 10.0));
    }
    __syncthreads();
    const float sigma = s_sigma;
    float *yb = y + J.y_offset;
    const int64_t e = min(b + NCH, n);
    int64_t i = b + threadIdx.x;
    if (i >= e) return;
    uint64_t m = (uint64_t)(i / npr);
    int64_t k = i - (int64_t)m * npr;
    // SplitMix64 input of pair k of mic m: key(m) + (k + 1) gamma, advanced
    // by 256 gamma per pair of this thread (recomputed when k wraps)
    uint64_t zs = sm64_out(seed, J.noise_id * 65536ull + m) + ((uint64_t)k + 1) * kSm64Gamma;
    constexpr uint64_t kStep = 256ull * kSm64Gamma;
    // U pairs per round: their loads are all issued before any is used, so
    // each thread keeps U read-modify-writes in flight
    constexpr int U = 4;
    while (i < e) {
        float *ptr[U];
        float v0[U], v1[U];
        uint64_t zz[U];
        bool ok[U], ok1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            ok[u] = i < e;
            ok1[u] = ok[u] && 2 * k + 1 < ylen;
            zz[u] = zs;
            ptr[u] = yb + (int64_t)m * ylen + 2 * k;
            v0[u] = ok[u] ? ptr[u][0] : 0.f;
            v1[u] = ok1[u] ? ptr[u][1] : 0.f;
            i += 256;
            k += 256;
            zs += kStep;
            if (k >= npr) {
                while (k >= npr) { k -= npr; ++m; }
                zs = sm64_out(seed, J.noise_id * 65536ull + m) + ((uint64_t)k + 1) * kSm64Gamma;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!ok[u]) continue;
            float z0, z1;
            box_muller(sm64_mix(zz[u]), sigma, z0, z1);
            ptr[u][0] = v0[u] + z0;
            if (ok1[u]) ptr[u][1] = v1[u] + z1;
        }
    }
}

}  // namespace

ISM_OOB_READER(conv)

int conv_f32_plan(const ConvLaunch &L, ConvPlan *P) {
    P->precision = ISM_F32;
    P->tiles.clear();
    for (int j = 0; j < L.n_jobs; ++j) {
        const ConvJob &J = L.jobs_host[j];
        for (int m0 = 0; m0 < J.n_mics; m0 += MG)
            for (int64_t t0 = 0; t0 < J.y_len; t0 += TT) P->tiles.push_back(Tile{j, m0, t0});
    }
    if (P->tiles.size() > 0x7fffffffULL) return fail(ISM_ERR_INVALID_ARG, "too many tiles");
    return ISM_OK;
}

int conv_f32_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                     cudaStream_t stream) {
    if (P.tiles.empty()) return ISM_OK;
    k_conv_f32<<<(unsigned)P.tiles.size(), CT, 0, stream>>>(
        L.jobs_dev, d_tiles, L.h_dev, L.src_dev, L.y_dev, L.noise_partials_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_conv_f32");
    return ISM_OK;
}

int launch_conv_f32(const ConvLaunch &L, cudaStream_t stream) {
    ConvPlan P;
    if (int st = conv_f32_plan(L, &P)) return st;
    if (P.tiles.empty()) return ISM_OK;
    void *d_tiles = nullptr;
    int st = scratch_alloc(&d_tiles, P.tiles.size() * sizeof(Tile), stream);
    if (st) return st;
    st = upload_async(d_tiles, P.tiles.data(), P.tiles.size() * sizeof(Tile), stream);
    if (!st) st = conv_f32_enqueue(L, P, (const Tile *)d_tiles, stream);
    scratch_free(d_tiles, stream);
    return st;
}

int launch_noise(const ConvLaunch &L, cudaStream_t stream) {
    if (!L.any_noise || L.n_jobs == 0) return ISM_OK;
    int64_t max_n = 0;  // pairs of the largest job
    for (int j = 0; j < L.n_jobs; ++j)
        max_n = std::max(max_n, (int64_t)L.jobs_host[j].n_mics * ((L.jobs_host[j].y_len + 1) / 2));
    const int64_t nb = (max_n + NCH - 1) / NCH;
    if (nb > 0x7fffffff) return fail(ISM_ERR_INVALID_ARG, "job too large for the noise grid");
    if (L.n_jobs > 65535) {
        // grid.y limit: one launch per group of 65535 jobs
        for (int j0 = 0; j0 < L.n_jobs; j0 += 65535) {
            const int nj = std::min(65535, L.n_jobs - j0);
            k_noise<<<dim3((unsigned)nb, nj), 256, 0, stream>>>(L.jobs_dev + j0, L.y_dev,
                                                               L.noise_partials_dev, L.seed);
        }
    } else {
        k_noise<<<dim3((unsigned)nb, L.n_jobs), 256, 0, stream>>>(L.jobs_dev, L.y_dev,
                                                                 L.noise_partials_dev, L.seed);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "launch k_noise");
    return ISM_OK;
}

int conv_plan(const ConvLaunch &L, ConvPlan *P) {
    return L.precision == ISM_BF16X3 ? conv_bf16x3_plan(L, P) : conv_f32_plan(L, P);
}

int conv_enqueue(const ConvLaunch &L, const ConvPlan &P, const ConvTile *d_tiles,
                 cudaStream_t stream) {
    return P.precision == ISM_BF16X3 ? conv_bf16x3_enqueue(L, P, d_tiles, stream)
                                     : conv_f32_enqueue(L, P, d_tiles, stream);
}

}  // namespace ism
