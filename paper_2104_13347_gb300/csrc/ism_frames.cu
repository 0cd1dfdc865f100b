// ism_frames.cu -- training frames cut from the convolved signals, with
// measurement noise at a per-frame SNR.
//
// The network of arXiv 2104.13347 reads multichannel windows of 1024
// samples (Sec. II.B: 23.2 ms at 44.1 kHz) and is trained with Gaussian
// measurement noise added at a drawn SNR (Sec. III.A).  For frame f:
//   x_m[i] = y_m[t0 + i] (0 outside [0, y_len)),  i < frame_len,
//   sigma^2 = mean over m, i of x_m[i]^2 / 10^(snr/10),
//   out_m[i] = x_m[i] + sigma z_m[i],
// z from SplitMix64 counters (key out(seed, noise_id * 65536 + m); samples
// 2k, 2k+1 share output k: two 24-bit uniforms, both Box--Muller branches),
// the same recipe as the convolution's noise.
//
// One CTA per frame.  The frame's power is a float-float sum per thread and
// an FP64 sum across threads in a fixed order, so results are bitwise
// reproducible; the second pass re-reads the frame (L1/L2-resident) and
// writes it.  HBM work: one read and one write of the frame; the noise
// generator's integer instructions set the pace.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ism_internal.h"

namespace ism {
namespace {

constexpr int FT = 256;  // threads per CTA

struct FrameJob {
    int64_t y_offset, y_len, t0, out_offset;
    uint64_t noise_id;
    int32_t n_mics;
    float snr_db;
};
static_assert(sizeof(FrameJob) == 48, "FrameJob layout");

// INSIDE: the frame lies within the signal ([t0, t0 + frame_len) inside
// [0, y_len)), so no sample needs a range check.
template <bool INSIDE>
__device__ __forceinline__ void frame_body(const FrameJob &J, int frame_len,
                                           const float *__restrict__ y, float *__restrict__ out,
                                           uint64_t seed) {
    const float *yb = y + J.y_offset;
    float *ob = out + J.out_offset;
    const int tid = threadIdx.x;
    const bool noisy = !isnan(J.snr_db) && !isinf(J.snr_db);
    float sigma = 0.f;
    if (noisy) {
        // 10^(snr/10) for thread 0, begun before the loads it waits behind
        const double den = tid == 0 ? pow(10.0, (double)J.snr_db / 10.0) : 1.0;
        float ss = 0.f, se = 0.f;
        for (int m = 0; m < J.n_mics; ++m) {
            const float *ym = yb + (int64_t)m * J.y_len;
#pragma unroll 4
            for (int i = tid; i < frame_len; i += FT) {
                const int64_t t = J.t0 + i;
                const float v = (INSIDE || (t >= 0 && t < J.y_len)) ? ym[t] : 0.f;
                ff_accumulate_sq(v, ss, se);
            }
        }
        __shared__ double s_red[FT / 32];
        __shared__ float s_sigma;
        const double r = warp_sum_f64((double)ss + (double)se);
        if ((tid & 31) == 0) s_red[tid >> 5] = r;
        __syncthreads();
        if (tid == 0) {
            double p = 0.0;
            for (int w = 0; w < FT / 32; ++w) p += s_red[w];
            p /= (double)J.n_mics * (double)frame_len;
            s_sigma = (float)sqrt(p / den);
        }
        __syncthreads();
        sigma = s_sigma;
    }
    for (int m = 0; m < J.n_mics; ++m) {
        const float *ym = yb + (int64_t)m * J.y_len;
        float *om = ob + (int64_t)m * frame_len;
        // samples 2k, 2k+1 of the frame share counter output k, whose
        // SplitMix64 input key(m) + (k + 1) gamma advances by FT gamma per step
        uint64_t zs = noisy ? sm64_out(seed, J.noise_id * 65536ull + (uint64_t)m) +
                                  ((uint64_t)tid + 1) * kSm64Gamma
                            : 0ull;
        for (int k = tid; 2 * k < frame_len; k += FT, zs += (uint64_t)FT * kSm64Gamma) {
            const int i = 2 * k;
            const int64_t t = J.t0 + i;
            float v0 = (INSIDE || (t >= 0 && t < J.y_len)) ? ym[t] : 0.f;
            float v1 = (INSIDE ? i + 1 < frame_len : (t + 1 >= 0 && t + 1 < J.y_len)) ? ym[t + 1]
                                                                                      : 0.f;
            if (noisy) {
                float z0, z1;
                box_muller(sm64_mix(zs), sigma, z0, z1);
                v0 += z0;
                v1 += z1;
            }
            om[i] = v0;
            if (i + 1 < frame_len) om[i + 1] = v1;
        }
    }
}

__global__ void __launch_bounds__(FT)
k_frames(const FrameJob *__restrict__ jobs, int frame_len, const float *__restrict__ y,
         float *__restrict__ out, uint64_t seed) {
    const FrameJob J = jobs[blockIdx.x];
    if (J.t0 >= 0 && J.t0 + frame_len <= J.y_len)
        frame_body<true>(J, frame_len, y, out, seed);
    else
        frame_body<false>(J, frame_len, y, out, seed);
}

}  // namespace
}  // namespace ism

using namespace ism;

extern "C" int ism_frames_batch(const ism_frame_job *jobs, int64_t n_frames, int32_t frame_len,
                                const float *y_dev, float *frames_dev, uint64_t seed,
                                void *stream_v) {
    set_error("");
    if (n_frames < 0) return fail(ISM_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return ISM_OK;
    if (!jobs || !y_dev || !frames_dev) return fail(ISM_ERR_INVALID_ARG, "NULL pointer");
    if (frame_len < 1) return fail(ISM_ERR_INVALID_ARG, "frame_len < 1");
    if (n_frames > 0x7fffffff) return fail(ISM_ERR_INVALID_ARG, "too many frames");
    std::vector<FrameJob> fj((size_t)n_frames);
    for (int64_t i = 0; i < n_frames; ++i) {
        const ism_frame_job &J = jobs[i];
        if (J.n_mics < 1 || J.n_mics > kMaxMics || J.y_len < 1 || J.y_len > kMaxSignal ||
            J.y_offset < 0 || J.out_offset < 0)
            return fail(ISM_ERR_INVALID_ARG, "frame " + std::to_string(i) + ": bad sizes/offsets");
        if (isinf(J.snr_db) && J.snr_db < 0)
            return fail(ISM_ERR_INVALID_ARG, "frame " + std::to_string(i) + ": snr -inf");
        FrameJob &f = fj[(size_t)i];
        f.y_offset = J.y_offset;
        f.y_len = J.y_len;
        f.t0 = J.t0;
        f.out_offset = J.out_offset;
        f.noise_id = J.noise_id;
        f.n_mics = J.n_mics;
        f.snr_db = J.snr_db;
    }
    cudaStream_t stream = (cudaStream_t)stream_v;
    const size_t bytes = fj.size() * sizeof(FrameJob);
    void *scr = nullptr;
    if (int st = scratch_alloc(&scr, bytes, stream)) return st;
    int st = upload_async(scr, fj.data(), bytes, stream);
    if (!st) {
        k_frames<<<(unsigned)n_frames, FT, 0, stream>>>((const FrameJob *)scr, frame_len, y_dev,
                                                        frames_dev, seed);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "launch k_frames");
    }
    scratch_free(scr, stream);
    return st;
}
