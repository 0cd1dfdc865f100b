// ism_api.cu -- C ABI entry points: validation, job tables, scratch and
// staging, and dispatch to the kernels (see include/ism.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "ism_internal.h"

namespace ism {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }
int fail(int status, const std::string &msg) {
    g_err = msg;
    return status;
}
int cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return ISM_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// device info, scratch pool, pinned staging
// ---------------------------------------------------------------------------
namespace {
constexpr int kMaxDev = 64;
std::mutex g_mu;
int g_sms[kMaxDev];
cudaMemPool_t g_pool[kMaxDev];
bool g_pool_ok[kMaxDev];

struct Stage {
    int dev;
    void *ptr;
    size_t size;
    cudaEvent_t ev;
    bool used;
};
std::vector<Stage> g_stage;

int cur_device(int *d) {
    cudaError_t e = cudaGetDevice(d);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (*d < 0 || *d >= kMaxDev) return fail(ISM_ERR_INTERNAL, "device ordinal out of range");
    return ISM_OK;
}
}  // namespace

int device_sm_count() {
    int d = 0;
    if (cur_device(&d)) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_sms[d]) cudaDeviceGetAttribute(&g_sms[d], cudaDevAttrMultiProcessorCount, d);
    return g_sms[d] > 0 ? g_sms[d] : 1;
}

int scratch_alloc(void **p, size_t bytes, cudaStream_t stream) {
    int d = 0;
    if (int st = cur_device(&d)) return st;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_pool_ok[d]) {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = d;
            cudaError_t e = cudaMemPoolCreate(&g_pool[d], &props);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(g_pool[d], cudaMemPoolAttrReleaseThreshold, &thr);
            g_pool_ok[d] = true;
        }
        pool = g_pool[d];
    }
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, stream);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(ISM_ERR_OUT_OF_MEMORY, "device scratch allocation failed");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaMallocFromPoolAsync");
    return ISM_OK;
}

void scratch_free(void *p, cudaStream_t stream) {
    if (p) cudaFreeAsync(p, stream);
}

int upload_async(void *dev_dst, const void *host_src, size_t bytes, cudaStream_t stream) {
    if (bytes == 0) return ISM_OK;
    int d = 0;
    if (int st = cur_device(&d)) return st;
    std::lock_guard<std::mutex> lk(g_mu);
    Stage *slot = nullptr;
    for (auto &s : g_stage) {
        if (s.dev != d || s.size < bytes) continue;
        if (s.used && cudaEventQuery(s.ev) != cudaSuccess) continue;
        slot = &s;
        break;
    }
    if (!slot) {
        Stage s{d, nullptr, std::max<size_t>(bytes, 1 << 16), nullptr, false};
        cudaError_t e = cudaHostAlloc(&s.ptr, s.size, cudaHostAllocDefault);
        if (e != cudaSuccess) return cuda_fail(e, "cudaHostAlloc(staging)");
        e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaFreeHost(s.ptr);
            return cuda_fail(e, "cudaEventCreate(staging)");
        }
        g_stage.push_back(s);
        slot = &g_stage.back();
    }
    cudaGetLastError();  // clear a not-ready status left by the queries
    memcpy(slot->ptr, host_src, bytes);
    cudaError_t e = cudaMemcpyAsync(dev_dst, slot->ptr, bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(upload)");
    e = cudaEventRecord(slot->ev, stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(staging)");
    slot->used = true;
    return ISM_OK;
}

// ---------------------------------------------------------------------------
// validation
// ---------------------------------------------------------------------------
static bool inside(const double *p, const double *dims) {
    for (int a = 0; a < 3; ++a)
        if (!(p[a] > 0.0 && p[a] < dims[a])) return false;
    return true;
}

int validate_room(const ism_room &r, int64_t idx) {
    auto bad = [&](const std::string &why) {
        return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(idx) + ": " + why);
    };
    for (int a = 0; a < 3; ++a)
        if (!(r.dims[a] > 0.0) || !isfinite(r.dims[a])) return bad("dims must be finite and > 0");
    for (int w = 0; w < 6; ++w)
        if (!(r.beta[w] >= 0.0 && r.beta[w] <= 1.0)) return bad("beta must lie in [0, 1]");
    if (!inside(r.src, r.dims)) return bad("source not strictly inside the room");
    if (r.n_mics < 1 || r.n_mics > kMaxMics) return bad("n_mics must lie in [1, 65536]");
    if (!r.mics) return bad("mics is NULL");
    for (int m = 0; m < r.n_mics; ++m) {
        const double *p = r.mics + 3 * m;
        if (!inside(p, r.dims)) return bad("mic " + std::to_string(m) + " not strictly inside");
        const double dx = p[0] - r.src[0], dy = p[1] - r.src[1], dz = p[2] - r.src[2];
        if (dx * dx + dy * dy + dz * dz < 1e-12) return bad("mic coincides with the source");
    }
    if (!(r.fs > 0.0) || !isfinite(r.fs)) return bad("fs must be > 0");
    if (!(r.c > 0.0) || !isfinite(r.c)) return bad("c must be > 0");
    if (r.rir_len < 1 || r.rir_len > (int64_t)1 << 30) return bad("rir_len must lie in [1, 2^30]");
    if (r.fd_kind == ISM_FD_HANN_SINC) {
        if (r.n_taps < 1 || r.n_taps % 2 == 0 || r.n_taps > 255)
            return bad("Hann-sinc n_taps must be odd and in [1, 255]");
    } else if (r.fd_kind == ISM_FD_LAGRANGE) {
        if (r.n_taps < 2 || r.n_taps % 2 != 0 || r.n_taps > 32)
            return bad("Lagrange n_taps must be even and in [2, 32]");
    } else {
        return bad("unknown fd_kind");
    }
    int order = r.order;
    for (int m = 0; m < r.n_mics; ++m) order = std::max(order, room_order(r, m));
    if (order > 200)
        return bad(r.order < 0 ? "the delay-limited lattice needs an order above 200"
                               : "order must lie in [0, 200] (or ISM_ORDER_AUTO)");
    // largest delay must stay representable in the FP32 integer part
    double reach = 0.0;
    for (int a = 0; a < 3; ++a) reach += pow((2.0 * order + 1.0) * r.dims[a] * 2.0, 2.0);
    if (sqrt(reach) * r.fs / r.c > 8.0e6) return bad("lattice delays exceed 8e6 samples");
    return ISM_OK;
}

// Output window per work item when the caller leaves it to the library:
// 1024 samples, halved (down to 64) while the call has fewer than four work
// items per SM.  A single 4096-sample RIR then runs as 64 items instead of 4
// (latency-bound calls: 38 us instead of 85 us per call on GB300), while
// batches with enough RIRs keep the 1024 that serves them best.  Below 64 an
// image's taps would straddle three windows and be summed in each.
int auto_window(const ism_room *rooms, int64_t n_rooms) {
    const int64_t target = 4 * (int64_t)device_sm_count();
    int W = 1024;
    while (W > 64) {
        int64_t items = 0;
        for (int64_t r = 0; r < n_rooms && items < target; ++r)
            items += (int64_t)rooms[r].n_mics * ((rooms[r].rir_len + W - 1) / W);
        if (items >= target) break;
        W /= 2;
    }
    return W;
}

// Lattice order of RIR (room r, mic m): the room's order, or for
// ISM_ORDER_AUTO the smallest N whose lattice holds every image able to put
// a tap into [0, rir_len): the first tap of an image at delay tau is at or
// after tau - n_taps, so only images within reach = (rir_len + n_taps) c/fs
// matter, and along axis a the offset (1-2p) s + 2 q L - r stays within
// reach only for |q| <= (reach + |(1-2p) s - r|) / (2 L).
int room_order(const ism_room &r, int m) {
    if (r.order >= 0) return r.order;
    const double reach = ((double)r.rir_len + (double)r.n_taps) * r.c / r.fs;
    const double *mic = r.mics + 3 * m;
    int n = 0;
    for (int a = 0; a < 3; ++a) {
        const double e = std::max(fabs(r.src[a] - mic[a]), fabs(-r.src[a] - mic[a]));
        const double na = floor((reach + e) / (2.0 * r.dims[a]));
        n = std::max(n, na > 1e6 ? 1000000 : (int)na);
    }
    return n;
}

// ---------------------------------------------------------------------------
// Sorted column lists of one sparse launch at most this many entries (4 B
// each): a batch whose lists would need more runs as several launches.
constexpr long long kColBudget = 1ll << 28;

// Chebyshev tables of the fractional-delay filters (FP64, cached)
// ---------------------------------------------------------------------------
namespace {
constexpr double kPi = 3.14159265358979323846;

// Hann-windowed sinc tap at continuous offset t (the filter's definition).
double hann_sinc_tap(double t, int H) {
    const double s = (t == 0.0) ? 1.0 : sin(kPi * t) / (kPi * t);
    return s * 0.5 * (1.0 + cos(kPi * t / (double)(H + 1)));
}

// Lagrange coefficient j of order P at delay D.
double lagrange_tap(int j, int P, double D) {
    double c = 1.0;
    for (int i = 0; i <= P; ++i)
        if (i != j) c *= (D - (double)i) / (double)(j - i);
    return c;
}

// Truncation of the Chebyshev expansion: the largest tail a tap may lose,
// relative to the peak tap.  Hann sinc: 1e-6, which keeps 8 terms for 81
// taps (tail 7.7e-7; 9 terms would leave 3.3e-8): the truncation adds about
// 1.2e-6 rel-L2 to a RIR, under the 1e-5 bar, for one sparse-array atomic
// and 81 FIR multiply-adds fewer per image and output (K1 -7 % on GB300).
// Lagrange: 5e-8, below FP32 resolution, so that the P + 1 terms of an
// order-P filter -- exact, its taps being degree-P polynomials in the
// delay -- are all kept.
constexpr double kChebTailHann = 1e-6;
constexpr double kChebTailLagrange = 5e-8;

ChebTable build_cheb(int kind, int n_taps) {
    // Chebyshev interpolation at M first-kind nodes: each tap, as a function
    // of x in [-1, 1], is sampled at x_k = cos(pi (k + 1/2) / M) and
    // c_p = (2/M) sum_k g(x_k) T_p(x_k) (c_0 halved).  Terms are kept while
    // the largest remaining tail, over all taps, exceeds the filter's
    // truncation (above) of the peak tap (about 1).
    const int M = 64;
    std::vector<double> c((size_t)M * n_taps);
    std::vector<double> vals(M);
    for (int j = 0; j < n_taps; ++j) {
        for (int k = 0; k < M; ++k) {
            const double x = cos(kPi * (k + 0.5) / M);
            if (kind == ISM_FD_HANN_SINC) {
                const int H = (n_taps - 1) / 2;
                vals[k] = hann_sinc_tap((double)(j - H) - 0.5 * x, H);
            } else {
                const int P = n_taps - 1;
                vals[k] = lagrange_tap(j, P, 0.5 * (P - 1) + 0.5 * (x + 1.0));
            }
        }
        for (int p = 0; p < M; ++p) {
            double acc = 0.0;
            for (int k = 0; k < M; ++k) acc += vals[k] * cos(p * kPi * (k + 0.5) / M);
            c[(size_t)p * n_taps + j] = (p == 0 ? 1.0 : 2.0) * acc / M;
        }
    }
    ChebTable t;
    t.n_cheb = 0;
    for (int P = 1; P <= kMaxCheb; ++P) {
        double worst = 0.0;
        for (int j = 0; j < n_taps; ++j) {
            double tail = 0.0;
            for (int p = P; p < M; ++p) tail += fabs(c[(size_t)p * n_taps + j]);
            worst = std::max(worst, tail);
        }
        if (worst <= (kind == ISM_FD_HANN_SINC ? kChebTailHann : kChebTailLagrange)) {
            t.n_cheb = P;
            break;
        }
    }
    if (t.n_cheb) {
        t.coef.resize((size_t)t.n_cheb * n_taps);
        for (size_t i = 0; i < t.coef.size(); ++i) t.coef[i] = (float)c[i];
    }
    return t;
}

std::mutex g_cheb_mu;
std::vector<std::pair<std::pair<int, int>, ChebTable *>> g_cheb;
}  // namespace

const ChebTable &cheb_table(int fd_kind, int n_taps) {
    std::lock_guard<std::mutex> lk(g_cheb_mu);
    for (auto &e : g_cheb)
        if (e.first.first == fd_kind && e.first.second == n_taps) return *e.second;
    ChebTable *t = new ChebTable(build_cheb(fd_kind, n_taps));
    g_cheb.push_back({{fd_kind, n_taps}, t});
    return *t;
}

// ---------------------------------------------------------------------------
// K1 calls: host preparation and launches
// ---------------------------------------------------------------------------
int rir_prepare(const ism_room *rooms, int64_t n_rooms, const int64_t *h_offsets,
                const ism_rir_opts &o, int W, const int *order_caps, RirPrep *out) {
    RirPrep &P = *out;
    P.W = W;
    // jobs, one per RIR; grouped by filter kind (one launch per group)
    std::vector<int64_t> room_of[kRirGroups];
    int64_t j = 0, packed = 0;
    for (int g = 0; g < kRirGroups; ++g) {
        P.k[g] = RirKindPrep();
        P.k[g].kind = g == 1 ? ISM_FD_LAGRANGE : ISM_FD_HANN_SINC;
    }
    for (int64_t r = 0; r < n_rooms; ++r) {
        const ism_room &R = rooms[r];
        const int kind = R.fd_kind;
        for (int m = 0; m < R.n_mics; ++m, ++j) {
            // a Hann-sinc RIR that ends before its direct arrival holds only
            // filter tails: the direct per-tap kernel (group 2)
            int grp = kind;
            if (kind == ISM_FD_HANN_SINC && o.variant == ISM_RIR_SPARSE) {
                double d2 = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double dd = R.src[a] - R.mics[3 * m + a];
                    d2 += dd * dd;
                }
                if (rint(sqrt(d2) * (R.fs / R.c)) >= (double)R.rir_len) grp = 2;
            }
            RirKindPrep &K = P.k[grp];
            RirJob J;
            memset(&J, 0, sizeof(J));
            for (int a = 0; a < 3; ++a) {
                J.src[a] = R.src[a];
                J.mic[a] = R.mics[3 * m + a];
                J.dims[a] = R.dims[a];
            }
            J.q = R.fs / R.c;
            for (int w = 0; w < 6; ++w) J.beta[w] = (float)R.beta[w];
            J.order = room_order(R, m);
            J.n_taps = R.n_taps;
            J.fd_kind = (int16_t)kind;
            J.rir_len = R.rir_len;
            J.n_windows = (int32_t)((R.rir_len + W - 1) / W);
            J.h_offset = h_offsets ? h_offsets[j] : packed;
            J.stat_index = (int32_t)j;  // statistics slot: RIR index in the caller's order
            packed += R.rir_len;
            if (J.h_offset < 0) return fail(ISM_ERR_INVALID_ARG, "negative h offset");
            const int cap = order_caps ? order_caps[j] : J.order;
            if (J.order > cap)
                return fail(ISM_ERR_INVALID_ARG, "RIR " + std::to_string(j) +
                                                     ": lattice order above the plan's capacity");
            K.jobs.push_back(J);
            K.caps.push_back(cap);
            room_of[grp].push_back(r);
            K.max_order = std::max(K.max_order, cap);
            K.max_taps = std::max(K.max_taps, R.n_taps);
            K.min_taps = std::min(K.min_taps, R.n_taps);
            K.wmax = std::max(K.wmax, J.n_windows);
        }
    }
    if (j > 0x3fffffff) return fail(ISM_ERR_INVALID_ARG, "too many RIRs");

    for (int grp = 0; grp < kRirGroups; ++grp) {
        RirKindPrep &K = P.k[grp];
        const int kind = K.kind;
        auto &jv = K.jobs;
        if (jv.empty()) continue;
        // sparse path: one Chebyshev table per distinct filter length
        K.sparse = o.variant == ISM_RIR_SPARSE && grp != 2;
        K.max_cheb = 0;
        K.min_cheb = kMaxCheb;
        if (K.sparse) {
            std::vector<std::pair<int, int>> seen;  // (n_taps, offset)
            for (auto &J : jv) {
                int off = -1;
                for (auto &pr : seen)
                    if (pr.first == J.n_taps) off = pr.second;
                const ChebTable &ct = cheb_table(kind, J.n_taps);
                if (ct.n_cheb == 0) { K.sparse = false; break; }
                if (off < 0) {
                    // rows padded with zeros to a multiple of 4 taps (the
                    // kernel reads them as 16-byte vectors)
                    off = (int)K.tabs.size();
                    const int tp = (J.n_taps + 3) & ~3;
                    K.tabs.resize(K.tabs.size() + (size_t)ct.n_cheb * tp, 0.f);
                    for (int p = 0; p < ct.n_cheb; ++p)
                        for (int jj = 0; jj < J.n_taps; ++jj)
                            K.tabs[off + (size_t)p * tp + jj] = ct.coef[(size_t)p * J.n_taps + jj];
                    seen.push_back({J.n_taps, off});
                }
                J.tab_offset = off;
                J.n_cheb = (int16_t)ct.n_cheb;
                K.max_cheb = std::max(K.max_cheb, ct.n_cheb);
                K.min_cheb = std::min(K.min_cheb, ct.n_cheb);
            }
            if (K.sparse && rir_sparse_smem_bytes(W, K.max_order, K.max_taps, K.max_cheb) >
                                kMaxDynSmem)
                K.sparse = false;
            if (!K.sparse) {
                K.tabs.clear();
                K.max_cheb = 0;
                K.min_cheb = kMaxCheb;
            }
        }
        if (!K.sparse && rir_smem_bytes(W, K.max_order, K.max_taps) > kMaxDynSmem)
            return fail(ISM_ERR_INVALID_ARG, "window/order/taps need too much shared memory");
        // launches: one per room on the unbatched path; otherwise the whole
        // kind, cut where the sparse kernel's sorted column lists would pass
        // kColBudget entries
        {
            size_t b = 0;
            long long acc = 0;
            for (size_t k = 0; k < jv.size(); ++k) {
                const long long ce = K.sparse ? rir_col_entries(K.caps[k]) : 0;
                const bool cut = o.per_room ? room_of[grp][k] != room_of[grp][b]
                                            : (k > b && acc + ce > kColBudget);
                if (cut) {
                    K.chunks.push_back({b, k});
                    b = k;
                    acc = 0;
                }
                acc += ce;
            }
            K.chunks.push_back({b, jv.size()});
        }
        // per RIR: column-list and window-range offsets, relative to its
        // launch; the lists are sized for the RIR's order capacity
        long long max_cols = 0, max_wins = 0;
        if (K.sparse) {
            K.offs.resize(2 * jv.size());
            for (auto &c : K.chunks) {
                long long co = 0, wo = 0;
                for (size_t k = c.first; k < c.second; ++k) {
                    K.offs[2 * k] = co;
                    K.offs[2 * k + 1] = wo;
                    co += rir_col_entries(K.caps[k]);
                    wo += jv[k].n_windows;
                }
                max_cols = std::max(max_cols, co);
                max_wins = std::max(max_wins, wo);
            }
        }
        size_t max_chunk = 0;
        for (auto &c : K.chunks) max_chunk = std::max(max_chunk, c.second - c.first);
        auto al = [](size_t n) { return (n + 255) & ~(size_t)255; };
        K.jb = al(jv.size() * sizeof(RirJob));
        K.tb = al(K.sparse ? K.tabs.size() * sizeof(float) : 0);
        K.ob = al(K.offs.size() * sizeof(long long));
        K.up_bytes = K.jb + 256 + K.tb + K.ob;
        K.cb = al((size_t)max_cols * sizeof(uint32_t));
        K.wb = al((size_t)max_wins * sizeof(int2));
        K.gb = K.sparse ? al(rir_tables_bytes((long long)max_chunk, K.max_order)) : 0;
        K.blob.assign(K.up_bytes, 0);
        memcpy(K.blob.data(), jv.data(), jv.size() * sizeof(RirJob));
        if (K.sparse) {
            memcpy(K.blob.data() + K.jb + 256, K.tabs.data(), K.tabs.size() * sizeof(float));
            memcpy(K.blob.data() + K.jb + 256 + K.tb, K.offs.data(),
                   K.offs.size() * sizeof(long long));
        }
    }
    return ISM_OK;
}

int rir_enqueue(const RirKindPrep &K, char *sp, int W, float *h_dev, long long *stats,
                int *err_dev, cudaStream_t stream) {
    (void)err_dev;  // the image-source kernels have no waits
    RirJob *d_jobs = (RirJob *)sp;
    unsigned int *d_counter = (unsigned int *)(sp + K.jb);
    const float *d_tabs = (const float *)(sp + K.jb + 256);
    long long *d_offs = (long long *)(sp + K.jb + 256 + K.tb);
    uint32_t *d_cols = (uint32_t *)(sp + K.up_bytes);
    int2 *d_wr = (int2 *)(sp + K.up_bytes + K.cb);
    void *d_tables = K.sparse ? (void *)(sp + K.up_bytes + K.cb + K.wb) : nullptr;
    int st = ISM_OK;
    for (size_t ci = 0; !st && ci < K.chunks.size(); ++ci) {
        const size_t b = K.chunks[ci].first, n = K.chunks[ci].second - b;
        int wm = 0;
        for (size_t k = b; k < b + n; ++k) wm = std::max(wm, K.jobs[k].n_windows);
        if (ci > 0) {
            cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned int), stream);
            if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counter)");
        }
        RirLaunch L{d_jobs + b, (int)n, wm, W, K.max_order, K.max_taps, K.kind, h_dev,
                    stats, d_counter, nullptr, 0, d_tabs, K.max_cheb, K.min_cheb, K.min_taps};
        if (K.sparse) {
            L.cols_dev = d_cols;
            L.wr_dev = d_wr;
            L.offs_dev = d_offs + 2 * b;
            L.tables_dev = d_tables;
        }
        st = K.sparse ? launch_rir_sparse(L, stream) : launch_rir(L, stream);
    }
    return st;
}

}  // namespace ism

using namespace ism;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *ism_last_error_string(void) { return g_err.c_str(); }

const char *ism_version(void) { return "ism-gb300 0.1 (sm_103a)"; }

int ism_rir_batch_size(const ism_room *rooms, int64_t n_rooms, int64_t *n_rirs, int64_t *h_len) {
    if (n_rooms < 0 || (n_rooms > 0 && !rooms)) return fail(ISM_ERR_INVALID_ARG, "bad rooms");
    int64_t nr = 0, hl = 0;
    for (int64_t i = 0; i < n_rooms; ++i) {
        if (rooms[i].n_mics < 1 || rooms[i].rir_len < 1)
            return fail(ISM_ERR_INVALID_ARG, "room " + std::to_string(i) + ": bad size");
        nr += rooms[i].n_mics;
        hl += (int64_t)rooms[i].n_mics * rooms[i].rir_len;
    }
    if (n_rirs) *n_rirs = nr;
    if (h_len) *h_len = hl;
    return ISM_OK;
}

int ism_rir_batch_ex(const ism_room *rooms, int64_t n_rooms, float *h_dev,
                     const int64_t *h_offsets, const ism_rir_opts *opts, void *stream_v) {
    set_error("");
    if (n_rooms < 0) return fail(ISM_ERR_INVALID_ARG, "n_rooms < 0");
    if (n_rooms == 0) return ISM_OK;
    if (!rooms || !h_dev) return fail(ISM_ERR_INVALID_ARG, "NULL rooms or h_dev");
    cudaStream_t stream = (cudaStream_t)stream_v;
    ism_rir_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.window != 0 && o.window != ISM_WINDOW_TUNE &&
        (o.window % 32 != 0 || o.window < 32 || o.window > 8192))
        return fail(ISM_ERR_INVALID_ARG,
                    "window must be a multiple of 32 in [32, 8192], 0 or ISM_WINDOW_TUNE");
    if (o.variant != ISM_RIR_SPARSE && o.variant != ISM_RIR_DIRECT)
        return fail(ISM_ERR_INVALID_ARG, "unknown variant");
    if (o.per_room && o.window == ISM_WINDOW_TUNE)
        return fail(ISM_ERR_INVALID_ARG, "ISM_WINDOW_TUNE is for batched launches");
    for (int64_t r = 0; r < n_rooms; ++r)
        if (int st = validate_room(rooms[r], r)) return st;
    if (o.window == ISM_WINDOW_TUNE) return rir_batch_tuned(rooms, n_rooms, h_dev, h_offsets, o, stream);
    const int W = o.window > 0 ? o.window : auto_window(rooms, n_rooms);
    RirPrep P;
    {
        NvtxRange r("ism.rir.plan");
        if (int st = rir_prepare(rooms, n_rooms, h_offsets, o, W, nullptr, &P)) return st;
    }
    NvtxRange r("ism.rir.K1");
    for (int grp = 0; grp < kRirGroups; ++grp) {
        const RirKindPrep &K = P.k[grp];
        if (K.jobs.empty()) continue;
        // one scratch block and one upload: [jobs | counter | filter tables |
        // offsets] copied from the host, then the column lists, window
        // ranges and per-RIR tables the kernels fill
        void *scr = nullptr;
        if (int st = scratch_alloc(&scr, K.total(), stream)) return st;
        int st = upload_async(scr, K.blob.data(), K.up_bytes, stream);  // counter uploaded as 0
        if (!st) st = rir_enqueue(K, (char *)scr, W, h_dev, (long long *)o.stats_dev, nullptr, stream);
        scratch_free(scr, stream);
        if (st) return st;
    }
    return ISM_OK;
}

int ism_rir_filter_terms(int32_t fd_kind, int32_t n_taps, int32_t *n_terms) {
    set_error("");
    if (!n_terms) return fail(ISM_ERR_INVALID_ARG, "NULL n_terms");
    if (fd_kind == ISM_FD_HANN_SINC) {
        if (n_taps < 1 || n_taps % 2 == 0 || n_taps > 255)
            return fail(ISM_ERR_INVALID_ARG, "Hann-sinc n_taps must be odd and in [1, 255]");
    } else if (fd_kind == ISM_FD_LAGRANGE) {
        if (n_taps < 2 || n_taps % 2 != 0 || n_taps > 32)
            return fail(ISM_ERR_INVALID_ARG, "Lagrange n_taps must be even and in [2, 32]");
    } else {
        return fail(ISM_ERR_INVALID_ARG, "unknown fd_kind");
    }
    *n_terms = cheb_table(fd_kind, n_taps).n_cheb;
    return ISM_OK;
}

int ism_rir_batch(const ism_room *rooms, int64_t n_rooms, float *h_dev, const int64_t *h_offsets,
                  void *stream) {
    return ism_rir_batch_ex(rooms, n_rooms, h_dev, h_offsets, nullptr, stream);
}

int ism_convolve_batch(const ism_conv_job *jobs, int64_t n_jobs, const float *h_dev,
                       const float *src_dev, float *y_dev, uint64_t seed, int32_t precision,
                       void *stream_v) {
    return ism::convolve_batch(jobs, n_jobs, h_dev, src_dev, y_dev, seed, precision, stream_v);
}

}  // extern "C"

int ism::convolve_batch(const ism_conv_job *jobs, int64_t n_jobs, const float *h_dev,
                        const float *src_dev, float *y_dev, uint64_t seed, int32_t precision,
                        void *stream_v) {
    set_error("");
    if (n_jobs < 0) return fail(ISM_ERR_INVALID_ARG, "n_jobs < 0");
    if (n_jobs == 0) return ISM_OK;
    if (!jobs || !h_dev || !src_dev || !y_dev) return fail(ISM_ERR_INVALID_ARG, "NULL pointer");
    if (precision != ISM_F32 && precision != ISM_BF16X3)
        return fail(ISM_ERR_INVALID_ARG, "unknown precision");
    if (n_jobs > 0x7fffffff) return fail(ISM_ERR_INVALID_ARG, "too many jobs");
    cudaStream_t stream = (cudaStream_t)stream_v;
    NvtxRange nr("ism.conv");
    std::vector<ConvJob> cj(n_jobs);
    bool any_noise = false;
    int64_t n_part = 0;
    for (int64_t i = 0; i < n_jobs; ++i) {
        const ism_conv_job &J = jobs[i];
        if (J.n_mics < 1 || J.n_mics > kMaxMics || J.rir_len < 1 || J.rir_len > kMaxSignal ||
            J.src_len < 1 || J.src_len > kMaxSignal || J.h_offset < 0 || J.src_offset < 0 ||
            J.y_offset < 0)
            return fail(ISM_ERR_INVALID_ARG, "job " + std::to_string(i) + ": bad sizes/offsets");
        ConvJob &c = cj[i];
        memset(&c, 0, sizeof(c));
        c.rir_len = J.rir_len;
        c.src_len = J.src_len;
        c.h_offset = J.h_offset;
        c.src_offset = J.src_offset;
        c.y_offset = J.y_offset;
        c.y_len = J.src_len + J.rir_len - 1;
        c.noise_id = J.noise_id;
        c.n_mics = J.n_mics;
        c.snr_db = J.snr_db;
        if (!isnan(J.snr_db)) {
            if (!isfinite(J.snr_db))
                return fail(ISM_ERR_INVALID_ARG, "job " + std::to_string(i) + ": snr must be finite or NaN");
            any_noise = true;
        }
        const int64_t nt = (c.y_len + kConvTT - 1) / kConvTT;
        if ((J.n_mics + (int64_t)kConvMG - 1) / kConvMG * nt > 0x3fffffff)
            return fail(ISM_ERR_INVALID_ARG, "job " + std::to_string(i) + ": too many tiles");
        c.part_offset = n_part;
        n_part += conv_partials_per_job(J.n_mics, c.y_len);
    }
    // a kernel of an earlier call on this stream reported an error
    if (int st = status_collect(stream, false)) return st;
    const size_t jb = cj.size() * sizeof(ConvJob);
    const size_t pb = any_noise ? (size_t)n_part * sizeof(double) : 0;
    void *scr = nullptr;
    if (int st = scratch_alloc(&scr, jb + 256 + pb, stream)) return st;
    ConvLaunch L;
    memset(&L, 0, sizeof(L));
    L.jobs_dev = (const ConvJob *)scr;
    L.jobs_host = cj.data();
    L.n_jobs = (int)n_jobs;
    L.h_dev = h_dev;
    L.src_dev = src_dev;
    L.y_dev = y_dev;
    L.precision = precision;
    L.seed = seed;
    L.any_noise = any_noise;
    L.noise_partials_dev = any_noise ? (double *)((char *)scr + jb + 256) : nullptr;
    StatusTicket tk;
    int st = ISM_OK;
    if (precision == ISM_BF16X3) {
        // the tensor-core kernels' bounded waits report through a status cell
        st = status_begin(&tk);
        L.err_dev = tk.dev;
        L.inject = st ? 0 : take_injection(ISM_INJECT_CONV_WAIT);
    }
    if (!st) st = upload_async(scr, cj.data(), jb, stream);
    if (!st) {
        NvtxRange r("ism.conv.K2");
        if (precision == ISM_BF16X3) st = launch_conv_bf16x3(L, stream);
        else st = launch_conv_f32(L, stream);
    }
    if (!st) {
        NvtxRange r("ism.conv.noise");
        st = launch_noise(L, stream);
    }
    if (tk.cell >= 0) {
        const int se = status_end(tk, stream, st == ISM_OK);
        if (!st) st = se;
    }
    scratch_free(scr, stream);
    return st;
}
