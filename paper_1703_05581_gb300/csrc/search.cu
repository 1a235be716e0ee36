// Host driver and C ABI of the FFA search: the plan (Section 2.1 padding,
// Section 2.3 octaves and dereddening window), the search pipeline and the
// candidate extraction (first step of ffa2best, Section 2.3.3).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ffa {

namespace {
thread_local std::string g_err;
}

void set_error(const std::string& msg) { g_err = msg; }
ffa_status fail(ffa_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
ffa_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return FFA_ERR_CUDA;
}

static std::atomic<long long> g_launches{0};
void count_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int sm_count() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    cache[dev] = n;
    return n;
}

ffa_status ensure_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> done;
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(func, dev);
    auto it = done.find(key);
    if (it != done.end() && it->second >= bytes) return FFA_OK;
    FFA_CUDA_TRY(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done[key] = bytes;
    return FFA_OK;
}

// ---------------------------------------------------------------------------
// candidate extraction kernels
// ---------------------------------------------------------------------------
struct CandCtl {
    unsigned long long best_key;
    uint32_t count;  // records with snr >= snr_min
    uint32_t n_out;
    unsigned long long prefix, mask;
    uint32_t rank;
    uint32_t take;   // min(top_k, count)
    uint32_t hist[256];
};

struct CandOut {
    int64_t trial;
    float snr;
    int32_t width;
    int32_t phase;
    int32_t pad;
};

constexpr int CAND_MAX = 4096;

// ascending key = descending snr, then ascending trial index
__device__ __forceinline__ unsigned long long cand_key(float snr, int64_t idx) {
    return ((unsigned long long)(0xffffffffu - fkey(snr)) << 32) | (unsigned long long)(uint32_t)idx;
}

__global__ void k_cand_init(CandCtl* ctl) {
    int t = threadIdx.x;
    if (t == 0) {
        ctl->best_key = ~0ull;
        ctl->count = 0;
        ctl->n_out = 0;
        ctl->prefix = 0;
        ctl->mask = 0;
        ctl->rank = 0;
        ctl->take = 0;
    }
    for (int b = t; b < 256; b += blockDim.x) ctl->hist[b] = 0;
}

__global__ void k_cand_count(const ffa_record* __restrict__ rec, int64_t n, float snr_min,
                             CandCtl* ctl) {
    __shared__ unsigned long long s_best;
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) {
        s_best = ~0ull;
        s_cnt = 0;
    }
    __syncthreads();
    unsigned long long best = ~0ull;
    uint32_t cnt = 0;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float s = rec[i].snr;
        unsigned long long k = cand_key(s, i);
        best = k < best ? k : best;
        cnt += (s >= snr_min);
    }
    atomicMin(&s_best, best);
    atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMin(&ctl->best_key, s_best);
        atomicAdd(&ctl->count, s_cnt);
    }
}

__global__ void k_cand_hist(const ffa_record* __restrict__ rec, int64_t n, float snr_min,
                            int pass, CandCtl* ctl) {
    __shared__ uint32_t h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const unsigned long long prefix = ctl->prefix, mask = ctl->mask;
    const int shift = 56 - 8 * pass;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float s = rec[i].snr;
        if (!(s >= snr_min)) continue;
        unsigned long long k = cand_key(s, i);
        if ((k & mask) == prefix) atomicAdd(&h[(k >> shift) & 0xff], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&ctl->hist[b], h[b]);
}

__global__ void k_cand_pick(int pass, int top_k, CandCtl* ctl) {
    if (threadIdx.x != 0) return;
    if (pass == 0) {
        ctl->take = ctl->count < (uint32_t)top_k ? ctl->count : (uint32_t)top_k;
        ctl->rank = ctl->take > 0 ? ctl->take - 1 : 0;
    }
    if (ctl->take == 0) return;
    const int shift = 56 - 8 * pass;
    uint32_t c = 0;
    for (int b = 0; b < 256; ++b) {
        uint32_t h = ctl->hist[b];
        if (ctl->rank < c + h) {
            ctl->rank -= c;
            ctl->prefix |= (unsigned long long)b << shift;
            ctl->mask |= 0xffull << shift;
            break;
        }
        c += h;
    }
    for (int b = 0; b < 256; ++b) ctl->hist[b] = 0;
}

__global__ void k_cand_compact(const ffa_record* __restrict__ rec, int64_t n, float snr_min,
                               CandCtl* ctl, unsigned long long* keys) {
    if (ctl->take == 0) return;
    const unsigned long long thr = ctl->prefix;  // key of the take-th best
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float s = rec[i].snr;
        if (!(s >= snr_min)) continue;
        unsigned long long k = cand_key(s, i);
        if (k <= thr) {
            uint32_t slot = atomicAdd(&ctl->n_out, 1u);
            if (slot < CAND_MAX) keys[slot] = k;
        }
    }
}

__global__ void __launch_bounds__(1024) k_cand_sort(const ffa_record* __restrict__ rec,
                                                    CandCtl* ctl, const unsigned long long* keys,
                                                    CandOut* out) {
    __shared__ unsigned long long sk[CAND_MAX];
    uint32_t n = ctl->n_out < CAND_MAX ? ctl->n_out : CAND_MAX;
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (uint32_t t = threadIdx.x; t < np2; t += blockDim.x) sk[t] = t < n ? keys[t] : ~0ull;
    __syncthreads();
    for (uint32_t kk = 2; kk <= np2; kk <<= 1) {
        for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
            for (uint32_t t = threadIdx.x; t < np2; t += blockDim.x) {
                uint32_t u = t ^ jj;
                if (u > t) {
                    bool up = (t & kk) == 0;
                    unsigned long long a = sk[t], b = sk[u];
                    if ((a > b) == up) {
                        sk[t] = b;
                        sk[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        int64_t idx = (int64_t)(uint32_t)(sk[t] & 0xffffffffull);
        ffa_record r = rec[idx];
        CandOut o;
        o.trial = idx;
        o.snr = r.snr;
        o.width = r.width;
        o.phase = r.phase;
        o.pad = 0;
        out[t] = o;
    }
}

}  // namespace ffa

using namespace ffa;

namespace {
// benchmark instrumentation: event pairs around (phase, octave) intervals
struct TimingRec {
    int phase, octave;
    cudaEvent_t a, b;
};
std::mutex g_tmu;
bool g_timing = false;
std::vector<TimingRec> g_trec;
constexpr int64_t TIMING_SAMPLE = 64;  // per-kernel timing: every 64th base period of an octave

struct PhaseTimer {
    bool on = false;
    TimingRec r;
    cudaStream_t st;
    PhaseTimer(int phase, int octave, cudaStream_t s, bool enabled = true) : st(s) {
        {
            std::lock_guard<std::mutex> lk(g_tmu);
            on = g_timing && enabled;
        }
        if (!on) return;
        r.phase = phase;
        r.octave = octave;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
            on = false;
            return;
        }
        cudaEventRecord(r.a, st);
    }
    void stop() {
        if (!on) return;
        cudaEventRecord(r.b, st);
        std::lock_guard<std::mutex> lk(g_tmu);
        g_trec.push_back(r);
        on = false;
    }
};
}  // namespace

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// grouping of small base periods (see group_end)
constexpr int64_t GROUP_TRIALS = 1024;
constexpr int64_t GROUP_ELEMS = (int64_t)1 << 24;
// elements a base period's plane takes in a group (256-byte aligned)
static size_t plane_slot(const ffa_plan_entry& e) {
    return ((size_t)e.m_rows * (size_t)plane_pitch(e.p0) + 63) & ~(size_t)63;
}

extern "C" {

const char* ffa_status_string(ffa_status s) {
    switch (s) {
        case FFA_OK: return "ok";
        case FFA_ERR_ARG: return "invalid argument";
        case FFA_ERR_CUDA: return "CUDA error";
        case FFA_ERR_OOM: return "buffer too small";
        case FFA_ERR_TIMEOUT: return "timeout";
        case FFA_ERR_CANCELLED: return "cancelled";
        case FFA_ERR_UNSUPPORTED: return "unsupported";
        case FFA_ERR_DEVICE: return "device-side check failed";
    }
    return "unknown status";
}

const char* ffa_last_error(void) { return ffa::g_err.c_str(); }

ffa_status ffa_plan_create(const ffa_search_config* cfg, int64_t n, ffa_plan** out) {
    if (!cfg || !out) return fail(FFA_ERR_ARG, "plan: null argument");
    *out = nullptr;
    if (!(cfg->tsamp_s > 0.0) || !(cfg->period_min_s > 0.0) ||
        !(cfg->period_max_s > cfg->period_min_s))
        return fail(FFA_ERR_ARG, "plan: need tsamp > 0 and 0 < period_min < period_max");
    if (cfg->downsample0 < 1) return fail(FFA_ERR_ARG, "plan: downsample0 must be >= 1");
    if (n < 0) return fail(FFA_ERR_ARG, "plan: negative length");
    if (cfg->in_type != FFA_IN_F32 && cfg->in_type != FFA_IN_U8)
        return fail(FFA_ERR_ARG, "plan: in_type must be FFA_IN_F32 or FFA_IN_U8");
    if (cfg->precision != FFA_FOLD_F32 && cfg->precision != FFA_FOLD_I8)
        return fail(FFA_ERR_ARG, "plan: bad precision");
    if (cfg->scorer != FFA_SCORE_ALG1 && cfg->scorer != FFA_SCORE_ALG2)
        return fail(FFA_ERR_ARG, "plan: bad scorer");
    if (!(cfg->alg2_window >= 0.0f && cfg->alg2_window < 1.0f))
        return fail(FFA_ERR_ARG, "plan: alg2_window must be in [0, 1)");
    if (!(cfg->clip_sigma >= 0.0f) || std::isinf(cfg->clip_sigma))
        return fail(FFA_ERR_ARG, "plan: clip_sigma must be finite and >= 0");
    if (cfg->persistence && !std::isfinite(cfg->persist_cutoff))
        return fail(FFA_ERR_ARG, "plan: persist_cutoff must be finite");
    if (cfg->n_widths_fixed < 0 || cfg->n_widths_fixed > 16)
        return fail(FFA_ERR_ARG, "plan: n_widths_fixed must be in [0, 16]");
    if (cfg->n_widths_fixed == 0 && !(cfg->duty_max > 0.0))
        return fail(FFA_ERR_ARG, "plan: duty_max must be > 0 without fixed widths");
    for (int t = 0; t < cfg->n_widths_fixed; ++t) {
        int32_t w = cfg->widths_fixed[t];
        if (w < 1 || (w & (w - 1)) != 0 || (t > 0 && w <= cfg->widths_fixed[t - 1]))
            return fail(FFA_ERR_UNSUPPORTED, "plan: widths must be increasing powers of two");
    }
    ffa_plan* p = new (std::nothrow) ffa_plan();
    if (!p) return fail(FFA_ERR_OOM, "plan: host allocation failed");
    p->cfg = *cfg;
    p->n = n;
    const int64_t d0 = cfg->downsample0;
    p->n0 = n / d0;
    const double pmin = cfg->period_min_s / (cfg->tsamp_s * (double)d0);
    const double pmax = cfg->period_max_s / (cfg->tsamp_s * (double)d0);
    int64_t p_min = (int64_t)std::ceil(pmin - 1e-9);
    if (p_min < 1) p_min = 1;
    const int64_t p_max = (int64_t)std::ceil(pmax - 1e-9);
    int64_t w = cfg->detrend_window > 0 ? cfg->detrend_window : std::min(2 * p_max, 4 * p_min);
    if (cfg->detrend_window < 0) w = 1;
    w |= 1;
    if (w > INT32_MAX) w = INT32_MAX;
    p->window = (int32_t)w;
    const int64_t min_rows = cfg->min_rows > 0 ? cfg->min_rows : 2;
    int64_t n_o = p->n0;
    for (int32_t o = 0; o < 62; ++o) {
        if (o > 0) n_o /= 2;
        int64_t hi = std::min<int64_t>(2 * p_min, (int64_t)std::ceil(pmax / std::ldexp(1.0, o) - 1e-9));
        if (hi <= p_min || n_o <= 0) break;
        int64_t first = (int64_t)p->entries.size();
        for (int64_t p0 = p_min; p0 < hi; ++p0) {
            int64_t m_data = n_o / p0;
            if (m_data < min_rows) continue;
            int64_t m = 1;
            while (m < m_data) m *= 2;
            ffa_plan_entry e;
            std::memset(&e, 0, sizeof(e));
            e.octave = o;
            e.p0 = (int32_t)p0;
            e.m_data = (int32_t)m_data;
            e.m_rows = (int32_t)m;
            e.n_octave = n_o;
            e.first_trial = p->n_trials;
            if (cfg->n_widths_fixed > 0) {
                e.n_widths = cfg->n_widths_fixed;
                for (int t = 0; t < e.n_widths; ++t) e.widths[t] = cfg->widths_fixed[t];
            } else {
                int nw = 0;
                for (int64_t wd = 1;; wd *= 2) {
                    e.widths[nw++] = (int32_t)wd;
                    if ((double)wd > cfg->duty_max * (double)p0 || nw == 16) break;
                }
                e.n_widths = nw;
            }
            if (p0 > 32768) {
                delete p;
                return fail(FFA_ERR_UNSUPPORTED,
                            "plan: base periods above 32768 bins; raise downsample0");
            }
            if (cfg->precision == FFA_FOLD_I8) {
                // int32 box sums: |box| <= 127 * m_data * widest box
                double bound = 127.0 * (double)m_data * (double)e.widths[e.n_widths - 1];
                if (bound >= 2147483647.0) {
                    delete p;
                    return fail(FFA_ERR_UNSUPPORTED, "plan: int8 path would overflow int32 box sums");
                }
            }
            p->entries.push_back(e);
            p->n_trials += m;
            p->max_plane = std::max<int64_t>(p->max_plane, m * plane_pitch(p0));
        }
        int64_t cnt = (int64_t)p->entries.size() - first;
        if (cnt > 0) {
            p->oct_first.push_back(first);
            p->oct_count.push_back(cnt);
            p->oct_n.push_back(n_o);
            p->n_octaves = o + 1;
        } else {
            break;  // fewer rows at every later octave
        }
    }
    if (p->n_trials >= (int64_t)1 << 32) {
        delete p;
        return fail(FFA_ERR_UNSUPPORTED, "plan: more than 2^32 trials");
    }
    // workspace layout
    const int64_t n0 = std::max<int64_t>(p->n0, 1);
    size_t off = 0;
    p->off_raw_a = off;
    off = align256(off + sizeof(double) * n0);
    p->off_raw_b = off;
    off = align256(off + sizeof(double) * (n0 / 2 + 1));
    p->off_resid = off;
    off = align256(off + sizeof(double) * n0);
    p->off_z = off;
    off = align256(off + (cfg->precision == FFA_FOLD_F32 ? 4 : 1) * (size_t)n0);
    p->off_stats = off;
    off = align256(off + sizeof(double) * STATS_DOUBLES);
    // planes: the largest base period, or a group of small ones (GROUP_ELEMS)
    p->plane_elems = std::max<int64_t>(p->max_plane, 1);
    for (const ffa_plan_entry& e : p->entries)
        if (e.m_rows < GROUP_TRIALS) {
            const int64_t want = (GROUP_TRIALS / e.m_rows) * (int64_t)plane_slot(e);
            p->plane_elems = std::max<int64_t>(p->plane_elems, std::min<int64_t>(want, GROUP_ELEMS));
        }
    p->off_plane0 = off;
    off = align256(off + 4 * (size_t)p->plane_elems);
    p->off_plane1 = off;
    off = align256(off + 4 * (size_t)p->plane_elems);
    p->off_cand = off;
    off = align256(off + sizeof(CandCtl) + 256 + sizeof(unsigned long long) * CAND_MAX +
                   sizeof(CandOut) * CAND_MAX);
    p->off_best = off;
    off = align256(off + ffa::best_workspace_bytes((int64_t)p->entries.size(), p->n_trials));
    p->off_bits = off;
    if (cfg->persistence) off = align256(off + (size_t)n0);
    p->ws_bytes = off;
    *out = p;
    return FFA_OK;
}

void ffa_plan_destroy(ffa_plan* plan) { delete plan; }

ffa_status ffa_plan_info(const ffa_plan* p, int64_t* n_periods, int64_t* n_trials,
                         int32_t* n_octaves, int32_t* window, size_t* workspace_bytes) {
    if (!p) return fail(FFA_ERR_ARG, "plan_info: null plan");
    if (n_periods) *n_periods = (int64_t)p->entries.size();
    if (n_trials) *n_trials = p->n_trials;
    if (n_octaves) *n_octaves = p->n_octaves;
    if (window) *window = p->window;
    if (workspace_bytes) *workspace_bytes = p->ws_bytes;
    return FFA_OK;
}

ffa_status ffa_plan_entries(const ffa_plan* p, ffa_plan_entry* out, int64_t cap) {
    if (!p || (!out && cap > 0)) return fail(FFA_ERR_ARG, "plan_entries: null argument");
    int64_t m = std::min<int64_t>(cap, (int64_t)p->entries.size());
    if (m > 0) std::memcpy(out, p->entries.data(), sizeof(ffa_plan_entry) * (size_t)m);
    return FFA_OK;
}

ffa_status ffa_plan_periods(const ffa_plan* p, int64_t trial_begin, int64_t count, double* out) {
    if (!p) return fail(FFA_ERR_ARG, "plan_periods: null plan");
    if (count < 0 || trial_begin < 0 || trial_begin > p->n_trials || count > p->n_trials - trial_begin)
        return fail(FFA_ERR_ARG, "plan_periods: trial range outside the periodogram");
    if (count > 0 && !out) return fail(FFA_ERR_ARG, "plan_periods: null output");
    if (count == 0) return FFA_OK;
    // the entry holding trial_begin, then consecutive trials entry by entry
    size_t e = (size_t)(std::upper_bound(p->entries.begin(), p->entries.end(), trial_begin,
                                         [](int64_t t, const ffa_plan_entry& x) { return t < x.first_trial; }) -
                        p->entries.begin()) - 1;
    const double ts = p->cfg.tsamp_s * (double)p->cfg.downsample0;
    for (int64_t i = 0; i < count; ++i) {
        const int64_t t = trial_begin + i;
        while (t >= p->entries[e].first_trial + p->entries[e].m_rows) ++e;
        const ffa_plan_entry& en = p->entries[e];
        const int64_t k = t - en.first_trial;
        // Eq. 2 with the padded N = M * P0: P0 + k P0 / (N - P0) = P0 + k / (M - 1) samples
        const double frac = en.m_rows > 1 ? (double)k / (double)(en.m_rows - 1) : 0.0;
        out[i] = ((double)en.p0 + frac) * ts * std::ldexp(1.0, en.octave);
    }
    return FFA_OK;
}

// The pipeline for plan entries [e0, e1): every octave holding one of them is
// prepared (downsampled, dereddened, normalised); only those base periods are
// folded and scored.
// Consecutive base periods folded and scored by one set of launches: same
// octave, rows, widths and floor(log2 p0) (so the same tuned pass depth and
// CTA shape), together fewer than GROUP_TRIALS trials and within the plane
// buffers.  Base periods of GROUP_TRIALS rows or more go alone.

static int64_t group_end(const ffa_plan* p, int64_t t, int64_t b) {
    const ffa_plan_entry& e0 = p->entries[(size_t)t];
    if (e0.m_rows >= GROUP_TRIALS) return t + 1;
    auto lg = [](int64_t v) {
        int r = 0;
        while ((int64_t)2 << r <= v) ++r;
        return r;
    };
    int64_t j = t, trials = 0;
    size_t elems = 0;
    while (j < b && j - t < FOLD_GROUP_MAX) {
        const ffa_plan_entry& e = p->entries[(size_t)j];
        if (e.octave != e0.octave || e.m_rows != e0.m_rows || lg(e.p0) != lg(e0.p0) || e.n_widths != e0.n_widths ||
            std::memcmp(e.widths, e0.widths, sizeof(int32_t) * (size_t)e0.n_widths) != 0 ||
            score_shape(e.p0, e.widths[e.n_widths - 1]) != score_shape(e0.p0, e0.widths[e0.n_widths - 1]))
            break;
        if (elems + plane_slot(e) > (size_t)p->plane_elems || trials + e.m_rows > GROUP_TRIALS) break;
        elems += plane_slot(e);
        trials += e.m_rows;
        ++j;
    }
    return j > t ? j : t + 1;
}

// Prepare octave `oct` of the series in the workspace: the D0 sums, the
// octave downsampling chain on the raw series, the dereddening (resid) and the
// normalised fold input (z).  The debug outputs below use it.
static ffa_status prepare_octave(const ffa_plan* p, const void* d_series, char* ws, int32_t oct,
                                 int32_t* d_status, cudaStream_t st, int64_t* n_out) {
    const ffa_search_config& c = p->cfg;
    double* raw[2] = {(double*)(ws + p->off_raw_a), (double*)(ws + p->off_raw_b)};
    double* resid = (double*)(ws + p->off_resid);
    ffa_status s = launch_downsample(d_series, c.in_type, p->n, c.downsample0, raw[0], st);
    if (s != FFA_OK) return s;
    int64_t n_o = p->n0;
    for (int32_t o = 1; o <= oct; ++o) {
        s = launch_downsample(raw[(o - 1) & 1], FFA_IN_F64, n_o, 2, raw[o & 1], st);
        if (s != FFA_OK) return s;
        n_o /= 2;
    }
    double* cur = raw[oct & 1];
    if (p->window > 1) {
        s = launch_detrend(cur, n_o, p->window, resid, d_status, st);
    } else {
        cudaError_t e = cudaMemcpyAsync(resid, cur, sizeof(double) * n_o, cudaMemcpyDeviceToDevice, st);
        count_launch();
        s = e == cudaSuccess ? FFA_OK : cuda_fail(e, "prepare: copy");
    }
    if (s != FFA_OK) return s;
    s = launch_normalise(resid, n_o, c.precision, ws + p->off_z, (double*)(ws + p->off_stats), st,
                         c.clip_sigma, c.persist_cutoff, nullptr);
    *n_out = n_o;
    return s;
}

static ffa_status search_range(const ffa_plan* p, const void* d_series, void* d_ws, size_t ws_bytes,
                               ffa_record* d_records, int32_t* d_status, cudaStream_t st, int64_t e0,
                               int64_t e1, uint32_t* d_persist = nullptr) {
    if (!p) return fail(FFA_ERR_ARG, "search: null plan");
    const int64_t ne = (int64_t)p->entries.size();
    if (e0 < 0 || e1 > ne || e0 > e1) return fail(FFA_ERR_ARG, "search: entry range out of bounds");
    if (e0 == e1 || p->n_trials == 0) return FFA_OK;
    if (!d_series || !d_ws || !d_records) return fail(FFA_ERR_ARG, "search: null buffer");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "search: workspace too small");
    if ((uintptr_t)d_ws % 256 != 0) return fail(FFA_ERR_ARG, "search: workspace not 256-byte aligned");
    char* ws = (char*)d_ws;
    double* raw[2] = {(double*)(ws + p->off_raw_a), (double*)(ws + p->off_raw_b)};
    double* resid = (double*)(ws + p->off_resid);
    void* z = ws + p->off_z;
    double* stats = (double*)(ws + p->off_stats);
    int8_t* bits = d_persist ? (int8_t*)(ws + p->off_bits) : nullptr;
    void* plane0 = ws + p->off_plane0;
    void* plane1 = ws + p->off_plane1;
    const ffa_search_config& c = p->cfg;
    const int32_t last_oct = p->entries[(size_t)(e1 - 1)].octave;
    const int32_t first_oct = p->entries[(size_t)e0].octave;
    ffa_status s = launch_downsample(d_series, c.in_type, p->n, c.downsample0, raw[0], st);
    if (s != FFA_OK) return s;
    int64_t n_o = p->n0;
    for (int32_t o = 0; o <= last_oct; ++o) {
        double* cur = raw[o & 1];
        if (o > 0) {
            s = launch_downsample(raw[(o - 1) & 1], FFA_IN_F64, n_o, 2, cur, st);
            if (s != FFA_OK) return s;
            n_o /= 2;
        }
        if (o < first_oct) continue;  // only the downsampling chain is needed
        PhaseTimer prep_t(0, o, st);
        if (p->window > 1) {
            s = launch_detrend(cur, n_o, p->window, resid, d_status, st);
        } else {
            cudaError_t e = cudaMemcpyAsync(resid, cur, sizeof(double) * n_o, cudaMemcpyDeviceToDevice, st);
            count_launch();
            s = e == cudaSuccess ? FFA_OK : cuda_fail(e, "search: copy");
        }
        if (s != FFA_OK) return s;
        s = launch_normalise(resid, n_o, c.precision, z, stats, st, c.clip_sigma, c.persist_cutoff,
                             bits);
        if (s != FFA_OK) return s;
        prep_t.stop();
        PhaseTimer fold_t(1, o, st);
        const int64_t a = std::max<int64_t>(e0, p->oct_first[o]);
        const int64_t b = std::min<int64_t>(e1, p->oct_first[o] + p->oct_count[o]);
        for (int64_t t = a; t < b;) {
            const int64_t t1 = group_end(p, t, b);
            const ffa_plan_entry& e = p->entries[(size_t)t];
            int m = 0;
            while ((1 << m) < e.m_rows) ++m;
            ScoreWidths wd;
            wd.n = e.n_widths;
            for (int k = 0; k < 16; ++k) wd.w[k] = e.widths[k];
            const float excl = c.alg2_window > 0.0f ? c.alg2_window : 0.2f;
            if (t1 - t > 1) {
                // a group of small base periods: one set of fold launches, one scorer launch
                const int n = (int)(t1 - t);
                int64_t p0s[FOLD_GROUP_MAX], mds[FOLD_GROUP_MAX], offs[FOLD_GROUP_MAX];
                int64_t off = 0;
                for (int i = 0; i < n; ++i) {
                    const ffa_plan_entry& ei = p->entries[(size_t)(t + i)];
                    p0s[i] = ei.p0;
                    mds[i] = ei.m_data;
                    offs[i] = off;
                    off += (int64_t)plane_slot(ei);
                }
                // per-kernel timing of the groups holding an every-TIMING_SAMPLE-th base period
                const int64_t r0 = t - p->oct_first[o], r1 = t1 - 1 - p->oct_first[o];
                const bool gsample = (r0 % TIMING_SAMPLE) == 0 || r0 / TIMING_SAMPLE != r1 / TIMING_SAMPLE;
                PhaseTimer gfold_k(4, o, st, gsample);
                s = launch_fold_group(z, c.precision, n, p0s, mds, offs, e.m_rows, m > 0 ? m - 1 : 0, plane0,
                                      plane1, st);
                if (s != FFA_OK) return s;
                gfold_k.stop();
                PhaseTimer gscore_k(5, o, st, gsample);
                ffa_record* recs[FOLD_GROUP_MAX];
                for (int i = 0; i < n; ++i) recs[i] = d_records + p->entries[(size_t)(t + i)].first_trial;
                if (c.scorer == FFA_SCORE_ALG2)
                    s = launch_score_alg2_group(plane0, c.precision, n, p0s, offs, e.m_rows, wd, excl, recs, st);
                else
                    s = launch_score2_group(plane0, c.precision, n, p0s, offs, e.m_rows, wd, recs, d_status, st);
                if (s != FFA_OK) return s;
                gscore_k.stop();
                if (d_persist) {
                    s = launch_fold_group(bits, FFA_FOLD_I8, n, p0s, mds, offs, e.m_rows, m > 0 ? m - 1 : 0, plane0,
                                          plane1, st);
                    if (s != FFA_OK) return s;
                    for (int i = 0; i < n; ++i) {
                        const ffa_plan_entry& ei = p->entries[(size_t)(t + i)];
                        s = launch_persist((const int32_t*)plane0 + offs[i], ei.m_rows, ei.p0, plane_pitch(ei.p0),
                                           d_records + ei.first_trial, d_persist + ei.first_trial, st);
                        if (s != FFA_OK) return s;
                    }
                }
                t = t1;
                continue;
            }
            // per-kernel timing of every TIMING_SAMPLE-th base period of an octave
            const bool sample = ((t - p->oct_first[o]) % TIMING_SAMPLE) == 0;
            // all but the last stage; the scorer applies the last one while loading
            PhaseTimer fold_k(2, o, st, sample);
            const int64_t ld = plane_pitch(e.p0);
            s = launch_fold(z, c.precision, e.p0, e.m_data, e.m_rows, m > 0 ? m - 1 : 0, ld, plane0,
                            plane1, st);
            if (s != FFA_OK) return s;
            fold_k.stop();
            PhaseTimer score_k(3, o, st, sample);
            if (c.scorer == FFA_SCORE_ALG2)
                s = launch_score_alg2(plane0, c.precision, true, e.m_rows, 0, e.p0, ld, e.m_rows, wd, excl,
                                      d_records + e.first_trial, st);
            else
                s = launch_score2(plane0, c.precision, true, e.m_rows, 0, e.p0, ld, e.m_rows, wd,
                                  d_records + e.first_trial, d_status, st);
            if (s != FFA_OK) return s;
            score_k.stop();
            if (d_persist) {
                // the 0/1 series through the same fold, then each trial's window sum
                s = launch_fold(bits, FFA_FOLD_I8, e.p0, e.m_data, e.m_rows, m > 0 ? m - 1 : 0, ld,
                                plane0, plane1, st);
                if (s != FFA_OK) return s;
                s = launch_persist((const int32_t*)plane0, e.m_rows, e.p0, ld, d_records + e.first_trial,
                                   d_persist + e.first_trial, st);
                if (s != FFA_OK) return s;
            }
            ++t;
        }
        fold_t.stop();
    }
    return FFA_OK;
}

ffa_status ffa_autotune(const ffa_plan* p, void* d_ws, size_t ws_bytes, void* stream, int32_t* n_tuned) {
    if (!p) return fail(FFA_ERR_ARG, "autotune: null plan");
    if (n_tuned) *n_tuned = 0;
    if (p->n_trials == 0) return FFA_OK;
    if (!d_ws) return fail(FFA_ERR_ARG, "autotune: null workspace");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "autotune: workspace too small");
    char* ws = (char*)d_ws;
    // shapes: (stages before the fused last one, floor(log2 p0)) -> its entries
    std::map<std::pair<int, int>, std::vector<size_t>> groups;
    for (size_t i = 0; i < p->entries.size(); ++i) {
        const ffa_plan_entry& e = p->entries[i];
        int m = 0, lg = 0;
        while ((1 << m) < e.m_rows) ++m;
        while ((int64_t)2 << lg <= e.p0) ++lg;
        groups[{m > 0 ? m - 1 : 0, lg}].push_back(i);
    }
    int32_t n = 0;
    for (auto& g : groups) {
        const ffa_plan_entry& e = p->entries[g.second[g.second.size() / 2]];  // the median base period
        ffa_status s = tune_fold(ws + p->off_z, p->cfg.precision, e.p0, e.m_data, e.m_rows, g.first.first,
                                 plane_pitch(e.p0), ws + p->off_plane0, ws + p->off_plane1, as_stream(stream),
                                 nullptr);
        if (s != FFA_OK) return s;
        ++n;
    }
    if (n_tuned) *n_tuned = n;
    return FFA_OK;
}

ffa_status ffa_search_persistence(const ffa_plan* p, const void* d_series, void* d_ws,
                                  size_t ws_bytes, ffa_record* d_records, uint32_t* d_persist,
                                  int32_t* d_status, void* stream) {
    if (!p) return fail(FFA_ERR_ARG, "search_persistence: null plan");
    if (!p->cfg.persistence) return fail(FFA_ERR_ARG, "search_persistence: plan made without persistence");
    if (p->n_trials > 0 && !d_persist) return fail(FFA_ERR_ARG, "search_persistence: null output");
    return search_range(p, d_series, d_ws, ws_bytes, d_records, d_status, as_stream(stream), 0,
                        (int64_t)p->entries.size(), d_persist);
}

ffa_status ffa_search(const ffa_plan* p, const void* d_series, void* d_ws, size_t ws_bytes,
                      ffa_record* d_records, int32_t* d_status, void* stream) {
    if (!p) return fail(FFA_ERR_ARG, "search: null plan");
    return search_range(p, d_series, d_ws, ws_bytes, d_records, d_status, as_stream(stream), 0,
                        (int64_t)p->entries.size());
}

ffa_status ffa_search_entries(const ffa_plan* p, const void* d_series, int64_t entry_begin,
                              int64_t entry_end, void* d_ws, size_t ws_bytes, ffa_record* d_records,
                              int32_t* d_status, void* stream) {
    return search_range(p, d_series, d_ws, ws_bytes, d_records, d_status, as_stream(stream),
                        entry_begin, entry_end);
}

ffa_status ffa_search_series(const ffa_plan* p, const void* d_series, int32_t octave, int32_t what,
                             void* d_ws, size_t ws_bytes, void* d_out, int32_t* d_status, void* stream) {
    if (!p) return fail(FFA_ERR_ARG, "search_series: null plan");
    if (octave < 0 || octave >= p->n_octaves) return fail(FFA_ERR_ARG, "search_series: octave outside the plan");
    if (what != FFA_DUMP_RESID && what != FFA_DUMP_Z) return fail(FFA_ERR_ARG, "search_series: bad `what`");
    if (!d_series || !d_ws || !d_out) return fail(FFA_ERR_ARG, "search_series: null buffer");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "search_series: workspace too small");
    if ((uintptr_t)d_ws % 256 != 0) return fail(FFA_ERR_ARG, "search_series: workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    int64_t n_o = 0;
    ffa_status s = prepare_octave(p, d_series, ws, octave, d_status, st, &n_o);
    if (s != FFA_OK) return s;
    const void* src = what == FFA_DUMP_RESID ? (const void*)(ws + p->off_resid) : (const void*)(ws + p->off_z);
    const size_t esz = what == FFA_DUMP_RESID ? 8 : (p->cfg.precision == FFA_FOLD_F32 ? 4 : 1);
    cudaError_t e = cudaMemcpyAsync(d_out, src, esz * (size_t)n_o, cudaMemcpyDeviceToDevice, st);
    count_launch();
    return e == cudaSuccess ? FFA_OK : cuda_fail(e, "search_series: copy");
}

ffa_status ffa_search_plane(const ffa_plan* p, const void* d_series, int64_t entry, void* d_ws, size_t ws_bytes,
                            void* d_plane, int32_t* d_status, void* stream) {
    if (!p) return fail(FFA_ERR_ARG, "search_plane: null plan");
    if (entry < 0 || entry >= (int64_t)p->entries.size()) return fail(FFA_ERR_ARG, "search_plane: entry outside the plan");
    if (!d_series || !d_ws || !d_plane) return fail(FFA_ERR_ARG, "search_plane: null buffer");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "search_plane: workspace too small");
    if ((uintptr_t)d_ws % 256 != 0) return fail(FFA_ERR_ARG, "search_plane: workspace not 256-byte aligned");
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    const ffa_plan_entry& e = p->entries[(size_t)entry];
    int64_t n_o = 0;
    ffa_status s = prepare_octave(p, d_series, ws, e.octave, d_status, st, &n_o);
    if (s != FFA_OK) return s;
    // every stage on the search's padded-pitch planes, then the rows packed
    // densely into the caller's plane
    const int64_t ld = plane_pitch(e.p0);
    s = launch_fold(ws + p->off_z, p->cfg.precision, e.p0, e.m_data, e.m_rows, -1, ld, ws + p->off_plane0,
                    ws + p->off_plane1, st);
    if (s != FFA_OK) return s;
    const size_t esz = 4;  // float or int32
    cudaError_t ce = cudaMemcpy2DAsync(d_plane, esz * (size_t)e.p0, ws + p->off_plane0, esz * (size_t)ld,
                                       esz * (size_t)e.p0, (size_t)e.m_rows, cudaMemcpyDeviceToDevice, st);
    count_launch();
    return ce == cudaSuccess ? FFA_OK : cuda_fail(ce, "search_plane: copy");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched search: many series (e.g. dedispersion trials of uneven length)
// with one configuration.  Octave by octave, every series is prepared into
// its own slice of the workspace, then the base periods of all series are
// folded and scored together: items with the same rows, widths, scorer
// shape and floor(log2 P0) -- from any series -- share one set of fold
// launches and one persistent scorer launch (up to FOLD_GROUP_MAX base
// periods and BATCH_GROUP_ELEMS plane elements per group), each reading its
// own series and writing its own series' records.  Every base period runs
// the same kernels with the same add tree and scorer shape as in ffa_search,
// so the records are those of each series searched alone.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t BATCH_GROUP_ELEMS = (int64_t)1 << 25;  // per plane buffer (32-bit elements)

struct BatchLayout {
    std::vector<size_t> raw_off, z_off;
    size_t off_tmp = 0, off_resid = 0, off_stats = 0, off_plane0 = 0, off_plane1 = 0, bytes = 0;
    int64_t plane_elems = 0;
};

ffa_status batch_layout(const ffa_plan* const* plans, int32_t count, BatchLayout* L) {
    if (count < 1 || !plans) return fail(FFA_ERR_ARG, "batch: need at least one plan");
    for (int32_t i = 0; i < count; ++i) {
        if (!plans[i]) return fail(FFA_ERR_ARG, "batch: null plan");
        if (std::memcmp(&plans[i]->cfg, &plans[0]->cfg, sizeof(ffa_search_config)) != 0)
            return fail(FFA_ERR_ARG, "batch: every plan needs the same configuration (lengths may differ)");
    }
    if (plans[0]->cfg.persistence) return fail(FFA_ERR_UNSUPPORTED, "batch: persistence plans are searched one by one");
    const size_t esz = plans[0]->cfg.precision == FFA_FOLD_F32 ? 4 : 1;
    int64_t max_n0 = 1, max_slot = 1;
    size_t off = 0;
    L->raw_off.resize((size_t)count);
    L->z_off.resize((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        const int64_t n0 = std::max<int64_t>(plans[i]->n0, 1);
        max_n0 = std::max(max_n0, n0);
        for (const ffa_plan_entry& e : plans[i]->entries) max_slot = std::max<int64_t>(max_slot, (int64_t)plane_slot(e));
        L->raw_off[(size_t)i] = off;
        off = align256(off + sizeof(double) * (size_t)n0);
    }
    for (int32_t i = 0; i < count; ++i) {
        L->z_off[(size_t)i] = off;
        off = align256(off + esz * (size_t)std::max<int64_t>(plans[i]->n0, 1));
    }
    L->off_tmp = off;
    off = align256(off + sizeof(double) * (size_t)(max_n0 / 2 + 1));
    L->off_resid = off;
    off = align256(off + sizeof(double) * (size_t)max_n0);
    L->off_stats = off;
    off = align256(off + sizeof(double) * STATS_DOUBLES);
    L->plane_elems = std::max<int64_t>(max_slot, std::min<int64_t>(BATCH_GROUP_ELEMS, (int64_t)count * max_slot));
    L->off_plane0 = off;
    off = align256(off + 4 * (size_t)L->plane_elems);
    L->off_plane1 = off;
    off = align256(off + 4 * (size_t)L->plane_elems);
    L->bytes = off;
    return FFA_OK;
}

struct BatchItem {
    int32_t series;
    const ffa_plan_entry* e;
    int shape, lg;
};

int lg2(int64_t v) {
    int r = 0;
    while ((int64_t)2 << r <= v) ++r;
    return r;
}

bool batch_compatible(const BatchItem& a, const BatchItem& b) {
    return a.e->m_rows == b.e->m_rows && a.shape == b.shape && a.lg == b.lg && a.e->n_widths == b.e->n_widths &&
           std::memcmp(a.e->widths, b.e->widths, sizeof(int32_t) * (size_t)a.e->n_widths) == 0;
}
}  // namespace

extern "C" {

ffa_status ffa_batch_workspace_bytes(const ffa_plan* const* plans, int32_t count, size_t* bytes) {
    if (!bytes) return fail(FFA_ERR_ARG, "batch_workspace_bytes: null output");
    BatchLayout L;
    ffa_status s = batch_layout(plans, count, &L);
    if (s != FFA_OK) return s;
    *bytes = L.bytes;
    return FFA_OK;
}

ffa_status ffa_search_batch(const ffa_plan* const* plans, const void* const* d_series, int32_t count,
                            void* d_ws, size_t ws_bytes, ffa_record* const* d_records,
                            int32_t* d_status, void* stream) {
    if (count < 0) return fail(FFA_ERR_ARG, "search_batch: negative count");
    if (count == 0) return FFA_OK;
    if (!d_series || !d_records) return fail(FFA_ERR_ARG, "search_batch: null argument");
    BatchLayout L;
    ffa_status s = batch_layout(plans, count, &L);
    if (s != FFA_OK) return s;
    if (!d_ws) return fail(FFA_ERR_ARG, "search_batch: null workspace");
    if (ws_bytes < L.bytes) return fail(FFA_ERR_OOM, "search_batch: workspace too small (ffa_batch_workspace_bytes)");
    if ((uintptr_t)d_ws % 256 != 0) return fail(FFA_ERR_ARG, "search_batch: workspace not 256-byte aligned");
    for (int32_t i = 0; i < count; ++i)
        if (plans[i]->n_trials > 0 && (!d_series[i] || !d_records[i]))
            return fail(FFA_ERR_ARG, "search_batch: null series or records");
    const ffa_search_config& c = plans[0]->cfg;
    const int32_t window = plans[0]->window;
    cudaStream_t st = as_stream(stream);
    char* ws = (char*)d_ws;
    double* tmp = (double*)(ws + L.off_tmp);
    double* resid = (double*)(ws + L.off_resid);
    double* stats = (double*)(ws + L.off_stats);
    void* plane0 = ws + L.off_plane0;
    void* plane1 = ws + L.off_plane1;
    const size_t esz = c.precision == FFA_FOLD_F32 ? 4 : 1;
    int32_t max_oct = 0;
    std::vector<int64_t> n_o((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        max_oct = std::max(max_oct, plans[i]->n_octaves);
        n_o[(size_t)i] = plans[i]->n0;
        if (plans[i]->n_octaves > 0) {
            s = launch_downsample(d_series[i], c.in_type, plans[i]->n, c.downsample0, (double*)(ws + L.raw_off[(size_t)i]),
                                  st);
            if (s != FFA_OK) return s;
        }
    }
    const float excl = c.alg2_window > 0.0f ? c.alg2_window : 0.2f;
    for (int32_t o = 0; o < max_oct; ++o) {
        PhaseTimer prep_t(0, o, st);
        std::vector<BatchItem> items;
        for (int32_t i = 0; i < count; ++i) {
            const ffa_plan* p = plans[i];
            if (p->n_octaves <= o) continue;
            double* raw = (double*)(ws + L.raw_off[(size_t)i]);
            int64_t& n = n_o[(size_t)i];
            if (o > 0) {
                s = launch_downsample(raw, FFA_IN_F64, n, 2, tmp, st);
                if (s != FFA_OK) return s;
                n /= 2;
                cudaError_t ce = cudaMemcpyAsync(raw, tmp, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
                count_launch();
                if (ce != cudaSuccess) return cuda_fail(ce, "search_batch: copy");
            }
            if (window > 1) {
                s = launch_detrend(raw, n, window, resid, d_status, st);
            } else {
                cudaError_t ce = cudaMemcpyAsync(resid, raw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st);
                count_launch();
                s = ce == cudaSuccess ? FFA_OK : cuda_fail(ce, "search_batch: copy");
            }
            if (s != FFA_OK) return s;
            s = launch_normalise(resid, n, c.precision, ws + L.z_off[(size_t)i], stats, st, c.clip_sigma, c.persist_cutoff,
                                 nullptr);
            if (s != FFA_OK) return s;
            const int64_t a = p->oct_first[(size_t)o], b = a + p->oct_count[(size_t)o];
            for (int64_t t = a; t < b; ++t) {
                const ffa_plan_entry& e = p->entries[(size_t)t];
                items.push_back(BatchItem{i, &e, score_shape(e.p0, e.widths[e.n_widths - 1]), lg2(e.p0)});
            }
        }
        prep_t.stop();
        PhaseTimer fold_t(1, o, st);
        std::stable_sort(items.begin(), items.end(), [](const BatchItem& x, const BatchItem& y) {
            if (x.e->m_rows != y.e->m_rows) return x.e->m_rows > y.e->m_rows;
            if (x.shape != y.shape) return x.shape < y.shape;
            if (x.lg != y.lg) return x.lg < y.lg;
            if (x.e->n_widths != y.e->n_widths) return x.e->n_widths < y.e->n_widths;
            const int wc = std::memcmp(x.e->widths, y.e->widths, sizeof(int32_t) * (size_t)x.e->n_widths);
            if (wc != 0) return wc < 0;
            return x.e->p0 < y.e->p0;
        });
        for (size_t t = 0; t < items.size();) {
            size_t j = t;
            int64_t elems = 0;
            while (j < items.size() && j - t < (size_t)FOLD_GROUP_MAX && batch_compatible(items[j], items[t]) &&
                   elems + (int64_t)plane_slot(*items[j].e) <= L.plane_elems) {
                elems += (int64_t)plane_slot(*items[j].e);
                ++j;
            }
            if (j == t) ++j;
            const int n = (int)(j - t);
            const ffa_plan_entry& e0 = *items[t].e;
            int m = 0;
            while ((1 << m) < e0.m_rows) ++m;
            int64_t p0s[FOLD_GROUP_MAX], mds[FOLD_GROUP_MAX], offs[FOLD_GROUP_MAX];
            const void* srcs[FOLD_GROUP_MAX];
            ffa_record* recs[FOLD_GROUP_MAX];
            int64_t off = 0;
            for (int k = 0; k < n; ++k) {
                const BatchItem& it = items[t + (size_t)k];
                p0s[k] = it.e->p0;
                mds[k] = it.e->m_data;
                offs[k] = off;
                off += (int64_t)plane_slot(*it.e);
                srcs[k] = ws + L.z_off[(size_t)it.series];
                recs[k] = d_records[it.series] + it.e->first_trial;
            }
            (void)esz;
            s = launch_fold_group(srcs[0], c.precision, n, p0s, mds, offs, e0.m_rows, m > 0 ? m - 1 : 0, plane0, plane1,
                                  st, srcs);
            if (s != FFA_OK) return s;
            ScoreWidths wd;
            wd.n = e0.n_widths;
            for (int k = 0; k < 16; ++k) wd.w[k] = e0.widths[k];
            if (c.scorer == FFA_SCORE_ALG2)
                s = launch_score_alg2_group(plane0, c.precision, n, p0s, offs, e0.m_rows, wd, excl, recs, st);
            else
                s = launch_score2_group(plane0, c.precision, n, p0s, offs, e0.m_rows, wd, recs, d_status, st);
            if (s != FFA_OK) return s;
            t = j;
        }
        fold_t.stop();
    }
    return FFA_OK;
}

int64_t ffa_launch_count(void) { return (int64_t)ffa::g_launches.load(); }

ffa_status ffa_timing_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_tmu);
    g_timing = on != 0;
    return FFA_OK;
}

ffa_status ffa_timing_read(double* ms, int32_t* counts, int32_t cap) {
    if (!ms || !counts || cap < 256) return fail(FFA_ERR_ARG, "timing_read: need cap >= 256");
    std::vector<TimingRec> recs;
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        recs.swap(g_trec);
    }
    for (int i = 0; i < cap; ++i) {
        ms[i] = 0.0;
        counts[i] = 0;
    }
    ffa_status st = FFA_OK;
    for (auto& r : recs) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess) st = cuda_fail(e, "timing_read");
        int idx = r.phase * 64 + (r.octave < 64 ? r.octave : 63);
        if (idx < cap) {
            ms[idx] += t;
            counts[idx] += 1;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    return st;
}

ffa_status ffa_wait(void* stream, const int32_t* d_status, int32_t timeout_ms) {
    cudaStream_t st = as_stream(stream);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(e, "wait: cudaStreamQuery");
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(
                      std::chrono::steady_clock::now() - t0).count();
        if (timeout_ms >= 0 && ms > timeout_ms) return fail(FFA_ERR_TIMEOUT, "wait: stream did not finish in time");
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    if (d_status) {
        int32_t h = 0;
        FFA_CUDA_TRY(cudaMemcpy(&h, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost));
        if (h != 0) return fail((ffa_status)h, "device-side check failed");
    }
    return FFA_OK;
}

// Candidates among the trials of plan entries [e0, e1) (records outside are
// not read).
static ffa_status candidates_range(const ffa_plan* p, int64_t e0, int64_t e1, const ffa_record* d_records,
                                   double snr_min, int32_t top_k, void* d_ws, size_t ws_bytes,
                                   ffa_candidate* out, int32_t* n_out, int64_t* best, int32_t* d_status,
                                   void* stream, int32_t timeout_ms) {
    if (!p || !n_out || !best) return fail(FFA_ERR_ARG, "candidates: null argument");
    if (top_k < 0 || top_k > CAND_MAX) return fail(FFA_ERR_ARG, "candidates: top_k must be in [0, 4096]");
    if (top_k > 0 && !out) return fail(FFA_ERR_ARG, "candidates: null output");
    const int64_t ne = (int64_t)p->entries.size();
    if (e0 < 0 || e1 > ne || e0 > e1) return fail(FFA_ERR_ARG, "candidates: entry range out of bounds");
    *n_out = 0;
    *best = -1;
    if (e0 == e1 || p->n_trials == 0) return FFA_OK;
    if (!d_records || !d_ws) return fail(FFA_ERR_ARG, "candidates: null buffer");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "candidates: workspace too small");
    cudaStream_t st = as_stream(stream);
    char* base = (char*)d_ws + p->off_cand;
    CandCtl* ctl = (CandCtl*)base;
    unsigned long long* keys = (unsigned long long*)(base + align256(sizeof(CandCtl)));
    CandOut* cout = (CandOut*)(base + align256(sizeof(CandCtl)) + sizeof(unsigned long long) * CAND_MAX);
    const int64_t t0 = p->entries[(size_t)e0].first_trial;
    const ffa_plan_entry& el = p->entries[(size_t)(e1 - 1)];
    const int64_t n = el.first_trial + el.m_rows - t0;
    const ffa_record* rec = d_records + t0;
    const float smin = (float)snr_min;
    const int grid = sm_count() * 8;
    k_cand_init<<<1, 256, 0, st>>>(ctl);
    k_cand_count<<<grid, 256, 0, st>>>(rec, n, smin, ctl);
    for (int pass = 0; pass < 8; ++pass) {
        k_cand_hist<<<grid, 256, 0, st>>>(rec, n, smin, pass, ctl);
        k_cand_pick<<<1, 32, 0, st>>>(pass, top_k, ctl);
    }
    k_cand_compact<<<grid, 256, 0, st>>>(rec, n, smin, ctl, keys);
    k_cand_sort<<<1, 1024, 0, st>>>(rec, ctl, keys, cout);
    FFA_LAUNCH_CHECK("candidates kernels");
    count_launch(21);
    ffa_status s = ffa_wait(stream, d_status, timeout_ms);
    if (s != FFA_OK) return s;
    CandCtl h;
    FFA_CUDA_TRY(cudaMemcpy(&h, ctl, sizeof(CandCtl), cudaMemcpyDeviceToHost));
    uint32_t m = std::min<uint32_t>(h.n_out, (uint32_t)top_k);
    std::vector<CandOut> buf(m);
    if (m > 0) FFA_CUDA_TRY(cudaMemcpy(buf.data(), cout, sizeof(CandOut) * m, cudaMemcpyDeviceToHost));
    if (h.best_key != ~0ull) *best = t0 + (int64_t)(uint32_t)(h.best_key & 0xffffffffull);
    const ffa_search_config& c = p->cfg;
    for (uint32_t t = 0; t < m; ++t) {
        const CandOut& o = buf[t];
        const int64_t trial = t0 + o.trial;
        // entry holding this trial: the last one with first_trial <= trial
        auto it = std::upper_bound(p->entries.begin(), p->entries.end(), trial,
                                   [](int64_t v, const ffa_plan_entry& e) { return v < e.first_trial; });
        const ffa_plan_entry& e = *(it - 1);
        ffa_candidate& d = out[t];
        d.trial = trial;
        d.octave = e.octave;
        d.p0 = e.p0;
        d.k = (int32_t)(trial - e.first_trial);
        d.snr = o.snr;
        d.width = o.width;
        d.phase = o.phase;
        const double scale = c.tsamp_s * (double)c.downsample0 * std::ldexp(1.0, e.octave);
        d.period_s = ((double)e.p0 + (double)d.k / (double)(e.m_rows - 1)) * scale;
    }
    *n_out = (int32_t)m;
    return FFA_OK;
}

ffa_status ffa_candidates(const ffa_plan* p, const ffa_record* d_records, double snr_min,
                          int32_t top_k, void* d_ws, size_t ws_bytes, ffa_candidate* out,
                          int32_t* n_out, int64_t* best, int32_t* d_status, void* stream,
                          int32_t timeout_ms) {
    if (!p) return fail(FFA_ERR_ARG, "candidates: null plan");
    return candidates_range(p, 0, (int64_t)p->entries.size(), d_records, snr_min, top_k, d_ws, ws_bytes,
                            out, n_out, best, d_status, stream, timeout_ms);
}

ffa_status ffa_candidates_entries(const ffa_plan* p, int64_t entry_begin, int64_t entry_end,
                                  const ffa_record* d_records, double snr_min, int32_t top_k,
                                  void* d_ws, size_t ws_bytes, ffa_candidate* out, int32_t* n_out,
                                  int64_t* best, int32_t* d_status, void* stream, int32_t timeout_ms) {
    return candidates_range(p, entry_begin, entry_end, d_records, snr_min, top_k, d_ws, ws_bytes, out,
                            n_out, best, d_status, stream, timeout_ms);
}

// ---- step entry points ------------------------------------------------------

ffa_status ffa_downsample(const void* d_in, int32_t in_type, int64_t n, int64_t factor,
                          double* d_out, void* stream) {
    if (n < 0 || factor < 1) return fail(FFA_ERR_ARG, "downsample: need n >= 0 and factor >= 1");
    if (n / factor > 0 && (!d_in || !d_out)) return fail(FFA_ERR_ARG, "downsample: null buffer");
    return launch_downsample(d_in, in_type, n, factor, d_out, as_stream(stream));
}

ffa_status ffa_detrend(const double* d_raw, int64_t n, int32_t window, double* d_resid,
                       int32_t* d_status, void* stream) {
    if (n < 0 || window < 1) return fail(FFA_ERR_ARG, "detrend: need n >= 0 and window >= 1");
    if (n > 0 && (!d_raw || !d_resid)) return fail(FFA_ERR_ARG, "detrend: null buffer");
    if (n >= ((int64_t)1 << 31)) return fail(FFA_ERR_UNSUPPORTED, "detrend: n >= 2^31");
    return launch_detrend(d_raw, n, window, d_resid, d_status, as_stream(stream));
}

ffa_status ffa_normalise(const double* d_resid, int64_t n, int32_t precision, void* d_out,
                         double* d_stats, void* stream) {
    if (n < 0) return fail(FFA_ERR_ARG, "normalise: negative length");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8) return fail(FFA_ERR_ARG, "normalise: bad precision");
    if (n > 0 && (!d_resid || !d_out || !d_stats)) return fail(FFA_ERR_ARG, "normalise: null buffer");
    return launch_normalise(d_resid, n, precision, d_out, d_stats, as_stream(stream));
}

ffa_status ffa_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                    void* d_plane, void* d_tmp, void* stream) {
    if (p0 < 1 || m_data < 0 || m_rows < 1 || (m_rows & (m_rows - 1)) != 0 || m_data > m_rows)
        return fail(FFA_ERR_ARG, "fold: need p0 >= 1, m_rows a power of two >= m_data");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8) return fail(FFA_ERR_ARG, "fold: bad precision");
    if (!d_z || !d_plane || !d_tmp) return fail(FFA_ERR_ARG, "fold: null buffer");
    if (p0 > INT64_MAX / 4 / m_rows) return fail(FFA_ERR_ARG, "fold: m_rows * p0 elements overflow");
    return launch_fold(d_z, precision, p0, m_data, m_rows, -1, p0, d_plane, d_tmp, as_stream(stream));
}

ffa_status ffa_score(const void* d_profiles, int32_t precision, int64_t count, int64_t p0,
                     const int32_t* widths, int32_t n_widths, ffa_record* d_records,
                     int32_t* d_status, void* stream) {
    if (count < 0 || p0 < 1) return fail(FFA_ERR_ARG, "score: need count >= 0 and p0 >= 1");
    if (n_widths < 1 || n_widths > 16 || !widths) return fail(FFA_ERR_ARG, "score: 1..16 widths");
    ScoreWidths wd;
    wd.n = n_widths;
    for (int t = 0; t < 16; ++t) wd.w[t] = t < n_widths ? widths[t] : 0;
    for (int t = 0; t < n_widths; ++t) {
        int32_t w = widths[t];
        if (w < 1 || (w & (w - 1)) != 0 || (t > 0 && w <= widths[t - 1]))
            return fail(FFA_ERR_UNSUPPORTED, "score: widths must be increasing powers of two");
    }
    if (count > 0 && (!d_profiles || !d_records)) return fail(FFA_ERR_ARG, "score: null buffer");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8) return fail(FFA_ERR_ARG, "score: bad precision");
    return launch_score2(d_profiles, precision, false, count, 0, p0, p0, 1, wd, d_records, d_status,
                         as_stream(stream));
}

ffa_status ffa_score_alg2(const void* d_profiles, int32_t precision, int64_t count, int64_t p0,
                          const int32_t* widths, int32_t n_widths, float excl_frac,
                          ffa_record* d_records, void* stream) {
    if (count < 0 || p0 < 1) return fail(FFA_ERR_ARG, "score_alg2: need count >= 0 and p0 >= 1");
    if (n_widths < 1 || n_widths > 16 || !widths) return fail(FFA_ERR_ARG, "score_alg2: 1..16 widths");
    if (!(excl_frac >= 0.0f && excl_frac < 1.0f)) return fail(FFA_ERR_ARG, "score_alg2: excl_frac in [0, 1)");
    ScoreWidths wd;
    wd.n = n_widths;
    for (int t = 0; t < 16; ++t) wd.w[t] = t < n_widths ? widths[t] : 0;
    for (int t = 0; t < n_widths; ++t) {
        int32_t w = widths[t];
        if (w < 1 || (w & (w - 1)) != 0 || (t > 0 && w <= widths[t - 1]))
            return fail(FFA_ERR_UNSUPPORTED, "score_alg2: widths must be increasing powers of two");
    }
    if (count > 0 && (!d_profiles || !d_records)) return fail(FFA_ERR_ARG, "score_alg2: null buffer");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8) return fail(FFA_ERR_ARG, "score_alg2: bad precision");
    return launch_score_alg2(d_profiles, precision, false, count, 0, p0, p0, 1, wd, excl_frac, d_records,
                             as_stream(stream));
}

}  // extern "C"
