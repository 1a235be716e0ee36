// ffa2best (Section 2.3.3): from a periodogram to a candidate list.
//
//   1. peak separation over the whole periodogram in three phases, since the
//      state machine is sequential: k_best_spec walks every chunk of records
//      in parallel as if no candidate were open at its start, checkpointing
//      its state before every 32-record batch; k_best_fix, one warp, carries
//      the true state across the chunks in order, walking each chunk only
//      until its state equals the speculative checkpoint (from there the two
//      walks are the same: the same state sees the same records); k_best_tail
//      resumes every chunk's speculative walk from that point in parallel.
//      Two walks meet at the first record that raises or ends both of their
//      candidates, so the sequential part is short.  Every peak is reported
//      once, by the phase that processes the record ending its candidate;
//      the sequential phase's peaks are kept (k_best_refix replays them in
//      the later passes instead of walking again).
//      The first pass (phases B and C) stores up to PEAK_CAP peak keys and
//      counts every peak by its top 16 key bits.  With more peaks than that,
//      k_best_plan narrows a radix select of the SEL_MAX-th strongest key 16
//      bits at a time, each level one more pass histogramming the next 16
//      bits of the keys still in play, until the keys at or above a
//      threshold fit PEAK_CAP; a last pass stores exactly those.  Keys are
//      unique (they hold the trial), so four levels always suffice.
//   2. k_best_select one CTA: the strongest SEL_MAX stored peaks (an MSB radix
//                    select when there are more), a bitonic sort (S/N down,
//                    trial up), the period and duty of each, then the greedy
//                    grouping / harmonic filter, strongest first, every test
//                    of a candidate against the kept list in parallel.
//
// The arithmetic of every decision is IEEE binary64 with explicit
// round-to-nearest operations (no contraction), in the order the thresholds
// are defined in the header, so that it decides exactly as a plain FP64
// evaluation of the same definitions does.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ffa {

namespace {

constexpr int PEAK_CAP = 1 << 16;   // peaks the walk may store
constexpr int SEL_MAX = 4096;       // strongest peaks the filter considers
constexpr int FR_MAX = 2112;        // prime fractions for primes <= 97 (2 x 1035)
constexpr int WALK_CHUNK = 16384;   // records per warp chunk (a multiple of 32)
constexpr int SEL_THREADS = 1024;

constexpr int HIST_BINS = 1 << 16;
constexpr int FIX_CAP = 1 << 20;    // peaks of the sequential phase kept for the later passes

struct BestCtl {
    uint32_t n_peaks;   // peaks in the periodogram (counted by the first walk)
    uint32_t n_stored;  // peak keys in the buffer
    uint32_t n_kept;
    uint32_t n_sel;     // peaks the filter considered
    // radix narrowing of the SEL_MAX-th strongest key
    int32_t done;       // the buffer holds what the filter needs
    int32_t emit;       // next walk: store every key <= thr
    int32_t shift;      // next walk: histogram bits [shift, shift + 16)
    uint32_t need;      // keys still wanted within the prefix group
    uint32_t taken;     // keys known to be stronger than the prefix group
    uint32_t n_fix;     // peaks the first sequential pass reported
    unsigned long long prefix, mask, thr;
};

// one base period: first trial, P0, M, octave
struct BestEntry {
    int64_t first;
    int32_t p0;
    int32_t m_rows;
    int32_t octave;
    int32_t pad;
};

struct WalkArgs {
    float base_f;    // smallest float >= snr_min
    double keep;     // 1 - drop_frac
    double drop_abs;
};

struct SelArgs {
    double scale0;   // tsamp * D0 (seconds per bin at octave 0)
    double t_obs;    // n * tsamp
    double shrink;   // 1 - group_margin
    double tol;
    int32_t group;
    int32_t n_fr;    // entries of the prime-fraction table (0: no harmonics)
    int32_t cap;
    int32_t n_entries;
};

struct Layout {
    size_t hist, peaks, ent, fr, out, ck, end_state, merge, fix, total;
};

Layout layout(int64_t n_entries, int64_t n_trials) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    Layout L;
    const size_t n_chunks = (size_t)((n_trials + WALK_CHUNK - 1) / WALK_CHUNK);
    size_t off = al(sizeof(BestCtl));
    L.hist = off;
    off = al(off + sizeof(uint32_t) * HIST_BINS);
    L.peaks = off;
    off = al(off + sizeof(unsigned long long) * PEAK_CAP);
    L.ent = off;
    off = al(off + sizeof(BestEntry) * (size_t)std::max<int64_t>(n_entries, 1));
    L.fr = off;
    off = al(off + (sizeof(double) + sizeof(int32_t)) * FR_MAX);
    L.out = off;
    off = al(off + sizeof(ffa_candidate) * SEL_MAX);
    L.ck = off;
    off = al(off + sizeof(unsigned long long) * (size_t)((std::max<int64_t>(n_trials, 1) + 31) / 32));
    L.end_state = off;
    off = al(off + sizeof(unsigned long long) * std::max<size_t>(n_chunks, 1));
    L.merge = off;
    off = al(off + sizeof(int32_t) * std::max<size_t>(n_chunks, 1));
    L.fix = off;
    off = al(off + sizeof(unsigned long long) * FIX_CAP);
    L.total = off;
    return L;
}

// ascending key = descending S/N, then ascending trial
__device__ __forceinline__ unsigned long long peak_key(float snr, int64_t trial) {
    return ((unsigned long long)(0xffffffffu - fkey(snr)) << 32) | (unsigned long long)(uint32_t)trial;
}

__global__ void k_best_init(BestCtl* ctl, uint32_t* hist) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        ctl->n_peaks = 0;
        ctl->n_stored = 0;
        ctl->n_kept = 0;
        ctl->n_sel = 0;
        ctl->done = 0;
        ctl->emit = 0;
        ctl->shift = 48;
        ctl->need = SEL_MAX;
        ctl->taken = 0;
        ctl->n_fix = 0;
        ctl->prefix = 0;
        ctl->mask = 0;
        ctl->thr = 0;
    }
    for (int b = t; b < HIST_BINS; b += gridDim.x * blockDim.x) hist[b] = 0;
}

// What a walk does with each peak it finds (warp-uniform; lane 0 acts).
struct WalkMode {
    int first;   // count, store up to PEAK_CAP, histogram the top 16 bits
    int emit;    // store keys <= thr
    int shift;   // otherwise: histogram bits [shift, shift + 16) of keys in the prefix group
    unsigned long long prefix, mask, thr;
    unsigned long long* fixlist;  // non-null: also keep the key for the later passes
};

__device__ __forceinline__ void emit_peak(BestCtl* ctl, unsigned long long* peaks, uint32_t* hist,
                                          const WalkMode& md, float pk, int64_t pi, int lane) {
    if (lane != 0) return;
    const unsigned long long key = peak_key(pk, pi);
    if (md.fixlist) {
        const uint32_t f = atomicAdd(&ctl->n_fix, 1u);
        if (f < (uint32_t)FIX_CAP) md.fixlist[f] = key;
    }
    if (md.first) {
        atomicAdd(&ctl->n_peaks, 1u);
        atomicAdd(&hist[key >> 48], 1u);
        const uint32_t slot = atomicAdd(&ctl->n_stored, 1u);
        if (slot < (uint32_t)PEAK_CAP) peaks[slot] = key;
    } else if (md.emit) {
        if (key <= md.thr) {
            const uint32_t slot = atomicAdd(&ctl->n_stored, 1u);
            if (slot < (uint32_t)PEAK_CAP) peaks[slot] = key;
        }
    } else if ((key & md.mask) == md.prefix) {
        atomicAdd(&hist[(key >> md.shift) & 0xffffu], 1u);
    }
}

// One step of the radix narrowing (one CTA): after a walk's histogram, pick
// the 16-bit digit holding the need-th strongest key of the prefix group;
// switch to the storing walk once every key up to that digit fits PEAK_CAP.
__global__ void __launch_bounds__(1024) k_best_plan(BestCtl* ctl, uint32_t* hist) {
    __shared__ uint32_t part[1024];
    __shared__ int s_skip;
    const int tid = threadIdx.x;
    if (tid == 0) {
        if (ctl->emit) ctl->done = 1;  // the storing walk has run
        int skip = ctl->done;
        if (!skip && ctl->shift == 48 && ctl->n_peaks <= (uint32_t)PEAK_CAP) {
            ctl->done = 1;  // the first walk stored every peak
            skip = 1;
        }
        if (!skip && ctl->shift == 48 && ctl->n_stored > 0) ctl->n_stored = 0;  // overflowed: restart the buffer
        s_skip = skip;
    }
    __syncthreads();
    if (s_skip) return;
    constexpr int PER = HIST_BINS / 1024;
    uint32_t sum = 0;
    for (int i = 0; i < PER; ++i) sum += hist[tid * PER + i];
    part[tid] = sum;
    __syncthreads();
    if (tid == 0) {
        const uint32_t need = ctl->need;
        uint32_t cum = 0;
        int chunk = 0;
        while (chunk < 1024 && cum + part[chunk] < need) cum += part[chunk++];
        int b = chunk * PER;
        uint32_t h = 0;
        for (; b < (chunk + 1) * PER; ++b) {
            h = hist[b];
            if (cum + h >= need) break;
            cum += h;
        }
        // cum = keys of the group before digit b; h = keys with digit b
        const int shift = ctl->shift;
        const unsigned long long dig = (unsigned long long)b << shift;
        const unsigned long long low = shift > 0 ? ((1ull << shift) - 1ull) : 0ull;
        if (ctl->taken + cum + h <= (uint32_t)PEAK_CAP || shift == 0) {
            ctl->emit = 1;
            ctl->thr = ctl->prefix | dig | low;
            ctl->n_stored = 0;
        } else {
            ctl->taken += cum;
            ctl->need = need - cum;
            ctl->prefix |= dig;
            ctl->mask |= 0xffffull << shift;
            ctl->shift = shift - 16;
        }
    }
    __syncthreads();
    for (int b = tid; b < HIST_BINS; b += 1024) hist[b] = 0;
}

// Walk state: outside a candidate, or inside with running peak pk at pi.
// Encoded for checkpoints as fkey(pk) << 32 | pi, or all ones outside
// (pi < 2^32 - 1 since a plan has fewer than 2^32 trials).
struct WalkState {
    bool inside;
    float pk;
    uint32_t pi;
    // the end test s < pk * (1 - drop_frac) && s < pk - drop_abs, both sides
    // FP64, as one float compare: for a float s, s < d exactly when s is below
    // the smallest float >= d (d rounded towards +inf)
    float end_below;
};

constexpr unsigned long long OUTSIDE = ~0ull;

__device__ __forceinline__ unsigned long long encode(const WalkState& w) {
    return w.inside ? (((unsigned long long)fkey(w.pk) << 32) | w.pi) : OUTSIDE;
}

__device__ __forceinline__ void set_peak(WalkState& w, float pk, uint32_t pi, const WalkArgs& a) {
    w.inside = true;
    w.pk = pk;
    w.pi = pi;
    const double t = fmin(__dmul_rn((double)pk, a.keep), __dsub_rn((double)pk, a.drop_abs));
    w.end_below = __double2float_ru(t);
}

__device__ __forceinline__ WalkState decode(unsigned long long e, const WalkArgs& a) {
    WalkState w;
    w.inside = false;
    w.pk = 0.0f;
    w.pi = 0;
    w.end_below = 0.0f;
    if (e != OUTSIDE) set_peak(w, fkey_inv((uint32_t)(e >> 32)), (uint32_t)(e & 0xffffffffull), a);
    return w;
}

// The state machine over records [b, lim), lim - b <= 32, one warp
// (warp-uniform state; lane j holds record b + j's S/N in s).  EMIT: report
// the peak of every candidate that ends here.
template <bool EMIT>
__device__ __forceinline__ void walk_batch(float s, int64_t b, int64_t lim, const WalkArgs& a, WalkState& w,
                                           BestCtl* ctl, unsigned long long* peaks, uint32_t* hist,
                                           const WalkMode& md, int lane) {
    const bool valid = b + lane < lim;
    const unsigned starts = __ballot_sync(0xffffffffu, valid && s >= a.base_f);
    if (!w.inside && !starts) return;
    const int nvalid = (int)min((int64_t)32, lim - b);
    for (int j = w.inside ? 0 : __ffs(starts) - 1; j < nvalid; ++j) {
        const float sj = __shfl_sync(0xffffffffu, s, j);
        if (w.inside) {
            if (sj > w.pk) {
                set_peak(w, sj, (uint32_t)(b + j), a);
            } else if (sj < w.end_below) {
                if (EMIT) emit_peak(ctl, peaks, hist, md, w.pk, w.pi, lane);
                w.inside = false;
            }
        }
        if (!w.inside && sj >= a.base_f) set_peak(w, sj, (uint32_t)(b + j), a);
    }
}

__device__ __forceinline__ float snr_at(const ffa_record* __restrict__ rec, int64_t i, int64_t lim) {
    return i < lim ? rec[i].snr : 0.0f;
}

__device__ __forceinline__ WalkMode load_mode(int first, const BestCtl* ctl) {
    WalkMode md;
    md.first = first;
    md.emit = 0;
    md.shift = 48;
    md.prefix = md.mask = md.thr = 0;
    md.fixlist = nullptr;
    if (!first) {
        md.emit = ctl->emit;
        md.shift = ctl->shift;
        md.prefix = ctl->prefix;
        md.mask = ctl->mask;
        md.thr = ctl->thr;
    }
    return md;
}

// Phase A (parallel, once): every chunk walked as if no candidate were open
// at its start; the state before each 32-record batch is checkpointed, and
// the state at the chunk's end kept.
__global__ void __launch_bounds__(256) k_best_spec(const ffa_record* __restrict__ rec, int64_t n, WalkArgs a,
                                                   unsigned long long* __restrict__ ck,
                                                   unsigned long long* __restrict__ end_state) {
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
    WalkMode none{};
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += n_warps) {
        const int64_t c0 = c * WALK_CHUNK, c1 = min(n, c0 + WALK_CHUNK);
        WalkState w = decode(OUTSIDE, a);
        float s = snr_at(rec, c0 + lane, c1);
        for (int64_t b = c0; b < c1; b += 32) {
            const float sn = snr_at(rec, b + 32 + lane, c1);  // next batch, in flight meanwhile
            if (lane == 0) ck[b >> 5] = encode(w);
            walk_batch<false>(s, b, c1, a, w, nullptr, nullptr, nullptr, none, lane);
            s = sn;
        }
        if (lane == 0) end_state[c] = encode(w);
    }
}

// Phase B (one warp, per radix level): the true state carried across the
// chunks in order.  In each chunk the true walk runs only until its state
// equals the speculative checkpoint at a batch boundary (the two walks
// coincide from there on); merge[c] is that batch, and the chunk's end state
// is then the speculative one.  The peaks that end before the merge, and a
// candidate still open at the end of the periodogram, are reported here.
__global__ void __launch_bounds__(32) k_best_fix(const ffa_record* __restrict__ rec, int64_t n, WalkArgs a,
                                                 int first, const unsigned long long* __restrict__ ck,
                                                 const unsigned long long* __restrict__ end_state,
                                                 int32_t* __restrict__ merge, BestCtl* ctl,
                                                 unsigned long long* peaks, uint32_t* hist,
                                                 unsigned long long* fixlist) {
    // later passes replay the first pass's peaks from fixlist (k_best_refix)
    // unless there were too many to keep
    if (!first && (ctl->done || ctl->n_fix <= (uint32_t)FIX_CAP)) return;
    WalkMode md = load_mode(first, ctl);
    if (first) md.fixlist = fixlist;
    const int lane = threadIdx.x & 31;
    const int64_t n_chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
    WalkState w = decode(OUTSIDE, a);
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t c0 = c * WALK_CHUNK, c1 = min(n, c0 + WALK_CHUNK);
        const int32_t nb = (int32_t)((c1 - c0 + 31) >> 5);
        int32_t t = 0;
        float s = snr_at(rec, c0 + lane, c1);
        unsigned long long cke = ck[c0 >> 5];
        for (; t < nb; ++t) {
            const int64_t b = c0 + 32 * (int64_t)t;
            if (encode(w) == cke) break;
            // the next batch's values and checkpoint, in flight meanwhile
            const float sn = snr_at(rec, b + 32 + lane, c1);
            const unsigned long long ckn = t + 1 < nb ? ck[(b >> 5) + 1] : OUTSIDE;
            walk_batch<true>(s, b, c1, a, w, ctl, peaks, hist, md, lane);
            s = sn;
            cke = ckn;
        }
        if (lane == 0) merge[c] = t;
        if (t < nb) w = decode(end_state[c], a);
    }
    if (w.inside) emit_peak(ctl, peaks, hist, md, w.pk, w.pi, lane);
}

// Phase B of a later pass, replayed: the first pass's sequential-phase peaks,
// reported again in the current pass's mode.
__global__ void __launch_bounds__(256) k_best_refix(BestCtl* ctl, const unsigned long long* __restrict__ fixlist,
                                                    unsigned long long* peaks, uint32_t* hist) {
    if (ctl->done || ctl->n_fix > (uint32_t)FIX_CAP) return;
    const WalkMode md = load_mode(0, ctl);
    const uint32_t nf = ctl->n_fix;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        const unsigned long long key = fixlist[i];
        emit_peak(ctl, peaks, hist, md, fkey_inv(0xffffffffu - (uint32_t)(key >> 32)),
                  (int64_t)(uint32_t)(key & 0xffffffffull), 0);
    }
}

// Phase C (parallel, per radix level): each chunk's speculative walk resumed
// from its merge checkpoint, reporting the peaks that end inside the chunk
// (a candidate open at the chunk's end belongs to the next chunk's phase B).
__global__ void __launch_bounds__(256) k_best_tail(const ffa_record* __restrict__ rec, int64_t n, WalkArgs a,
                                                   int first, const unsigned long long* __restrict__ ck,
                                                   const int32_t* __restrict__ merge, BestCtl* ctl,
                                                   unsigned long long* peaks, uint32_t* hist) {
    if (!first && ctl->done) return;
    const WalkMode md = load_mode(first, ctl);
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_chunks = (n + WALK_CHUNK - 1) / WALK_CHUNK;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += n_warps) {
        const int64_t c0 = c * WALK_CHUNK, c1 = min(n, c0 + WALK_CHUNK);
        const int64_t b0 = c0 + 32 * (int64_t)merge[c];
        if (b0 >= c1) continue;
        WalkState w = decode(ck[b0 >> 5], a);
        float s = snr_at(rec, b0 + lane, c1);
        for (int64_t b = b0; b < c1; b += 32) {
            const float sn = snr_at(rec, b + 32 + lane, c1);
            walk_batch<true>(s, b, c1, a, w, ctl, peaks, hist, md, lane);
            s = sn;
        }
    }
}

// period of a trial in seconds (Eq. 2 with N = M * P0) and its entry
__device__ __forceinline__ int find_entry(const BestEntry* __restrict__ ent, int n_ent, int64_t t) {
    int lo = 0, hi = n_ent - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ent[mid].first <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct SelShared {
    unsigned long long key[SEL_MAX];
    double per[SEL_MAX];
    double duty[SEL_MAX];
    float snr[SEL_MAX];
    uint16_t kept[SEL_MAX];
    double frg[FR_MAX];       // approximate value of each fraction (sorted)
    int32_t frc[FR_MAX];      // n | x << 8 | kind << 16 (kind 1: divide)
    uint32_t hist[256];
    uint32_t cnt;
    uint32_t n_kept;
    unsigned long long prefix, mask;
    uint32_t rank;
};

__device__ __forceinline__ bool smeared_match(float s_i, double p, float s_j, double q, double d_j,
                                              const SelArgs& a) {
    const double dq = fabs(__dsub_rn(p, q));
    const double drift = __ddiv_rn(__dmul_rn(a.t_obs, dq), __dmul_rn(q, q));
    const double de = __dadd_rn(d_j, drift);
    const double resp = de >= 1.0 ? 0.0 : __dmul_rn((double)s_j, __dsqrt_rn(__ddiv_rn(d_j, de)));
    return __dmul_rn((double)s_i, a.shrink) <= resp;
}

__device__ bool harmonic_match(double p, double q, const SelShared& sh, const SelArgs& a) {
    const double r = __ddiv_rn(p, q);
    const double w = 2.0 * a.tol + 1e-12;
    const double glo = r * (1.0 - w), ghi = r * (1.0 + w);
    int lo = 0, hi = a.n_fr;  // first entry with frg >= glo
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (sh.frg[mid] < glo) lo = mid + 1;
        else hi = mid;
    }
    for (int t = lo; t < a.n_fr && sh.frg[t] <= ghi; ++t) {
        const int32_t c = sh.frc[t];
        const double f = __ddiv_rn((double)(c & 0xff), (double)((c >> 8) & 0xff));
        const double v = (c >> 16) ? __ddiv_rn(q, f) : __dmul_rn(q, f);
        if (fabs(__dsub_rn(p, v)) <= __dmul_rn(a.tol, v)) return true;
    }
    return false;
}

__global__ void __launch_bounds__(SEL_THREADS) k_best_select(
    const ffa_record* __restrict__ rec, const BestEntry* __restrict__ ent,
    const double* __restrict__ fr_g, const int32_t* __restrict__ fr_c,
    const unsigned long long* __restrict__ peaks, BestCtl* ctl, SelArgs a, ffa_candidate* out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SelShared& sh = *reinterpret_cast<SelShared*>(smem_raw);
    const int tid = threadIdx.x;
    const uint32_t n_all = ctl->n_stored;
    const uint32_t n = n_all < (uint32_t)PEAK_CAP ? n_all : (uint32_t)PEAK_CAP;
    const uint32_t take = n < (uint32_t)SEL_MAX ? n : (uint32_t)SEL_MAX;
    for (int t = tid; t < a.n_fr; t += SEL_THREADS) {
        sh.frg[t] = fr_g[t];
        sh.frc[t] = fr_c[t];
    }
    if (tid == 0) {
        sh.cnt = 0;
        sh.n_kept = 0;
        sh.prefix = 0;
        sh.mask = 0;
        sh.rank = take > 0 ? take - 1 : 0;
    }
    __syncthreads();
    if (n > (uint32_t)SEL_MAX) {
        // the take-th smallest key, 8 bits at a time from the top (keys are unique)
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 56 - 8 * pass;
            for (int b = tid; b < 256; b += SEL_THREADS) sh.hist[b] = 0;
            __syncthreads();
            const unsigned long long prefix = sh.prefix, mask = sh.mask;
            for (uint32_t i = tid; i < n; i += SEL_THREADS) {
                const unsigned long long k = peaks[i];
                if ((k & mask) == prefix) atomicAdd(&sh.hist[(k >> shift) & 0xff], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t c = 0;
                for (int b = 0; b < 256; ++b) {
                    const uint32_t h = sh.hist[b];
                    if (sh.rank < c + h) {
                        sh.rank -= c;
                        sh.prefix |= (unsigned long long)b << shift;
                        sh.mask |= 0xffull << shift;
                        break;
                    }
                    c += h;
                }
            }
            __syncthreads();
        }
        const unsigned long long thr = sh.prefix;
        for (uint32_t i = tid; i < n; i += SEL_THREADS) {
            const unsigned long long k = peaks[i];
            if (k <= thr) {
                const uint32_t slot = atomicAdd(&sh.cnt, 1u);
                if (slot < (uint32_t)SEL_MAX) sh.key[slot] = k;
            }
        }
    } else {
        for (uint32_t i = tid; i < n; i += SEL_THREADS) sh.key[i] = peaks[i];
    }
    // bitonic sort of the first pow2 >= take keys (padding sorts last)
    uint32_t sp = 1;
    while (sp < take) sp <<= 1;
    for (uint32_t i = take + tid; i < sp; i += SEL_THREADS) sh.key[i] = ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= sp; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = tid; i < sp; i += SEL_THREADS) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const unsigned long long x = sh.key[i], y = sh.key[l];
                    const bool up = (i & k) == 0;
                    if ((x > y) == up) {
                        sh.key[i] = y;
                        sh.key[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
    // period and duty of each considered peak
    for (uint32_t t = tid; t < take; t += SEL_THREADS) {
        const unsigned long long k = sh.key[t];
        const int64_t trial = (int64_t)(uint32_t)(k & 0xffffffffull);
        const BestEntry e = ent[find_entry(ent, a.n_entries, trial)];
        const int64_t kk = trial - e.first;
        const double scale = __dmul_rn(a.scale0, ldexp(1.0, e.octave));
        const double frac = e.m_rows > 1 ? __ddiv_rn((double)kk, (double)(e.m_rows - 1)) : 0.0;
        sh.per[t] = __dmul_rn(__dadd_rn((double)e.p0, frac), scale);
        sh.duty[t] = __ddiv_rn((double)rec[trial].width, (double)e.p0);
        sh.snr[t] = fkey_inv(0xffffffffu - (uint32_t)(k >> 32));
    }
    __syncthreads();
    // greedy filter, strongest first
    const bool harm = a.n_fr > 0;
    for (uint32_t c = 0; c < take; ++c) {
        const uint32_t nk = sh.n_kept;
        if (nk >= (uint32_t)a.cap) break;
        const double p = sh.per[c];
        const float s_c = sh.snr[c];
        int hit = 0;
        for (uint32_t j = tid; j < nk && !hit; j += SEL_THREADS) {
            const int idx = sh.kept[j];
            const double q = sh.per[idx];
            if (a.group && smeared_match(s_c, p, sh.snr[idx], q, sh.duty[idx], a)) hit = 1;
            else if (harm && harmonic_match(p, q, sh, a)) hit = 1;
        }
        hit = __syncthreads_or(hit);
        if (!hit && tid == 0) sh.kept[sh.n_kept++] = (uint16_t)c;
        __syncthreads();
    }
    // kept candidates, strongest first
    const uint32_t nk = sh.n_kept;
    for (uint32_t j = tid; j < nk; j += SEL_THREADS) {
        const int c = sh.kept[j];
        const unsigned long long k = sh.key[c];
        const int64_t trial = (int64_t)(uint32_t)(k & 0xffffffffull);
        const BestEntry e = ent[find_entry(ent, a.n_entries, trial)];
        const ffa_record r = rec[trial];
        ffa_candidate o;
        o.trial = trial;
        o.period_s = sh.per[c];
        o.snr = sh.snr[c];
        o.octave = e.octave;
        o.p0 = e.p0;
        o.k = (int32_t)(trial - e.first);
        o.width = r.width;
        o.phase = r.phase;
        out[j] = o;
    }
    if (tid == 0) {
        ctl->n_kept = nk;
        ctl->n_sel = take;
    }
}

bool is_prime(int x) {
    if (x < 2) return false;
    for (int d = 2; d * d <= x; ++d)
        if (x % d == 0) return false;
    return true;
}

}  // namespace

size_t best_workspace_bytes(int64_t n_entries, int64_t n_trials) {
    return layout(n_entries, n_trials).total;
}

}  // namespace ffa

using namespace ffa;

extern "C" ffa_status ffa2best(const ffa_plan* p, const ffa_record* d_records,
                               const ffa2best_config* cfg, void* d_ws, size_t ws_bytes,
                               ffa_candidate* out, int32_t cap, int32_t* n_out, int64_t* n_peaks,
                               int32_t* d_status, void* stream, int32_t timeout_ms) {
    if (!p || !cfg || !n_out || !n_peaks) return fail(FFA_ERR_ARG, "ffa2best: null argument");
    if (cap < 0 || cap > SEL_MAX) return fail(FFA_ERR_ARG, "ffa2best: cap must be in [0, 4096]");
    if (cap > 0 && !out) return fail(FFA_ERR_ARG, "ffa2best: null output");
    if (!std::isfinite(cfg->snr_min) || !(cfg->drop_frac >= 0.0 && cfg->drop_frac <= 1.0) ||
        !(cfg->drop_abs >= 0.0 && std::isfinite(cfg->drop_abs)))
        return fail(FFA_ERR_ARG, "ffa2best: need finite snr_min, drop_frac in [0, 1], drop_abs >= 0");
    if (!(cfg->harm_tol >= 0.0 && cfg->harm_tol <= 0.1))
        return fail(FFA_ERR_ARG, "ffa2best: harm_tol must be in [0, 0.1]");
    if (!(cfg->group_margin >= 0.0 && cfg->group_margin < 1.0))
        return fail(FFA_ERR_ARG, "ffa2best: group_margin must be in [0, 1)");
    if (cfg->primes_max > 97) return fail(FFA_ERR_UNSUPPORTED, "ffa2best: primes_max above 97");
    *n_out = 0;
    *n_peaks = 0;
    if (p->n_trials == 0) return FFA_OK;
    if (!d_records || !d_ws) return fail(FFA_ERR_ARG, "ffa2best: null buffer");
    if (ws_bytes < p->ws_bytes) return fail(FFA_ERR_OOM, "ffa2best: workspace too small");
    cudaStream_t st = as_stream(stream);
    const int64_t n_ent = (int64_t)p->entries.size();
    const Layout L = layout(n_ent, p->n_trials);
    char* base = (char*)d_ws + p->off_best;
    BestCtl* ctl = (BestCtl*)base;
    uint32_t* hist = (uint32_t*)(base + L.hist);
    unsigned long long* peaks = (unsigned long long*)(base + L.peaks);
    BestEntry* ent = (BestEntry*)(base + L.ent);
    double* fr_g = (double*)(base + L.fr);
    int32_t* fr_c = (int32_t*)(base + L.fr + sizeof(double) * FR_MAX);
    ffa_candidate* dout = (ffa_candidate*)(base + L.out);
    unsigned long long* ck = (unsigned long long*)(base + L.ck);
    unsigned long long* end_state = (unsigned long long*)(base + L.end_state);
    int32_t* merge = (int32_t*)(base + L.merge);
    unsigned long long* fixlist = (unsigned long long*)(base + L.fix);

    // host tables: base periods, and the prime fractions sorted by value
    std::vector<BestEntry> he((size_t)n_ent);
    for (int64_t i = 0; i < n_ent; ++i) {
        const ffa_plan_entry& e = p->entries[(size_t)i];
        he[(size_t)i] = BestEntry{e.first_trial, e.p0, e.m_rows, e.octave, 0};
    }
    std::vector<std::pair<double, int32_t>> fr;
    for (int x = 2; x <= cfg->primes_max; ++x) {
        if (!is_prime(x)) continue;
        for (int k = 1; k < x; ++k) {
            fr.emplace_back((double)k / (double)x, k | (x << 8));
            fr.emplace_back((double)x / (double)k, k | (x << 8) | (1 << 16));
        }
    }
    std::sort(fr.begin(), fr.end());
    std::vector<double> hg(fr.size());
    std::vector<int32_t> hc(fr.size());
    for (size_t i = 0; i < fr.size(); ++i) {
        hg[i] = fr[i].first;
        hc[i] = fr[i].second;
    }
    FFA_CUDA_TRY(cudaMemcpyAsync(ent, he.data(), sizeof(BestEntry) * he.size(), cudaMemcpyHostToDevice, st));
    if (!fr.empty()) {
        FFA_CUDA_TRY(cudaMemcpyAsync(fr_g, hg.data(), sizeof(double) * hg.size(), cudaMemcpyHostToDevice, st));
        FFA_CUDA_TRY(cudaMemcpyAsync(fr_c, hc.data(), sizeof(int32_t) * hc.size(), cudaMemcpyHostToDevice, st));
    }

    // thresholds as exact float bounds
    WalkArgs wa;
    wa.keep = 1.0 - cfg->drop_frac;
    wa.drop_abs = cfg->drop_abs;
    auto ceil_f = [](double v) {
        float f = (float)v;
        if ((double)f < v) f = std::nextafter(f, INFINITY);
        return f;
    };
    wa.base_f = ceil_f(cfg->snr_min);

    SelArgs sa;
    sa.scale0 = p->cfg.tsamp_s * (double)p->cfg.downsample0;
    sa.t_obs = (double)p->n * p->cfg.tsamp_s;
    sa.shrink = 1.0 - cfg->group_margin;
    sa.tol = cfg->harm_tol;
    sa.group = cfg->group != 0;
    sa.n_fr = (int32_t)fr.size();
    sa.cap = cap;
    sa.n_entries = (int32_t)n_ent;

    const size_t smem = sizeof(SelShared);
    ffa_status es = ensure_smem((const void*)k_best_select, smem);
    if (es != FFA_OK) return es;
    const int64_t nt = p->n_trials;
    const int nsm = sm_count();
    k_best_init<<<64, 1024, 0, st>>>(ctl, hist);
    k_best_spec<<<nsm * 8, 256, 0, st>>>(d_records, nt, wa, ck, end_state);
    k_best_fix<<<1, 32, 0, st>>>(d_records, nt, wa, 1, ck, end_state, merge, ctl, peaks, hist, fixlist);
    k_best_tail<<<nsm * 8, 256, 0, st>>>(d_records, nt, wa, 1, ck, merge, ctl, peaks, hist);
    for (int level = 0; level < 4; ++level) {  // narrowing passes; no-ops once done
        k_best_plan<<<1, 1024, 0, st>>>(ctl, hist);
        k_best_refix<<<nsm, 256, 0, st>>>(ctl, fixlist, peaks, hist);
        k_best_fix<<<1, 32, 0, st>>>(d_records, nt, wa, 0, ck, end_state, merge, ctl, peaks, hist, fixlist);
        k_best_tail<<<nsm * 8, 256, 0, st>>>(d_records, nt, wa, 0, ck, merge, ctl, peaks, hist);
    }
    k_best_select<<<1, SEL_THREADS, smem, st>>>(d_records, ent, fr_g, fr_c, peaks, ctl, sa, dout);
    FFA_LAUNCH_CHECK("ffa2best kernels");
    count_launch(20);
    ffa_status s = ffa_wait(stream, d_status, timeout_ms);
    if (s != FFA_OK) return s;
    BestCtl h;
    FFA_CUDA_TRY(cudaMemcpy(&h, ctl, sizeof(BestCtl), cudaMemcpyDeviceToHost));
    *n_peaks = (int64_t)h.n_peaks;
    if (!h.done && (!h.emit || h.n_stored > (uint32_t)PEAK_CAP))
        return fail(FFA_ERR_DEVICE, "ffa2best: peak selection did not converge");
    const uint32_t m = std::min<uint32_t>(h.n_kept, (uint32_t)cap);
    if (m > 0) FFA_CUDA_TRY(cudaMemcpy(out, dout, sizeof(ffa_candidate) * m, cudaMemcpyDeviceToHost));
    *n_out = (int32_t)m;
    return FFA_OK;
}
