// Algorithm 1 (Section 2.2.1, Eq. 3-4) on the GPU, one CTA per folded
// profile at a time (persistent over trials), with the last FFA stage
// (Section 2.1) fused into the load.
//
// Layout.  The profile x (p0 bins) is extended cyclically to p0 + wmax bins
// and cut into blocks of R consecutive bins; thread t owns block t in
// registers.  Blocks beyond the first T (the cyclic extension) only take part
// in the prefix step.  The CTA shape (T threads of R bins) follows the
// profile length: 256 x 8 up to 2048 bins (several CTAs per SM), 512 x 16 up
// to 8192, 1024 x 16 up to 16384, 1024 x 32 up to 32768 (one per SM), so that
// short profiles do not leave most of a CTA idle.
//
// Median and MAD (exact).  A monotone bucket function (affine map of the
// value, rounded, clamped) feeds a shared-memory histogram; the
// bucket(s) holding the wanted ranks are gathered and ranked, which gives the
// exact order statistics because a monotone bucket map preserves order
// between buckets.  The MAD reuses that histogram: its prefix counts bound
// how many samples lie within d of the median, so two warps bracket the MAD
// between D1 and D2 and only the samples with D1 < |x - med| <= D2
// (classified exactly, by float bounds of med -+ D taken with directed
// rounding) are gathered and ranked by their exact deviations.  If the band
// misses the wanted ranks, a histogram of the FP32 deviations |x - fl(med)|
// (within E = max|x| * 2^-20 of the exact ones, so one extra bucket on each
// side catches every candidate) takes over; if a gather overflows its
// buffer, an exact radix select over the profile in shared memory does.
// The order statistics travel as integer keys held by every thread; each
// FP64 value of a profile (median, MAD, the S/N factors) is formed once by
// one thread and shared, as FP64 issues at a small fraction of the FP32 rate.
//
// Box sums.  With the in-block exclusive prefix c_t[o] (FP32) and the block
// offsets Cb[t] = sum of earlier blocks (float-float), the cyclic box sum of
// width w >= R starting at bin Rt + o is
//     (Cb[t + w/R] - Cb[t]) + (c_{t+w/R}[o] - c_t[o]),
// one shared-memory read, two adds and a max per bin; widths below R use the
// thread's own prefix and the next block's.  Int profiles use the same
// formulas in wrapping int32 arithmetic, which is exact for box sums below
// 2^31.  Only the maximum of each width is kept; the winning width's first
// argmax is found afterwards by recomputing that width, bit-identically.  The
// block that runs past p0 scores all its bins: its extra boxes are cyclic
// boxes of the first bins again, so no per-bin bound check is needed.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace ffa {

namespace {

// CTA shapes.  A profile of p0 bins is cut into blocks of R bins, one per
// thread; T * R >= p0.  Long profiles take 1024-thread CTAs, one per SM;
// short ones smaller CTAs, several per SM, each on its own profile.  The
// shape is the first of 256 x 8, 512 x 16, 1024 x 16, 1024 x 32 that fits.
template <int TH>
struct Cfg;
template <>
struct Cfg<1024> {
    static constexpr int T = 1024, R = 32, MAXB = 2048, NBK = 2048, CAPM = 1024, MINB = 1;
    static constexpr bool DIST = true;  // int profiles only (see k_score2)
};
template <>
struct Cfg<512> {
    static constexpr int T = 512, R = 16, MAXB = 1024, NBK = 1024, CAPM = 512, MINB = 2;
    static constexpr bool DIST = false;
};
template <>
struct Cfg<256> {
    static constexpr int T = 256, R = 8, MAXB = 512, NBK = 512, CAPM = 512, MINB = 4;
    static constexpr bool DIST = false;
};
// 1024 threads of 16 bins: profiles of 8193..16384 bins, which would leave
// half or more of a 1024 x 32 CTA idle
struct CMid {
    static constexpr int T = 1024, R = 16, MAXB = 2048, NBK = 2048, CAPM = 1024, MINB = 1;
    static constexpr bool DIST = false;
};
using CBig = Cfg<1024>;
constexpr double KMAD = 1.4826;   // printed after Eq. 4

#define FFA_CFG_ALIASES                                   \
    constexpr int T2 = C::T, R2 = C::R, MAXB = C::MAXB;   \
    constexpr int NBK = C::NBK, CAPM = C::CAPM;           \
    constexpr int NW = T2 / 32;                           \
    (void)T2; (void)R2; (void)MAXB; (void)NBK; (void)CAPM; (void)NW;

// Shared-memory index of bin t: 4 pad words per 32-bin block keep every block
// 16-byte aligned (vector loads) and spread blocked accesses over the banks.
__device__ __forceinline__ int sidx(int t) { return t + 4 * (t >> 5); }

template <class C>
struct Sh2 {
    uint32_t hist[C::NBK];
    unsigned long long cand[C::CAPM];  // order-preserving keys of the candidates
    float candf[C::CAPM];    // gathered values; FP64 is applied per candidate afterwards
    double bw_max[16];       // per-width block maxima
    float cbh[C::MAXB + 1];  // block offsets (hi) / int offsets reinterpreted
    float cbl[C::MAXB + 1];  // block offsets (lo)
    float wred[16][32];   // per-width warp maxima (float profiles)
    int wredi[16][32];    // per-width warp maxima (int profiles)
    float fred[32];
    double dred[64];
    int ired[32];
    int ired2[C::CAPM];      // gathered int values
    unsigned long long ukey[2];
    uint32_t cnt, below;
    float mthr[4];  // MAD bracket: |x - med| <= D1 <=> mthr[0] <= x <= mthr[1]; D2: mthr[2], mthr[3]
    long long mthri[4];  // the same bounds for int profiles
    int mok;
    // Per-profile FP64 scalars, computed by one thread and broadcast: FP64
    // issues at a small fraction of the FP32 rate on this part, so a value
    // every thread needs is never recomputed by every thread.
    double smed, skmad;        // median, K * MAD
    float snr_mh, snr_ml, snr_kf;  // float S/N: median as a float pair, fl(K * MAD)
    int madpos;                // MAD > 0
    float bw_maxf[16];         // per-width block maxima (float profiles)
    int bin_a, bin_b;
    uint32_t below_a, below_b;
    uint32_t wkey[16];  // per-width maxima as order-preserving keys (item-distributed widths)
    int phase;
};

// ---- block helpers (T2 threads) --------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Warp maxima in one instruction (redux.sync; the .f32 form is new with the
// sm_100 family).  Inputs here are never NaN; -0 and +0 compare equal in
// every use of the result.
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ int warp_maxi(int v) { return __reduce_max_sync(0xffffffffu, v); }
__device__ __forceinline__ int warp_mini(int v) { return __reduce_min_sync(0xffffffffu, v); }

// block sums of a and b and the max of c (one barrier pair)
template <class C>
__device__ void blk_stats(float& a, float& b, float& c, Sh2<C>& sh) {
    FFA_CFG_ALIASES
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_max(c);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh.fred[w] = a;
        sh.wred[0][w] = b;
        sh.wred[1][w] = c;
    }
    __syncthreads();
    a = warp_sum(l < NW ? sh.fred[l] : 0.0f);
    b = warp_sum(l < NW ? sh.wred[0][l] : 0.0f);
    c = warp_max(l < NW ? sh.wred[1][l] : 0.0f);
    __syncthreads();
}
// The same statistics split around a barrier the caller already has: warp
// partials before it, the block values after it (the partials' slots are
// not written again before the caller's next barrier).
template <class C>
__device__ __forceinline__ void blk_stats_part(float a, float b, float c, Sh2<C>& sh) {
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_max(c);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh.fred[w] = a;
        sh.wred[0][w] = b;
        sh.wred[1][w] = c;
    }
}
template <class C>
__device__ __forceinline__ void blk_stats_fin(float& a, float& b, float& c, const Sh2<C>& sh) {
    FFA_CFG_ALIASES
    const int l = threadIdx.x & 31;
    a = warp_sum(l < NW ? sh.fred[l] : 0.0f);
    b = warp_sum(l < NW ? sh.wred[0][l] : 0.0f);
    c = warp_max(l < NW ? sh.wred[1][l] : 0.0f);
}
template <class C>
__device__ int blk_mini(int v, Sh2<C>& sh) {
    FFA_CFG_ALIASES
    v = warp_mini(v);
    if ((threadIdx.x & 31) == 0) sh.ired[threadIdx.x >> 5] = v;
    __syncthreads();
    const int l = threadIdx.x & 31;
    int r = warp_mini(l < NW ? sh.ired[l] : 0x7fffffff);
    __syncthreads();
    return r;
}

// exclusive scan of one uint32 per thread
template <class C>
__device__ uint32_t blk_exscan_u(uint32_t v, Sh2<C>& sh, uint32_t* total) {
    FFA_CFG_ALIASES
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    uint32_t* s = reinterpret_cast<uint32_t*>(sh.ired);
    if (lane == 31) s[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t y = lane < NW ? s[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += u;
        }
        s[lane] = y;
    }
    __syncthreads();
    uint32_t r = (warp ? s[warp - 1] : 0u) + x - v;
    if (total) *total = s[NW - 1];
    __syncthreads();
    return r;
}

// exclusive scan of float-float values (hi, lo) in block order
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& sh_, float& sl_) {
    float s, e;
    two_sum(ah, bh, s, e);
    e = __fadd_rn(e, __fadd_rn(al, bl));
    float s2 = __fadd_rn(s, e);
    sl_ = __fsub_rn(e, __fsub_rn(s2, s));
    sh_ = s2;
}

template <class C>
__device__ void blk_exscan_ff(float vh, Sh2<C>& sh, float& oh, float& ol, float& th, float& tl) {
    FFA_CFG_ALIASES
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float xh = vh, xl = 0.0f;
    for (int o = 1; o < 32; o <<= 1) {
        float uh = __shfl_up_sync(0xffffffffu, xh, o);
        float ul = __shfl_up_sync(0xffffffffu, xl, o);
        if (lane >= o) ff_add(xh, xl, uh, ul, xh, xl);
    }
    // inclusive warp result in (xh, xl)
    if (lane == 31) {
        sh.fred[warp] = xh;
        sh.wred[0][warp] = xl;
    }
    __syncthreads();
    if (warp == 0) {
        float yh = lane < NW ? sh.fred[lane] : 0.0f, yl = lane < NW ? sh.wred[0][lane] : 0.0f;
        for (int o = 1; o < 32; o <<= 1) {
            float uh = __shfl_up_sync(0xffffffffu, yh, o);
            float ul = __shfl_up_sync(0xffffffffu, yl, o);
            if (lane >= o) ff_add(yh, yl, uh, ul, yh, yl);
        }
        sh.fred[lane] = yh;
        sh.wred[0][lane] = yl;
    }
    __syncthreads();
    float bh = warp ? sh.fred[warp - 1] : 0.0f, bl = warp ? sh.wred[0][warp - 1] : 0.0f;
    // exclusive = base + inclusive - own  ->  compute base + (inclusive warp prefix excluding own)
    float eh, el;
    {
        float ph = __shfl_up_sync(0xffffffffu, xh, 1), pl = __shfl_up_sync(0xffffffffu, xl, 1);
        if (lane == 0) {
            ph = 0.0f;
            pl = 0.0f;
        }
        ff_add(bh, bl, ph, pl, eh, el);
    }
    oh = eh;
    ol = el;
    th = sh.fred[NW - 1];
    tl = sh.wred[0][NW - 1];
    __syncthreads();
}

// ranks ra <= rb -> their bins and the counts below those bins, one scan.
// PREFIX: also leave in hist[b] the count of every bin before b.
template <bool PREFIX = false, class C>
__device__ void blk_find2(Sh2<C>& sh, uint32_t ra, uint32_t rb) {
    FFA_CFG_ALIASES
    const int per = NBK / T2;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int t = 0; t < per; ++t) s += sh.hist[b0 + t];
    const uint32_t ex = blk_exscan_u(s, sh, nullptr);
    uint32_t c = ex;
    for (int t = 0; t < per; ++t) {
        const uint32_t h = sh.hist[b0 + t];
        if (ra >= c && ra < c + h) {
            sh.bin_a = b0 + t;
            sh.below_a = c;
        }
        if (rb >= c && rb < c + h) {
            sh.bin_b = b0 + t;
            sh.below_b = c;
        }
        if (PREFIX) sh.hist[b0 + t] = c;  // each thread rewrites only the bins it read
        c += h;
    }
    __syncthreads();
}

// single-rank variant (radix fallback)
template <class C>
__device__ void blk_find(Sh2<C>& sh, uint32_t rank, int* bin, uint32_t* below) {
    blk_find2(sh, rank, rank);
    *bin = sh.bin_a;
    *below = sh.below_a;
    __syncthreads();
}

// Keys of ranks ta <= tb among the keys sh.cand[0..n) (ties broken by index):
// the n x n integer comparisons are spread over the whole CTA and each
// candidate's rank is accumulated in shared memory.  Integer keys, not
// doubles: FP64 compares are slow on this part.  The rank counters live in
// ired2 (the int gather buffer, already turned into keys), so the median
// histogram stays intact for the MAD bracket; ZEROED: the caller cleared
// counters 0..n) before its last barrier.  Every caller passes a barrier
// before it writes cand, ired2 or ukey again.
template <bool ZEROED = false, class C>
__device__ void cand_pick2(Sh2<C>& sh, uint32_t n, uint32_t ta, uint32_t tb, unsigned long long* ka,
                           unsigned long long* kb) {
    FFA_CFG_ALIASES
    uint32_t* rank = reinterpret_cast<uint32_t*>(sh.ired2);
    if (!ZEROED) {
        for (uint32_t i = threadIdx.x; i < n; i += T2) rank[i] = 0;
        __syncthreads();
    }
    const uint32_t chunks = (T2 + n - 1) / (n ? n : 1);  // threads per candidate
    const uint32_t pairs = n * chunks;
    for (uint32_t p = threadIdx.x; p < pairs; p += T2) {
        const uint32_t i = p % n, part = p / n;
        const unsigned long long ci = sh.cand[i];
        uint32_t rk = 0;
        for (uint32_t j = part; j < n; j += chunks) {
            const unsigned long long cj = sh.cand[j];
            rk += (cj < ci) || (cj == ci && j < i);
        }
        if (rk) atomicAdd(&rank[i], rk);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += T2) {
        const uint32_t rk = rank[i];
        if (rk == ta) sh.ukey[0] = sh.cand[i];
        if (rk == tb) sh.ukey[1] = sh.cand[i];
    }
    __syncthreads();
    *ka = sh.ukey[0];
    *kb = sh.ukey[1];
}

// Exact rank-`rank` 64-bit key of keyf(j), j < n, by an 8-pass radix select
// over the profile still held in shared memory (fallback when a gather
// overflows; rare).
template <class C, class KeyF>
__device__ __noinline__ uint64_t smem_select64(Sh2<C>& sh, int n, uint32_t rank, KeyF keyf) {
    FFA_CFG_ALIASES
    uint64_t prefix = 0, mask = 0;
    for (int pass = 0; pass < 8; ++pass) {
        const int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < NBK; b += T2) sh.hist[b] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += T2) {
            const uint64_t kk = keyf(j);
            if ((kk & mask) == prefix) atomicAdd(&sh.hist[(kk >> shift) & 0xff], 1u);
        }
        __syncthreads();
        blk_find(sh, rank, &sh.bin_a, &sh.below_a);
        rank -= sh.below_a;
        prefix |= (uint64_t)sh.bin_a << shift;
        mask |= (uint64_t)0xff << shift;
        __syncthreads();
    }
    return prefix;
}

template <class T>
struct Traits;
template <>
struct Traits<float> {
    static constexpr bool is_int = false;
};
template <>
struct Traits<int32_t> {
    static constexpr bool is_int = true;
};

// bucket of a float value: rint((v - base) * inv + NBK/2) clamped, monotone in v
template <int NBK>
__device__ __forceinline__ int fbucket(float v, float base, float inv) {
    float f = __fmaf_rn(__fsub_rn(v, base), inv, (float)(NBK / 2));
    f = fminf(fmaxf(f, 0.0f), (float)(NBK - 1));
    return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000;
}
// int profiles (|x| < 2^28): floor((v - base) / 2^sh) + NBK/2, clamped; monotone
template <int NBK>
__device__ __forceinline__ int ibucket(int v, int base, int sh) {
    const int d = ((v - base) >> sh) + NBK / 2;  // arithmetic shift = floor division
    return d < 0 ? 0 : (d > NBK - 1 ? NBK - 1 : d);
}

}  // namespace

// Box-sum helpers.  C(32t + o) = Cb[t] + c_t[o]; a box of width w at bin
// 32t + r is C(32t + r + w) - C(32t + r).
template <class T>
struct BoxOps;
template <>
struct BoxOps<float> {
    template <class C>
    static __device__ __forceinline__ float blockdiff(const Sh2<C>& sh, int b2, int b1) {
        return __fadd_rn(__fsub_rn(sh.cbh[b2], sh.cbh[b1]), __fsub_rn(sh.cbl[b2], sh.cbl[b1]));
    }
    static __device__ __forceinline__ float box(float D, float c2, float c1) {
        return __fadd_rn(D, __fsub_rn(c2, c1));
    }
    static __device__ __forceinline__ float diff(float c2, float c1) { return __fsub_rn(c2, c1); }
    static __device__ __forceinline__ float lowest() { return -INFINITY; }
};
template <>
struct BoxOps<int32_t> {
    template <class C>
    static __device__ __forceinline__ int32_t blockdiff(const Sh2<C>& sh, int b2, int b1) {
        const int* cbi = reinterpret_cast<const int*>(sh.cbh);
        return (int32_t)((uint32_t)cbi[b2] - (uint32_t)cbi[b1]);
    }
    static __device__ __forceinline__ int32_t box(int32_t D, int32_t c2, int32_t c1) {
        return (int32_t)((uint32_t)D + ((uint32_t)c2 - (uint32_t)c1));
    }
    static __device__ __forceinline__ int32_t diff(int32_t c2, int32_t c1) {
        return (int32_t)((uint32_t)c2 - (uint32_t)c1);
    }
    static __device__ __forceinline__ int32_t lowest() { return INT32_MIN; }
};

// Width W < 32 (compile time): own prefix, next block past the end.  With
// FIND, returns the first position whose box equals `target` (else -1).
template <class T, int W, bool FIND, class C>
__device__ __forceinline__ T small_width(const T (&c)[C::R], const Sh2<C>& sh, const T* buf, int tid,
                                         int nvalid, T target, int* first) {
    FFA_CFG_ALIASES
    using B = BoxOps<T>;
    const T Town = B::blockdiff(sh, tid + 1, tid);
    constexpr int NC = W < 4 ? 4 : W;  // next block's first values, 128-bit loads
    T cn[NC];
    const T* nb = buf + sidx((tid + 1) * R2);
#pragma unroll
    for (int k = 0; k < NC; k += 4) *reinterpret_cast<int4*>(&cn[k]) = *reinterpret_cast<const int4*>(nb + k);
    T m0 = B::lowest(), m1 = B::lowest();
#pragma unroll
    for (int r = 0; r < R2; ++r) {
        T bx;
        if (r + W < R2) bx = B::diff(c[r + W], c[r]);
        else bx = B::box(Town, cn[r + W - R2], c[r]);
        if (r < nvalid) {
            if (r & 1) m1 = bx > m1 ? bx : m1;
            else m0 = bx > m0 ? bx : m0;
            if (FIND && *first < 0 && bx == target) *first = r;
        }
    }
    return m0 > m1 ? m0 : m1;
}

// Width w >= 32 (multiple of 32): block tid + w/32 at the same offsets.
template <class T, bool FIND, class C>
__device__ __forceinline__ T wide_width(const T (&c)[C::R], const Sh2<C>& sh, const T* buf, int tid,
                                        int w, int nvalid, T target, int* first) {
    FFA_CFG_ALIASES
    using B = BoxOps<T>;
    const int b2 = tid + w / R2;
    const T D = B::blockdiff(sh, b2, tid);
    const T* cb = buf + sidx(b2 * R2);  // block b2's bins are contiguous, 16-byte aligned
    T m = B::lowest();
#pragma unroll
    for (int r = 0; r < R2; r += 4) {
        T c2[4];
        *reinterpret_cast<int4*>(c2) = *reinterpret_cast<const int4*>(cb + r);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const T bx = B::box(D, c2[i], c[r + i]);
            if (r + i < nvalid) {
                m = bx > m ? bx : m;
                if (FIND && *first < 0 && bx == target) *first = r + i;
            }
        }
    }
    return m;
}

__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

// Wide widths, float profiles, maxima only: the same per-bin arithmetic as
// wide_width (D + (c2 - c1), each rounded to nearest) on packed pairs.
template <class C>
__device__ __forceinline__ float wide_width_f32x2(const float (&c)[C::R], const Sh2<C>& sh, const float* buf,
                                                  int tid, int w, int nvalid) {
    FFA_CFG_ALIASES
    const int b2 = tid + w / R2;
    const float D = BoxOps<float>::blockdiff(sh, b2, tid);
    const unsigned long long DD = pk2(D, D);
    const float* cb = buf + sidx(b2 * R2);
    float m = -INFINITY, ma = -INFINITY;
#pragma unroll
    for (int r = 0; r < R2; r += 4) {
        const float4 c2 = *reinterpret_cast<const float4*>(cb + r);
        unsigned long long s01, s23, b01, b23;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s01) : "l"(pk2(c2.x, c2.y)), "l"(pk2(c[r], c[r + 1])));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(s23) : "l"(pk2(c2.z, c2.w)), "l"(pk2(c[r + 2], c[r + 3])));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(b01) : "l"(DD), "l"(s01));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(b23) : "l"(DD), "l"(s23));
        float v0, v1, v2, v3;
        upk2(b01, v0, v1);
        upk2(b23, v2, v3);
        if (r + 0 < nvalid) m = fmaxf(m, v0);
        if (r + 1 < nvalid) ma = fmaxf(ma, v1);
        if (r + 2 < nvalid) m = fmaxf(m, v2);
        if (r + 3 < nvalid) ma = fmaxf(ma, v3);
    }
    return fmaxf(m, ma);
}

template <class T, bool FIND, class C>
__device__ __forceinline__ T width_max(const T (&c)[C::R], const Sh2<C>& sh, const T* buf, int tid, int w,
                                       int nvalid, T target, int* first) {
    if (w < C::R) {
        switch (w) {
            case 1: return small_width<T, 1, FIND>(c, sh, buf, tid, nvalid, target, first);
            case 2: return small_width<T, 2, FIND>(c, sh, buf, tid, nvalid, target, first);
            case 4: return small_width<T, 4, FIND>(c, sh, buf, tid, nvalid, target, first);
            case 8:
                if constexpr (8 < C::R) return small_width<T, 8, FIND>(c, sh, buf, tid, nvalid, target, first);
                break;
            case 16:
                if constexpr (16 < C::R) return small_width<T, 16, FIND>(c, sh, buf, tid, nvalid, target, first);
                break;
            default: break;
        }
    }
    if constexpr (!FIND && !Traits<T>::is_int) return wide_width_f32x2(c, sh, buf, tid, w, nvalid);
    else return wide_width<T, FIND>(c, sh, buf, tid, w, nvalid, target, first);
}

// The base periods scored by one launch: records [t0[i], t0[i + 1]) belong
// to entry i, whose profiles have p0[i] bins and whose plane starts at
// element off[i] of `prof` with rows ld[i] elements apart (all share m_rows
// and the widths); record it of entry i goes to rec[i][it - t0[i]].  A
// single base period is a group of one.  Entries may come from different
// series (a batch): each has its own records.
struct ScoreGroup {
    int32_t n;
    int64_t t0[FOLD_GROUP_MAX + 1];
    int32_t p0[FOLD_GROUP_MAX];
    int64_t off[FOLD_GROUP_MAX];
    int64_t ld[FOLD_GROUP_MAX];
    ffa_record* rec[FOLD_GROUP_MAX];
};

__device__ __forceinline__ int score_entry(const ScoreGroup& g, int64_t it) {
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.t0[mid] <= it) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// prof: FUSED ? the stage-(m-1) planes (m_rows rows of p0 each) : profiles of
// p0.  Record it (< count) belongs to trial trial0 + it - t0[i] of entry i.
template <class C, class T, bool FUSED>
__global__ void __launch_bounds__(C::T, C::MINB) k_score2(const T* __restrict__ prof_all, const ScoreGroup sg,
                                                          int64_t m_rows, int64_t trial0, int64_t count,
                                                          ScoreWidths wd, int32_t* d_status) {
    FFA_CFG_ALIASES
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sh2<C>& sh = *reinterpret_cast<Sh2<C>*>(smem_raw);
    T* buf = reinterpret_cast<T*>(smem_raw + ((sizeof(Sh2<C>) + 15) & ~(size_t)15));
    using B = BoxOps<T>;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int wmax = wd.w[wd.n - 1];
    // persistent: this CTA scores trials it, it + gridDim.x, ...
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
    const int ei = score_entry(sg, it);
    const int64_t p0_ = sg.p0[ei];
    const int p0 = (int)p0_;
    const T* __restrict__ prof = prof_all + sg.off[ei];
    const int nbe = (p0 + wmax + R2) / R2 + 1;  // blocks incl. the cyclic extension
    const int64_t k = trial0 + (it - sg.t0[ei]);
    {
        // pull the next trial's rows towards L2 while this one is scored
        if (it + gridDim.x < count) {
            const int64_t itn = it + gridDim.x;
            const int en = score_entry(sg, itn);
            const int64_t pn = sg.p0[en], ln = sg.ld[en];
            const T* prn = prof_all + sg.off[en];
            const int64_t kn = trial0 + (itn - sg.t0[en]);
            const T* nh = FUSED ? (m_rows > 1 ? prn + (kn >> 1) * ln : prn) : prn + kn * ln;
            const T* nt = (FUSED && m_rows > 1) ? prn + ((m_rows >> 1) + (kn >> 1)) * ln : nullptr;
            const int lines = (int)((pn * (int64_t)sizeof(T) + 127) / 128);
            for (int l = tid; l < lines; l += T2) {
                asm volatile("prefetch.global.L2 [%0];" ::"l"(nh + l * (128 / sizeof(T))));
                if (nt) asm volatile("prefetch.global.L2 [%0];" ::"l"(nt + l * (128 / sizeof(T))));
            }
        }
    }

    // ---- load; fused last FFA stage: head row k>>1 plus tail row M/2 + (k>>1)
    // read ceil(k/2) bins further on
    const T* hrow;
    const T* trow = nullptr;
    int sft = 0;
    const int64_t ld_ = sg.ld[ei];
    if (FUSED && m_rows > 1) {
        hrow = prof + (k >> 1) * ld_;
        trow = prof + ((m_rows >> 1) + (k >> 1)) * ld_;
        sft = (int)((uint32_t)((k + 1) >> 1) % (uint32_t)p0);
    } else if (FUSED) {
        hrow = prof;
    } else {
        hrow = prof + k * ld_;
    }
    // the sum, sum of squares and largest |x| (they only scale the median's
    // buckets) accumulate as the profile is loaded
    float fs = 0.0f, fq = 0.0f, famax = 0.0f;
    auto acc = [&](T v) {
        const float f = (float)v;
        fs += f;
        fq = fmaf(f, f, fq);
        famax = fmaxf(famax, fabsf(f));
    };
    if (trow) {
        // the tail row read from column sft on: two contiguous runs
        const int n1 = p0 - sft;
#pragma unroll 4
        for (int j = tid; j < p0; j += T2) {
            const T t = j < n1 ? trow[j + sft] : trow[j - n1];
            const T v = hrow[j] + t;
            buf[sidx(j)] = v;
            acc(v);
        }
    } else {
#pragma unroll 4
        for (int j = tid; j < p0; j += T2) {
            const T v = hrow[j];
            buf[sidx(j)] = v;
            acc(v);
        }
    }
    blk_stats_part(fs, fq, famax, sh);
    __syncthreads();
    blk_stats_fin(fs, fq, famax, sh);
    T x[R2];
    const int base_pos = tid * R2;
    int nvalid = p0 - base_pos;
    nvalid = nvalid < 0 ? 0 : (nvalid > R2 ? R2 : nvalid);
    {
        const T* blk = buf + sidx(base_pos);
#pragma unroll
        for (int r = 0; r < R2; r += 4) {
            T v4[4];
            *reinterpret_cast<int4*>(v4) = *reinterpret_cast<const int4*>(blk + r);
#pragma unroll
            for (int i = 0; i < 4; ++i) x[r + i] = (r + i < nvalid) ? v4[i] : (T)0;
        }
    }

    // ---- median (Eq. 3), exact ----
    const uint32_t r1 = (uint32_t)((p0 - 1) / 2), r2 = (uint32_t)(p0 / 2);
    const float mean = fs / (float)p0;
    const float msq = fq / (float)p0;
    const float amax = famax;
    float sig = sqrtf(fmaxf(msq - mean * mean, 0.0f));
    if (!(sig > 0.0f)) sig = fmaxf(amax, 1.0f);

    for (int b = tid; b < NBK; b += T2) sh.hist[b] = 0;
    if (tid == 0) {
        sh.cnt = 0;
        sh.below = 0;
    }
    __syncthreads();
    const float inv_m = (float)NBK / (8.0f * sig);
    int ish = 0;
    int ibase = 0;
    if constexpr (Traits<T>::is_int) {
        ibase = (int)floorf(mean);
        // bucket width 2^ish: the power of two nearest to span = 8 sig / NBK
        // (the float buckets' width), within a factor sqrt(2) of it, so the
        // median's bucket holds about as many samples as a float profile's;
        // from the exponent and mantissa bits (span is exact in FP32: NBK is a
        // power of two), without the FP64 that every thread would otherwise
        // issue for every profile.  Any width gives a monotone bucket map.
        const float span = 8.0f * sig / (float)NBK;
        if (span > 1.0f) {
            const uint32_t b = __float_as_uint(span);
            ish = (int)((b >> 23) & 0xffu) - 127 + ((b & 0x7fffffu) > 0x3504f3u ? 1 : 0);  // 0x3504f3: sqrt(2)'s
            ish = ish < 40 ? ish : 40;
        }
    }
    auto bucket_m = [&](T v) -> int {
        if constexpr (Traits<T>::is_int) return ibucket<NBK>((int)v, ibase, ish);
        else return fbucket<NBK>((float)v, mean, inv_m);
    };
    if (nvalid > 0) {
#pragma unroll
        for (int r = 0; r < R2; ++r)
            if (r < nvalid) atomicAdd(&sh.hist[bucket_m(x[r])], 1u);
    }
    __syncthreads();
    blk_find2<true>(sh, r1, r2);  // hist becomes the prefix counts of the bins
    const int mb1 = sh.bin_a, mb2 = sh.bin_b;
    const uint32_t mbelow = sh.below_a;
    if (nvalid > 0) {
#pragma unroll
        for (int r = 0; r < R2; ++r)
            if (r < nvalid) {
                int b = bucket_m(x[r]);
                if (b >= mb1 && b <= mb2) {
                    uint32_t s = atomicAdd(&sh.cnt, 1u);
                    if (s < CAPM) {
                        if constexpr (Traits<T>::is_int) sh.ired2[s] = (int)x[r];
                        else sh.candf[s] = (float)x[r];
                    }
                }
            }
    }
    __syncthreads();
    // The two middle order statistics come out as keys (mka, mkb) in every
    // thread.  Every thread decodes what it needs without FP64: 2 * median
    // for int profiles (exact), fl(median) for float ones (it only guides the
    // MAD search).  The exact FP64 median is formed once (med_of), by the
    // last thread while the first warps search, and read from sh.smed after
    // the next barrier.
    unsigned long long mka = 0, mkb = 0;
    long long s2m = 0;  // int profiles: 2 * median
    float medf = 0.0f;  // float profiles: fl(median)
    auto med_of = [&]() -> double {
        double a, b;
        if constexpr (Traits<T>::is_int) {
            a = (double)(int32_t)((uint32_t)mka ^ 0x80000000u);
            b = (double)(int32_t)((uint32_t)mkb ^ 0x80000000u);
        } else {
            a = (double)fkey_inv((uint32_t)mka);
            b = (double)fkey_inv((uint32_t)mkb);
        }
        return (r1 == r2) ? a : (a + b) / 2;
    };
    bool med_hist;  // the median came from the histogram (its prefix counts are in hist)
    {
        const uint32_t cc = sh.cnt;
        med_hist = cc <= CAPM;
        for (uint32_t i = tid; i < cc && i < CAPM; i += T2) {
            if constexpr (Traits<T>::is_int) sh.cand[i] = ikey(sh.ired2[i]);
            else sh.cand[i] = fkey(sh.candf[i]);
            reinterpret_cast<uint32_t*>(sh.ired2)[i] = 0;  // rank counter (value read above)
        }
        __syncthreads();
        if (cc <= CAPM) {
            cand_pick2<true>(sh, cc, r1 - mbelow, r2 - mbelow, &mka, &mkb);
        } else {
            const T* vb = buf;
            auto key = [vb](int j) -> uint64_t {
                if constexpr (Traits<T>::is_int) return (uint64_t)ikey((int32_t)vb[sidx(j)]);
                else return (uint64_t)fkey((float)vb[sidx(j)]);
            };
            mka = smem_select64(sh, p0, r1, key);
            mkb = (r1 == r2) ? mka : smem_select64(sh, p0, r2, key);
        }
        if constexpr (Traits<T>::is_int) {
            const long long a = (int32_t)((uint32_t)mka ^ 0x80000000u);
            const long long b = (int32_t)((uint32_t)mkb ^ 0x80000000u);
            s2m = (r1 == r2) ? 2 * a : a + b;
        } else {
            const float a = fkey_inv((uint32_t)mka), b = fkey_inv((uint32_t)mkb);
            medf = (r1 == r2) ? a : __fmul_rn(__fadd_rn(a, b), 0.5f);
        }
        __syncthreads();
        if (tid == T2 - 1) sh.smed = med_of();
    }

    // ---- MAD (Eq. 3), exact ----
    // The two order statistics of the deviations come out as keys (mk1, mk2)
    // in every thread: exact integers e = |2x - 2 med| for int profiles,
    // FP64 keys (dkey) of |x - med| for float ones; the MAD itself is formed
    // once, with the S/N factors, before the widths.
    bool mad_done = false;  // block-uniform
    unsigned long long mk1 = 0, mk2 = 0;
    if constexpr (Traits<T>::is_int) {
        // The same bracket in integers: the deviation is e / 2 with the exact
        // integer e = |2x - s2| (s2 = 2 med), and |2x - s2| <= E exactly when
        // ceil((s2 - E) / 2) <= x <= floor((s2 + E) / 2).
        if (med_hist) {
            const long long s2 = s2m;
            const long long estep = 1ll << ish;  // half a bucket in units of e
            if (warp < 2) {
                const int K = NBK;
                auto pb = [&](int b) -> uint32_t { return b >= NBK ? (uint32_t)p0 : sh.hist[b]; };
                auto clampi = [](long long v) -> int {
                    return v < INT32_MIN ? INT32_MIN : (v > INT32_MAX ? INT32_MAX : (int)v);
                };
                auto lu = [&](int k, uint32_t& L, uint32_t& U) {
                    const long long E = (long long)k * estep;
                    const long long xl = (s2 - E + 1) >> 1, xh = (s2 + E) >> 1;  // ceil, floor
                    const int bl = ibucket<NBK>(clampi(xl), ibase, ish);
                    const int bh = ibucket<NBK>(clampi(xh), ibase, ish);
                    U = xl <= xh ? pb(bh + 1) - pb(bl) : 0u;
                    L = bh - 1 >= bl + 1 ? pb(bh) - pb(bl + 1) : 0u;
                };
                auto first_true = [&](auto pred) -> int {
                    int a = 0, b = K + 1;
                    while (a < b) {
                        const int step = (b - a + 31) / 32;
                        const int k = a + lane * step;
                        const unsigned m = __ballot_sync(0xffffffffu, k < b && pred(k));
                        if (m == 0) {
                            a = min(b, a + 32 * step);
                        } else {
                            const int f = __ffs(m) - 1;
                            b = a + f * step;
                            a = f == 0 ? a : a + (f - 1) * step + 1;
                        }
                    }
                    return b;
                };
                if (warp == 0) {
                    const int kA = first_true([&](int k) {
                        uint32_t L, U;
                        lu(k, L, U);
                        return U > r1;
                    }) - 1;
                    if (lane == 0) {
                        if (kA >= 0) {
                            const long long E1 = (long long)kA * estep;
                            sh.mthri[0] = (s2 - E1 + 1) >> 1;
                            sh.mthri[1] = (s2 + E1) >> 1;
                        } else {
                            sh.mthri[0] = 1;
                            sh.mthri[1] = 0;  // empty
                        }
                    }
                } else {
                    const int kB = first_true([&](int k) {
                        uint32_t L, U;
                        lu(k, L, U);
                        return L >= r2 + 1;
                    });
                    if (lane == 0) {
                        sh.mok = kB <= K;
                        const long long E2 = (long long)(kB <= K ? kB : K) * estep;
                        sh.mthri[2] = (s2 - E2 + 1) >> 1;
                        sh.mthri[3] = (s2 + E2) >> 1;
                    }
                }
            }
            if (tid == 0) {
                sh.cnt = 0;
                sh.below = 0;
            }
            __syncthreads();
            if (sh.mok) {
                // The profile values are int32, so each interval [lo, hi] is
                // applied as the int32 interval it contains (empty when it
                // holds no int32): the same classification in 32-bit compares.
                int l1, h1, l2, h2;
                auto narrow = [](long long lo, long long hi, int& l, int& h) {
                    if (lo > hi || lo > INT32_MAX || hi < INT32_MIN) {
                        l = 1;
                        h = 0;
                    } else {
                        l = lo < INT32_MIN ? INT32_MIN : (int)lo;
                        h = hi > INT32_MAX ? INT32_MAX : (int)hi;
                    }
                };
                narrow(sh.mthri[0], sh.mthri[1], l1, h1);
                narrow(sh.mthri[2], sh.mthri[3], l2, h2);
                uint32_t nbel = 0;
                if (nvalid > 0) {
#pragma unroll
                    for (int r = 0; r < R2; ++r)
                        if (r < nvalid) {
                            const int v = (int)x[r];
                            if (v >= l1 && v <= h1) {
                                ++nbel;
                            } else if (v >= l2 && v <= h2) {
                                const uint32_t q = atomicAdd(&sh.cnt, 1u);
                                const long long e = 2 * (long long)v - s2;
                                if (q < CAPM) sh.cand[q] = (unsigned long long)(e < 0 ? -e : e);
                            }
                        }
                }
                nbel = __reduce_add_sync(0xffffffffu, nbel);
                if (lane == 0 && nbel) atomicAdd(&sh.below, nbel);
                __syncthreads();
                const uint32_t cc = sh.cnt, cb = sh.below;
                if (cc <= CAPM && cb <= r1 && r2 - cb < cc) {
                    cand_pick2(sh, cc, r1 - cb, r2 - cb, &mk1, &mk2);
                    mad_done = true;
                }
                __syncthreads();
            }
        }
    }
    if constexpr (!Traits<T>::is_int) {
        // Bracket from the median histogram.  With B the (monotone) bucket map
        // and N(d) = #{x : |x - med| <= d}, every such x has B(lo) <= B(x) <=
        // B(hi) for lo, hi = med -+ d rounded to float, and every x with
        // B(lo) < B(x) < B(hi) is such an x; the prefix counts of the buckets
        // give U(d) >= N(d) >= L(d).  So the r1-th smallest deviation exceeds
        // any d with U(d) <= r1 (D1) and the r2-th is at most any d with
        // L(d) > r2 (D2): only samples with D1 < |x - med| <= D2 are gathered,
        // classified exactly by float bounds of med -+ D (directed rounding).
        if (med_hist) {
            if (warp < 2) {  // warp 0 finds D1, warp 1 finds D2
                // The search only chooses D1 and D2 (in FP32; any choice is
                // correct): the classification below is exact for the chosen
                // values and the rank check falls back if the band misses.
                const float hstep = 0.5f / inv_m;  // half a bucket
                const int K = NBK;                 // d up to 4 sigma
                auto pb = [&](int b) -> uint32_t { return b >= NBK ? (uint32_t)p0 : sh.hist[b]; };
                auto lu = [&](int k, uint32_t& L, uint32_t& U) {
                    const float d = (float)k * hstep;
                    const int bl = fbucket<NBK>(medf - d, mean, inv_m);
                    const int bh = fbucket<NBK>(medf + d, mean, inv_m);
                    U = pb(bh + 1) - pb(bl);
                    L = bh - 1 >= bl + 1 ? pb(bh) - pb(bl + 1) : 0u;
                };
                // first k in [0, K] where a monotone predicate holds (K + 1: none)
                auto first_true = [&](auto pred) -> int {
                    int a = 0, b = K + 1;
                    while (a < b) {
                        const int step = (b - a + 31) / 32;
                        const int k = a + lane * step;
                        const unsigned m = __ballot_sync(0xffffffffu, k < b && pred(k));
                        if (m == 0) {
                            a = min(b, a + 32 * step);
                        } else {
                            const int f = __ffs(m) - 1;
                            b = a + f * step;
                            a = f == 0 ? a : a + (f - 1) * step + 1;
                        }
                    }
                    return b;
                };
                if (warp == 0) {
                    const int kA = first_true([&](int k) {
                        uint32_t L, U;
                        lu(k, L, U);
                        return U > r1;
                    }) - 1;
                    if (lane == 0) {
                        if (kA >= 0) {
                            const double med = med_of();
                            const double d1 = (double)((float)kA * hstep);
                            sh.mthr[0] = __double2float_ru(__dsub_ru(med, d1));
                            sh.mthr[1] = __double2float_rd(__dadd_rd(med, d1));
                        } else {
                            sh.mthr[0] = INFINITY;
                            sh.mthr[1] = -INFINITY;
                        }
                    }
                } else {
                    const int kB = first_true([&](int k) {
                        uint32_t L, U;
                        lu(k, L, U);
                        return L >= r2 + 1;
                    });
                    if (lane == 0) {
                        sh.mok = kB <= K;
                        const double med = med_of();
                        const double d2 = (double)((float)(kB <= K ? kB : K) * hstep);
                        sh.mthr[2] = __double2float_ru(__dsub_ru(med, d2));
                        sh.mthr[3] = __double2float_rd(__dadd_rd(med, d2));
                    }
                }
            }
            if (tid == 0) {
                sh.cnt = 0;
                sh.below = 0;
            }
            __syncthreads();
            if (sh.mok) {
                const float l1 = sh.mthr[0], h1 = sh.mthr[1], l2 = sh.mthr[2], h2 = sh.mthr[3];
                uint32_t nbel = 0;
                if (nvalid > 0) {
#pragma unroll
                    for (int r = 0; r < R2; ++r)
                        if (r < nvalid) {
                            const float v = (float)x[r];
                            if (v >= l1 && v <= h1) {
                                ++nbel;
                            } else if (v >= l2 && v <= h2) {
                                const uint32_t q = atomicAdd(&sh.cnt, 1u);
                                if (q < CAPM) sh.candf[q] = v;
                            }
                        }
                }
                nbel = __reduce_add_sync(0xffffffffu, nbel);
                if (lane == 0 && nbel) atomicAdd(&sh.below, nbel);
                __syncthreads();
                const uint32_t cc = sh.cnt, cb = sh.below;
                if (cc <= CAPM && cb <= r1 && r2 - cb < cc) {
                    const double med = sh.smed;
                    for (uint32_t i = tid; i < cc; i += T2) {
                        sh.cand[i] = dkey(fabs((double)sh.candf[i] - med));
                        reinterpret_cast<uint32_t*>(sh.ired2)[i] = 0;  // rank counter
                    }
                    __syncthreads();
                    cand_pick2<true>(sh, cc, r1 - cb, r2 - cb, &mk1, &mk2);
                    mad_done = true;
                }
                __syncthreads();
            }
        }
    }
    if (!mad_done) {
    for (int b = tid; b < NBK; b += T2) sh.hist[b] = 0;
    if (tid == 0) {
        sh.cnt = 0;
        sh.below = 0;
    }
    __syncthreads();
    const double med = sh.smed;  // written before this barrier
    if constexpr (Traits<T>::is_int) {
        // e = |2x - (a + b)| is exact; the deviation is e / 2
        const int s2 = (int)s2m;
        int esh = 0;
        const double span = 8.0 * (double)sig / (double)NBK;
        while ((double)(1ll << esh) < span && esh < 40) ++esh;
        auto eval = [&](T v) -> int {
            const int e = 2 * (int)v - s2;
            return e < 0 ? -e : e;
        };
        auto eb = [&](int e) -> int {
            const int b = e >> esh;
            return b > NBK - 1 ? NBK - 1 : b;
        };
        if (nvalid > 0) {
#pragma unroll
            for (int r = 0; r < R2; ++r)
                if (r < nvalid) atomicAdd(&sh.hist[eb(eval(x[r]))], 1u);
        }
        __syncthreads();
        blk_find2(sh, r1, r2);
        const int c1 = sh.bin_a, c2 = sh.bin_b;
        const uint32_t cbel = sh.below_a;
        if (nvalid > 0) {
#pragma unroll
            for (int r = 0; r < R2; ++r)
                if (r < nvalid) {
                    const int e = eval(x[r]);
                    const int b = eb(e);
                    if (b >= c1 && b <= c2) {
                        uint32_t s = atomicAdd(&sh.cnt, 1u);
                        if (s < CAPM) sh.cand[s] = (unsigned long long)(uint32_t)e;
                    }
                }
        }
        __syncthreads();
        const uint32_t cc = sh.cnt;
        if (cc <= CAPM) {
            cand_pick2(sh, cc, r1 - cbel, r2 - cbel, &mk1, &mk2);
        } else {
            const T* vb = buf;
            auto key = [vb, s2](int j) -> uint64_t {
                const int e = 2 * (int)vb[sidx(j)] - s2;
                return (uint64_t)(uint32_t)(e < 0 ? -e : e);
            };
            mk1 = smem_select64(sh, p0, r1, key);
            mk2 = (r1 == r2) ? mk1 : smem_select64(sh, p0, r2, key);
        }
        __syncthreads();
    } else {
        const float m32 = __double2float_rn(med);
        const float E = ldexpf(amax, -20);
        const float inv_d = (float)NBK / (4.0f * sig);
        auto dt = [&](T v) -> float { return fabsf(__fsub_rn((float)v, m32)); };
        auto db = [&](float d) -> int {
            const float f = fminf(__fmul_rn(d, inv_d), (float)(NBK - 1));
            return __float_as_int(__fadd_rn(f, 12582912.0f)) - 0x4B400000;
        };
        if (nvalid > 0) {
#pragma unroll
            for (int r = 0; r < R2; ++r)
                if (r < nvalid) atomicAdd(&sh.hist[db(dt(x[r]))], 1u);
        }
        __syncthreads();
        blk_find2(sh, r1, r2);
        // one extra bucket on each side (more if 3E spans buckets) holds every
        // sample whose exact deviation can be the MAD
        const int marg = 1 + (int)ceilf(3.0f * E * inv_d);
        const int c1 = sh.bin_a - marg, c2 = sh.bin_b + marg;
        uint32_t nbel = 0;
        if (nvalid > 0) {
#pragma unroll
            for (int r = 0; r < R2; ++r)
                if (r < nvalid) {
                    const int b = db(dt(x[r]));
                    if (b < c1) {
                        ++nbel;
                    } else if (b <= c2) {
                        uint32_t s = atomicAdd(&sh.cnt, 1u);
                        if (s < CAPM) sh.candf[s] = (float)x[r];
                    }
                }
        }
        nbel = __reduce_add_sync(0xffffffffu, nbel);
        if (lane == 0 && nbel) atomicAdd(&sh.below, nbel);
        __syncthreads();
        const uint32_t cc = sh.cnt, cb = sh.below;
        for (uint32_t i = tid; i < cc && i < CAPM; i += T2) sh.cand[i] = dkey(fabs((double)sh.candf[i] - med));
        __syncthreads();
        if (cc <= CAPM && cb <= r1 && r2 - cb < cc) {
            cand_pick2(sh, cc, r1 - cb, r2 - cb, &mk1, &mk2);
        } else {
            if (cc <= CAPM) dev_fail(d_status, FFA_ERR_DEVICE);  // bracket invariant broken
            const T* vb = buf;
            auto key = [vb, med](int j) -> uint64_t { return dkey(fabs((double)vb[sidx(j)] - med)); };
            mk1 = smem_select64(sh, p0, r1, key);
            mk2 = (r1 == r2) ? mk1 : smem_select64(sh, p0, r2, key);
        }
        __syncthreads();
    }

    }  // !mad_done

    // ---- blocked cyclic prefix (bins past p0 repeat the profile) ----
    // Extension blocks (index >= T2) start at bin 32768 > p0, above the value
    // region of the buffer, so their prefixes are stored at once; own blocks
    // overwrite values and wait until every thread has read its values.
    const int eb2 = tid + T2;  // this thread's extension block, if any
    T tot = 0, tot2 = 0;
    const bool one_wrap = nbe * R2 <= 2 * p0;  // extension bins map to j - p0
    if (eb2 < nbe) {
#pragma unroll 4
        for (int r = 0; r < R2; ++r) {
            const int j = eb2 * R2 + r;
            const T v = buf[sidx(one_wrap ? j - p0 : j % p0)];
            buf[sidx(eb2 * R2 + r)] = tot2;
            tot2 = tot2 + v;
        }
    }
#pragma unroll
    for (int r = 0; r < R2; ++r) {
        const int j = base_pos + r;
        T v = x[r];
        if (j >= p0) v = (tid < nbe) ? buf[sidx(one_wrap ? j - p0 : j % p0)] : (T)0;
        x[r] = tot;  // exclusive in-block prefix
        tot = tot + v;
    }
    if constexpr (C::DIST && Traits<T>::is_int) {
        if (tid < 16) sh.wkey[tid] = 0u;  // below every key
    }
    __syncthreads();  // every value read: own blocks now take the prefixes
    {
        T* blk = buf + sidx(base_pos);
#pragma unroll
        for (int r = 0; r < R2; r += 4) *reinterpret_cast<int4*>(blk + r) = *reinterpret_cast<const int4*>(&x[r]);
    }
    if constexpr (Traits<T>::is_int) {
        uint32_t t0, t1;
        const uint32_t ex0 = blk_exscan_u((uint32_t)tot, sh, &t0);
        int* cbi = reinterpret_cast<int*>(sh.cbh);
        cbi[tid] = (int)ex0;
        if (nbe > T2) {
            const uint32_t ex1 = blk_exscan_u(eb2 < nbe ? (uint32_t)tot2 : 0u, sh, &t1);
            if (eb2 <= MAXB) cbi[eb2] = (int)(t0 + ex1);
        } else if (tid == 0) {
            cbi[T2] = (int)t0;
        }
    } else {
        float oh, ol, th, tl, oh2, ol2, th2, tl2;
        blk_exscan_ff((float)tot, sh, oh, ol, th, tl);
        sh.cbh[tid] = oh;
        sh.cbl[tid] = ol;
        if (nbe > T2) {
            blk_exscan_ff(eb2 < nbe ? (float)tot2 : 0.0f, sh, oh2, ol2, th2, tl2);
            if (eb2 <= MAXB) {
                float h, l;
                ff_add(th, tl, oh2, ol2, h, l);
                sh.cbh[eb2] = h;
                sh.cbl[eb2] = l;
            }
        } else if (tid == 0) {
            sh.cbh[T2] = th;
            sh.cbl[T2] = tl;
        }
    }
    __syncthreads();

    // The MAD and the S/N factors, once, by the last thread (usually one
    // without bins, so the FP64 latency hides behind the widths); read after
    // the barrier that ends the widths.
    if (tid == T2 - 1) {
        const double med = sh.smed;
        double mad;
        if constexpr (Traits<T>::is_int) {
            const double e1 = (double)mk1, e2 = (double)mk2;  // exact integers
            mad = (r1 == r2) ? e1 / 2 : (e1 + e2) / 4;
        } else {
            const double d1 = dkey_inv(mk1), d2 = dkey_inv(mk2);
            mad = (r1 == r2) ? d1 : (d1 + d2) / 2;
        }
        const double kmad = __dmul_rn(KMAD, mad);
        sh.madpos = mad > 0.0;
        sh.skmad = kmad;
        if constexpr (!Traits<T>::is_int) {
            const float mh = __double2float_rn(med);
            sh.snr_mh = mh;
            sh.snr_ml = __double2float_rn(__dsub_rn(med, (double)mh));
            sh.snr_kf = __double2float_rn(kmad);
        }
    }

    // ---- widths (Section 2.2.1): per-thread maxima, warp-reduced ----
    // Every thread with profile bins scores all R bins of its block: in the
    // one block that runs past p0 the extra boxes start at bins p0 + i and
    // are the cyclic boxes at bin i again (from the extended prefix), so the
    // maxima are unchanged up to rounding (exactly, for int profiles) and no
    // per-bin bound check is needed.  A first argmax found there is reported
    // at bin i (i mod p0 for profiles shorter than a block).
    const bool own = base_pos < p0;
    int dummy = -1;
    if constexpr (C::DIST && Traits<T>::is_int) {
        // Item-distributed widths: item i = (width i / nblk, block i mod
        // nblk) over every thread of the CTA, each block's in-block prefix
        // read back from shared memory (the blocks with bins are only part of
        // the CTA for most profile lengths, and the registers that held the
        // profile are free again).  A warp's 32 consecutive items span at
        // most a few widths; each width's warp maximum goes to a shared
        // order-preserving key by one atomicMax.  Taken for int profiles of
        // the 1024 x 32 shape, whose register-held widths spill; for float
        // profiles the per-width re-read of each block costs more shared-
        // memory bandwidth than the idle threads save (measured).
        const int nblk = (p0 + R2 - 1) / R2;
        const int total = wd.n * nblk;
        const float inv = 1.0f / (float)nblk;
        for (int i0 = warp * 32; i0 < total; i0 += T2) {
            const int i = i0 + lane;
            const bool valid = i < total;
            int wi = -1;
            uint32_t key = 0u;
            if (valid) {
                wi = (int)((float)i * inv);  // floor(i / nblk) up to one step
                int b = i - wi * nblk;
                if (b < 0) {
                    --wi;
                    b += nblk;
                } else if (b >= nblk) {
                    ++wi;
                    b -= nblk;
                }
                T c[R2];
                const T* cb = buf + sidx(b * R2);
#pragma unroll
                for (int r = 0; r < R2; r += 4)
                    *reinterpret_cast<int4*>(&c[r]) = *reinterpret_cast<const int4*>(cb + r);
                const T m = width_max<T, false>(c, sh, buf, b, wd.w[wi], R2, (T)0, &dummy);
                if constexpr (Traits<T>::is_int) key = ikey((int32_t)m);
                else key = fkey((float)m);
            }
            unsigned pend = __ballot_sync(0xffffffffu, valid);
            while (pend) {
                const int src = __ffs(pend) - 1;
                const int wa = __shfl_sync(0xffffffffu, wi, src);
                const bool mine = valid && wi == wa;
                const uint32_t km = __reduce_max_sync(0xffffffffu, mine ? key : 0u);
                if (lane == src) atomicMax(&sh.wkey[wa], km);
                pend &= ~__ballot_sync(0xffffffffu, mine);
            }
        }
        __syncthreads();
        if (tid < wd.n) {
            const uint32_t k = sh.wkey[tid];
            if constexpr (Traits<T>::is_int) sh.bw_max[tid] = (double)(int32_t)(k ^ 0x80000000u);
            else sh.bw_maxf[tid] = fkey_inv(k);
        }
    } else {
        for (int wi = 0; wi < wd.n; ++wi) {
            T m = B::lowest();
            if (own) m = width_max<T, false>(x, sh, buf, tid, wd.w[wi], R2, (T)0, &dummy);
            if constexpr (Traits<T>::is_int) {
                m = warp_maxi(m);
                if (lane == 0) sh.wredi[wi][warp] = m;
            } else {
                m = warp_max(m);
                if (lane == 0) sh.wred[wi][warp] = m;
            }
        }
        __syncthreads();
        // per-width block maxima: warp w reduces the warp maxima of widths w, w + NW, ...
        for (int wi = warp; wi < wd.n; wi += NW) {
            if constexpr (Traits<T>::is_int) {
                const double Bw = (double)warp_maxi(lane < NW ? sh.wredi[wi][lane] : INT32_MIN);
                if (lane == 0) sh.bw_max[wi] = Bw;
            } else {
                const float bf = warp_max(lane < NW ? sh.wred[wi][lane] : -INFINITY);
                if (lane == 0) sh.bw_maxf[wi] = bf;
            }
        }
    }
    __syncthreads();
    // S/N_w = (B_w - w*med) / (K*MAD*sqrt(w)).  sqrt(w) for w = 2^n is
    // 2^(n/2), or 2^((n-1)/2) times the correctly rounded sqrt(2) for odd n
    // (the correctly rounded square root, without computing one).  Int
    // profiles: FP64 with round-to-nearest intrinsics, the correctly rounded
    // quotient of the exact numerator (widths ranked by an FP32 key first).
    // Float profiles: the numerator in float-float (med split into two
    // floats; w * part is exact) and one FP32 division, within a few ulp of
    // the FP64 quotient (GB300's FP64 rate is a small fraction of FP32's).
    // Ties go to the smaller width.
    if (warp == 0) {
        const double kmad = sh.skmad, med = sh.smed;
        constexpr double SQRT2 = 1.4142135623730951;  // sqrt(2) rounded to nearest
        float key = -INFINITY;
        if constexpr (Traits<T>::is_int) {
            if (lane < wd.n) {
                const double w = (double)wd.w[lane];
                const double num = __dsub_rn(sh.bw_max[lane], __dmul_rn(w, med));
                const int n = __ffs(wd.w[lane]) - 1;
                // 1/sqrt(w) for w = 2^n: 2^(-n/2) for even n, else 2^(-(n-1)/2)/sqrt(2)
                const float rs = (n & 1) ? ldexpf(0.70710678f, -(n - 1) / 2) : ldexpf(1.0f, -n / 2);
                key = __double2float_rn(num) * rs;
            }
        } else {
            const float mh = sh.snr_mh, ml = sh.snr_ml, kf = sh.snr_kf;
            if (lane < wd.n) {
                const float w = (float)wd.w[lane];
                const float bx = sh.bw_maxf[lane];
                float hi, lo;
                two_sum(bx, -(w * mh), hi, lo);  // w * mh, w * ml exact (w a power of two)
                const float num = __fadd_rn(hi, __fsub_rn(lo, w * ml));
                const int n = __ffs(wd.w[lane]) - 1;
                // fl(sqrt 2) * 2^((n-1)/2) is exactly fl(sqrt(2) * 2^((n-1)/2))
                constexpr float SQRT2F = (float)SQRT2;
                const float sq = (n & 1) ? ldexpf(SQRT2F, (n - 1) / 2) : ldexpf(1.0f, n / 2);
                key = __fdiv_rn(num, __fmul_rn(kf, sq));
            }
        }
        int bw = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const float ok = __shfl_xor_sync(0xffffffffu, key, o);
            const int ob = __shfl_xor_sync(0xffffffffu, bw, o);
            if (ok > key || (ok == key && ob < bw)) {
                key = ok;
                bw = ob;
            }
        }
        if (lane == 0) {
            if constexpr (Traits<T>::is_int) {
                const int n = __ffs(wd.w[bw]) - 1;
                const double w = (double)wd.w[bw];
                const double num = __dsub_rn(sh.bw_max[bw], __dmul_rn(w, med));
                const double sq = (n & 1) ? ldexp(SQRT2, (n - 1) / 2) : ldexp(1.0, n / 2);
                sh.fred[0] = __double2float_rn(__ddiv_rn(num, __dmul_rn(kmad, sq)));
            } else {
                sh.fred[0] = key;
            }
            sh.ired[0] = bw;
        }
    }
    __syncthreads();
    const float bestv = sh.fred[0];
    const int bw = sh.ired[0];
    const int madpos = sh.madpos;
    __syncthreads();
    // first argmax of the winning width, recomputed bit-identically
    T target;
    int first = -1;
    if constexpr (C::DIST && Traits<T>::is_int) {
        if constexpr (Traits<T>::is_int) target = (T)(int32_t)(sh.wkey[bw] ^ 0x80000000u);
        else target = (T)fkey_inv(sh.wkey[bw]);
        if (own && madpos) {
            T c[R2];
            const T* cb = buf + sidx(base_pos);
#pragma unroll
            for (int r = 0; r < R2; r += 4)
                *reinterpret_cast<int4*>(&c[r]) = *reinterpret_cast<const int4*>(cb + r);
            (void)width_max<T, true>(c, sh, buf, tid, wd.w[bw], R2, target, &first);
        }
    } else {
        if constexpr (Traits<T>::is_int) target = (T)warp_maxi(lane < NW ? sh.wredi[bw][lane] : INT32_MIN);
        else target = (T)warp_max(lane < NW ? sh.wred[bw][lane] : -INFINITY);
        if (own && madpos) (void)width_max<T, true>(x, sh, buf, tid, wd.w[bw], R2, target, &first);
    }
    int fpos = 0x7fffffff;
    if (first >= 0) {
        fpos = base_pos + first;
        if (fpos >= p0) fpos %= p0;  // a box of the wrapped tail (p0 < R wraps more than once)
    }
    const int pos = blk_mini(fpos, sh);
    if (tid == 0) {
        ffa_record out;
        if (!madpos) {
            out.snr = 0.0f;
            out.width = wd.w[0];
            out.phase = 0;
            out.flags = 1;
        } else {
            out.snr = bestv;
            out.width = wd.w[bw];
            out.phase = pos == 0x7fffffff ? 0 : pos;
            out.flags = 0;
            if (pos == 0x7fffffff) dev_fail(d_status, FFA_ERR_DEVICE);
        }
        sg.rec[ei][it - sg.t0[ei]] = out;
    }
    __syncthreads();
    }  // trials
}

// ---------------------------------------------------------------------------
// Algorithm 2 (Section 2.2.2, Eq. 5): boxcar first, then for each width the
// maximum I_max (first position j*), an exclusion window of the 2h+1 profile
// bins within cyclic distance h of the box's centre (j* + w/2) mod p0, and
// A_w = (I_max - w I_av) / (sigma sqrt(w)) with I_av and sigma the mean and
// population standard deviation of the other, unfiltered, profile bins;
// score = max over widths.  The profile's sum of squares about its mean is
// taken once; per width only the window's share is summed (its raw bins
// recovered as differences of the in-block prefix) and subtracted.  FP64
// per width, by one thread.
// ---------------------------------------------------------------------------
template <class T, class C>
__device__ __forceinline__ T box_at(const T (&c)[C::R], const Sh2<C>& sh, const T* buf, int tid, int w, int r) {
    FFA_CFG_ALIASES
    using B = BoxOps<T>;
    // cyclic box of width w starting at bin 32 tid + r, from the blocked prefix
    const int j2 = tid * R2 + r + w;
    const int b2 = j2 / R2, o2 = j2 % R2;
    return B::box(B::blockdiff(sh, b2, tid), buf[sidx(b2 * R2 + o2)], c[r]);
}

template <class C, class T, bool FUSED>
__global__ void __launch_bounds__(C::T, C::MINB) k_score_alg2(const T* __restrict__ prof_all, const ScoreGroup sg,
                                                              int64_t m_rows, int64_t trial0, int64_t count,
                                                              ScoreWidths wd, float excl_frac) {
    FFA_CFG_ALIASES
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sh2<C>& sh = *reinterpret_cast<Sh2<C>*>(smem_raw);
    T* buf = reinterpret_cast<T*>(smem_raw + ((sizeof(Sh2<C>) + 15) & ~(size_t)15));
    using B = BoxOps<T>;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int wmax = wd.w[wd.n - 1];
    for (int64_t it = blockIdx.x; it < count; it += gridDim.x) {
        const int ei = score_entry(sg, it);
        const int64_t p0_ = sg.p0[ei];
        const int p0 = (int)p0_;
        const T* __restrict__ prof = prof_all + sg.off[ei];
        const int nbe = (p0 + wmax + R2) / R2 + 1;
        const int h = (int)floorf(excl_frac * (float)p0 / 2.0f);
        const int n_off = p0 - min(p0, 2 * h + 1);
        const int64_t k = trial0 + (it - sg.t0[ei]);
        const T* hrow;
        const T* trow = nullptr;
        int sft = 0;
        const int64_t ld_ = sg.ld[ei];
        if (FUSED && m_rows > 1) {
            hrow = prof + (k >> 1) * ld_;
            trow = prof + ((m_rows >> 1) + (k >> 1)) * ld_;
            sft = (int)(((k + 1) >> 1) % p0_);
        } else if (FUSED) {
            hrow = prof;
        } else {
            hrow = prof + k * ld_;
        }
        if (trow) {
            const int n1 = p0 - sft;
            for (int j = tid; j < p0; j += T2) buf[sidx(j)] = hrow[j] + (j < n1 ? trow[j + sft] : trow[j - n1]);
        } else {
            for (int j = tid; j < p0; j += T2) buf[sidx(j)] = hrow[j];
        }
        __syncthreads();
        T x[R2];
        const int base_pos = tid * R2;
        int nvalid = p0 - base_pos;
        nvalid = nvalid < 0 ? 0 : (nvalid > R2 ? R2 : nvalid);
        float fs = 0.0f, fq = 0.0f, fm = 0.0f;
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            x[r] = (r < nvalid) ? buf[sidx(base_pos + r)] : (T)0;
            if (r < nvalid) fs += (float)x[r];
        }
        blk_stats(fs, fq, fm, sh);
        const float mean = fs / (float)p0;
        // the whole profile's sums of (x - mean) and (x - mean)^2
        float ps = 0.0f, pq = 0.0f, pm = 0.0f;
#pragma unroll
        for (int r = 0; r < R2; ++r)
            if (r < nvalid) {
                const float d = (float)x[r] - mean;
                ps += d;
                pq = fmaf(d, d, pq);
            }
        blk_stats(ps, pq, pm, sh);
        // blocked cyclic prefix (as in k_score2)
        const bool one_wrap = nbe * R2 <= 2 * p0;
        const int eb2 = tid + T2;
        T tot = 0, tot2 = 0;
        if (eb2 < nbe) {
            for (int r = 0; r < R2; ++r) {
                const int j = eb2 * R2 + r;
                const T v = buf[sidx(one_wrap ? j - p0 : j % p0)];
                buf[sidx(j)] = tot2;
                tot2 = tot2 + v;
            }
        }
#pragma unroll
        for (int r = 0; r < R2; ++r) {
            const int j = base_pos + r;
            T v = x[r];
            if (j >= p0) v = (tid < nbe) ? buf[sidx(one_wrap ? j - p0 : j % p0)] : (T)0;
            x[r] = tot;
            tot = tot + v;
        }
        __syncthreads();
        {
            T* blk = buf + sidx(base_pos);
#pragma unroll
            for (int r = 0; r < R2; r += 4) *reinterpret_cast<int4*>(blk + r) = *reinterpret_cast<const int4*>(&x[r]);
        }
        if constexpr (Traits<T>::is_int) {
            uint32_t t0, t1;
            const uint32_t ex0 = blk_exscan_u((uint32_t)tot, sh, &t0);
            int* cbi = reinterpret_cast<int*>(sh.cbh);
            cbi[tid] = (int)ex0;
            if (nbe > T2) {
                const uint32_t ex1 = blk_exscan_u(eb2 < nbe ? (uint32_t)tot2 : 0u, sh, &t1);
                if (eb2 <= MAXB) cbi[eb2] = (int)(t0 + ex1);
            } else if (tid == 0) {
                cbi[T2] = (int)t0;
            }
        } else {
            float oh, ol, th, tl, oh2, ol2, th2, tl2;
            blk_exscan_ff((float)tot, sh, oh, ol, th, tl);
            sh.cbh[tid] = oh;
            sh.cbl[tid] = ol;
            if (nbe > T2) {
                blk_exscan_ff(eb2 < nbe ? (float)tot2 : 0.0f, sh, oh2, ol2, th2, tl2);
                if (eb2 <= MAXB) {
                    float hh, ll;
                    ff_add(th, tl, oh2, ol2, hh, ll);
                    sh.cbh[eb2] = hh;
                    sh.cbl[eb2] = ll;
                }
            } else if (tid == 0) {
                sh.cbh[T2] = th;
                sh.cbl[T2] = tl;
            }
        }
        __syncthreads();
        double best = -INFINITY;
        int best_w = 0, best_j = 0;
        for (int wi = 0; wi < wd.n; ++wi) {
            const int w = wd.w[wi];
            T m = B::lowest();
            int mpos = 0x7fffffff;
            if (nvalid > 0) {
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    if (r < nvalid) {
                        const T bx = box_at(x, sh, buf, tid, w, r);
                        if (bx > m) {
                            m = bx;
                            mpos = base_pos + r;
                        }
                    }
                }
            }
            // block: max with its first position
            float mf = (float)m;
            for (int o = 16; o > 0; o >>= 1) {
                const float om = __shfl_xor_sync(0xffffffffu, mf, o);
                const int op = __shfl_xor_sync(0xffffffffu, mpos, o);
                if (om > mf || (om == mf && op < mpos)) {
                    mf = om;
                    mpos = op;
                }
            }
            __syncthreads();
            if (lane == 0) {
                sh.wred[0][warp] = mf;
                sh.wredi[0][warp] = mpos;
            }
            __syncthreads();
            mf = lane < NW ? sh.wred[0][lane] : -INFINITY;
            mpos = lane < NW ? sh.wredi[0][lane] : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                const float om = __shfl_xor_sync(0xffffffffu, mf, o);
                const int op = __shfl_xor_sync(0xffffffffu, mpos, o);
                if (om > mf || (om == mf && op < mpos)) {
                    mf = om;
                    mpos = op;
                }
            }
            const int jstar = mpos;
            const int centre = (int)(((int64_t)jstar + w / 2) % p0);
            // sums of (x - mean) and its square over the window's profile bins;
            // bin r's value is the difference of the in-block prefix (the last
            // bin's: the block total minus the last prefix)
            float w1 = 0.0f, w2 = 0.0f;
            if (nvalid > 0) {
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const int j = base_pos + r;
                    int d = j - centre;
                    if (d < 0) d = -d;
                    d = min(d, p0 - d);
                    if (r < nvalid && d <= h) {
                        const T v = B::diff(r + 1 < R2 ? x[r + 1] : tot, x[r]);
                        const float dd = (float)v - mean;
                        w1 += dd;
                        w2 = fmaf(dd, dd, w2);
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
                w2 += __shfl_xor_sync(0xffffffffu, w2, o);
            }
            __syncthreads();
            if (lane == 0) {
                sh.wred[3][warp] = w1;
                sh.wred[4][warp] = w2;
            }
            __syncthreads();
            w1 = lane < NW ? sh.wred[3][lane] : 0.0f;
            w2 = lane < NW ? sh.wred[4][lane] : 0.0f;
            for (int o = 16; o > 0; o >>= 1) {
                w1 += __shfl_xor_sync(0xffffffffu, w1, o);
                w2 += __shfl_xor_sync(0xffffffffu, w2, o);
            }
            if (tid == 0 && n_off >= 2) {  // only thread 0 keeps the score: FP64 once per width
                const double a1 = ((double)ps - (double)w1) / n_off;  // off-pulse mean - mean
                const double var = ((double)pq - (double)w2) / n_off - a1 * a1;
                const double sd = var > 0.0 ? sqrt(var) : 0.0;
                const double av = (double)mean + a1;
                if (sd > 0.0) {
                    const double a = ((double)mf - (double)w * av) / (sd * sqrt((double)w));
                    if (a > best) {
                        best = a;
                        best_w = wi;
                        best_j = jstar;
                    }
                }
            }
        }
        if (tid == 0) {
            ffa_record out;
            if (best == -INFINITY) {
                out.snr = 0.0f;
                out.width = wd.w[0];
                out.phase = 0;
                out.flags = 1;
            } else {
                out.snr = (float)best;
                out.width = wd.w[best_w];
                out.phase = best_j;
                out.flags = 0;
            }
            sg.rec[ei][it - sg.t0[ei]] = out;
        }
        __syncthreads();
    }
}

namespace {

// Resident CTAs of a kernel for a dynamic shared-memory size, times the SM
// count, per device: queried once (launches come per base period).
ffa_status resident_ctas(const void* fn, int threads, size_t smem, int64_t* out) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, size_t, int>, int64_t> cache;
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    const auto key = std::make_tuple(fn, smem, dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *out = it->second;
            return FFA_OK;
        }
    }
    int nsm = 0, per_sm = 0;
    FFA_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    FFA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    const int64_t r = (int64_t)nsm * (per_sm < 1 ? 1 : per_sm);
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = r;
    *out = r;
    return FFA_OK;
}

template <class C>
size_t score2_smem_bytes(int64_t p0, int wmax, size_t elem) {
    const int64_t nbe = (p0 + wmax + C::R) / C::R + 1;
    const int64_t nbins = (nbe > C::T ? nbe : C::T) * C::R + C::R;
    return ((sizeof(Sh2<C>) + 15) & ~(size_t)15) + (size_t)(nbins + 4 * (nbins / 32) + 64) * elem;
}

// does a profile of p0 bins with widths up to wmax fit configuration C?
template <class C>
bool fits(int64_t p0, int wmax) {
    return p0 >= 1 && (p0 + C::R - 1) / C::R <= C::T && (p0 + wmax + C::R) / C::R + 1 <= C::MAXB;
}

template <class C, class TT, bool FF>
ffa_status launch_score2_cfg(const void* d_prof, const ScoreGroup& sg, int64_t count, int64_t trial0, int64_t p0,
                             int64_t m_rows, const ScoreWidths& wd, ffa_record* d_rec, int32_t* d_status,
                             cudaStream_t st) {
    const int wmax = wd.w[wd.n - 1];
    const size_t smem = score2_smem_bytes<C>(p0, wmax, 4);
    if (smem > 227 * 1024) return fail(FFA_ERR_UNSUPPORTED, "score: profile too long for shared memory");
    const void* fn = (const void*)k_score2<C, TT, FF>;
    ffa_status es = ensure_smem(fn, smem);
    if (es != FFA_OK) return es;
    int64_t resident = 0;  // persistent: every CTA resident
    es = resident_ctas(fn, C::T, smem, &resident);
    if (es != FFA_OK) return es;
    const unsigned grid = (unsigned)(count < resident ? count : resident);
    (void)d_rec;  // the records go where sg.rec points
    k_score2<C, TT, FF><<<grid, C::T, smem, st>>>((const TT*)d_prof, sg, m_rows, trial0, count, wd, d_status);
    FFA_LAUNCH_CHECK("k_score2");
    count_launch();
    return FFA_OK;
}

// p0: the longest profile of the group (it picks the CTA shape and the
// shared-memory size)
template <class TT, bool FF>
ffa_status launch_score2_t(const void* d_prof, const ScoreGroup& sg, int64_t count, int64_t trial0, int64_t p0,
                           int64_t m_rows, const ScoreWidths& wd, ffa_record* d_rec, int32_t* d_status,
                           cudaStream_t st) {
    const int wmax = wd.w[wd.n - 1];
    if (fits<Cfg<256>>(p0, wmax))
        return launch_score2_cfg<Cfg<256>, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, d_rec, d_status, st);
    if (fits<Cfg<512>>(p0, wmax))
        return launch_score2_cfg<Cfg<512>, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, d_rec, d_status, st);
    if (fits<CMid>(p0, wmax))
        return launch_score2_cfg<CMid, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, d_rec, d_status, st);
    return launch_score2_cfg<CBig, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, d_rec, d_status, st);
}

}  // namespace

// The scorer's CTA shape for a profile of p0 bins (0: 256 x 8, 1: 512 x 16,
// 2: 1024 x 16, 3: 1024 x 32); grouped launches hold one shape only, so a
// profile's record does not depend on what it is grouped with.
int score_shape(int64_t p0, int wmax) {
    if (fits<Cfg<256>>(p0, wmax)) return 0;
    if (fits<Cfg<512>>(p0, wmax)) return 1;
    if (fits<CMid>(p0, wmax)) return 2;
    return 3;
}

namespace {

ScoreGroup single(int64_t p0, int64_t ld, int64_t count, ffa_record* d_rec) {
    ScoreGroup sg;
    sg.n = 1;
    sg.t0[0] = 0;
    sg.t0[1] = count;
    sg.p0[0] = (int32_t)p0;
    sg.off[0] = 0;
    sg.ld[0] = ld;
    sg.rec[0] = d_rec;
    return sg;
}

ffa_status score2_dispatch(const void* d_prof, const ScoreGroup& sg, int32_t precision, bool fused, int64_t count,
                           int64_t trial0, int64_t p0max, int64_t m_rows, const ScoreWidths& wd,
                           ffa_record* d_rec, int32_t* d_status, cudaStream_t st) {
    if (count <= 0) return FFA_OK;
    const int wmax = wd.w[wd.n - 1];
    if (!fits<CBig>(p0max, wmax)) return fail(FFA_ERR_UNSUPPORTED, "score: profile longer than 32768 bins");
    if (precision == FFA_FOLD_F32)
        return fused ? launch_score2_t<float, true>(d_prof, sg, count, trial0, p0max, m_rows, wd, d_rec, d_status, st)
                     : launch_score2_t<float, false>(d_prof, sg, count, trial0, p0max, m_rows, wd, d_rec, d_status, st);
    return fused ? launch_score2_t<int32_t, true>(d_prof, sg, count, trial0, p0max, m_rows, wd, d_rec, d_status, st)
                 : launch_score2_t<int32_t, false>(d_prof, sg, count, trial0, p0max, m_rows, wd, d_rec, d_status, st);
}

}  // namespace

ffa_status launch_score2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                         int64_t trial0, int64_t p0, int64_t ld, int64_t m_rows, const ScoreWidths& wd,
                         ffa_record* d_rec, int32_t* d_status, cudaStream_t st) {
    return score2_dispatch(d_prof, single(p0, ld, count, d_rec), precision, fused, count, trial0, p0, m_rows, wd, d_rec,
                           d_status, st);
}

ffa_status launch_score2_group(const void* d_plane, int32_t precision, int n, const int64_t* p0, const int64_t* off,
                               int64_t m_rows, const ScoreWidths& wd, ffa_record* const* recs, int32_t* d_status,
                               cudaStream_t st) {
    if (n < 1 || n > FOLD_GROUP_MAX) return fail(FFA_ERR_ARG, "score group: 1..FOLD_GROUP_MAX base periods");
    ScoreGroup sg;
    sg.n = n;
    int64_t p0max = 0;
    for (int i = 0; i < n; ++i) {
        sg.t0[i] = (int64_t)i * m_rows;
        sg.p0[i] = (int32_t)p0[i];
        sg.off[i] = off[i];
        sg.ld[i] = plane_pitch(p0[i]);
        sg.rec[i] = recs[i];
        p0max = p0[i] > p0max ? p0[i] : p0max;
    }
    sg.t0[n] = (int64_t)n * m_rows;
    return score2_dispatch(d_plane, sg, precision, true, (int64_t)n * m_rows, 0, p0max, m_rows, wd, recs[0],
                           d_status, st);
}

namespace {

template <class C, class TT, bool FF>
ffa_status launch_alg2_cfg(const void* d_prof, const ScoreGroup& sg, int64_t count, int64_t trial0, int64_t p0,
                           int64_t m_rows, const ScoreWidths& wd, float excl_frac, ffa_record* d_rec,
                           cudaStream_t st) {
    const int wmax = wd.w[wd.n - 1];
    const size_t smem = score2_smem_bytes<C>(p0, wmax, 4);
    if (smem > 227 * 1024) return fail(FFA_ERR_UNSUPPORTED, "score: profile too long for shared memory");
    const void* fn = (const void*)k_score_alg2<C, TT, FF>;
    ffa_status es = ensure_smem(fn, smem);
    if (es != FFA_OK) return es;
    int64_t resident = 0;
    es = resident_ctas(fn, C::T, smem, &resident);
    if (es != FFA_OK) return es;
    const unsigned grid = (unsigned)(count < resident ? count : resident);
    (void)d_rec;  // the records go where sg.rec points
    k_score_alg2<C, TT, FF><<<grid, C::T, smem, st>>>((const TT*)d_prof, sg, m_rows, trial0, count, wd,
                                                      excl_frac);
    FFA_LAUNCH_CHECK("k_score_alg2");
    count_launch();
    return FFA_OK;
}

template <class TT, bool FF>
ffa_status launch_alg2_t(const void* d_prof, const ScoreGroup& sg, int64_t count, int64_t trial0, int64_t p0,
                         int64_t m_rows, const ScoreWidths& wd, float excl_frac, ffa_record* d_rec,
                         cudaStream_t st) {
    const int wmax = wd.w[wd.n - 1];
    if (fits<Cfg<256>>(p0, wmax))
        return launch_alg2_cfg<Cfg<256>, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, excl_frac, d_rec, st);
    if (fits<Cfg<512>>(p0, wmax))
        return launch_alg2_cfg<Cfg<512>, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, excl_frac, d_rec, st);
    if (fits<CMid>(p0, wmax))
        return launch_alg2_cfg<CMid, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, excl_frac, d_rec, st);
    return launch_alg2_cfg<CBig, TT, FF>(d_prof, sg, count, trial0, p0, m_rows, wd, excl_frac, d_rec, st);
}

ffa_status alg2_dispatch(const void* d_prof, const ScoreGroup& sg, int32_t precision, bool fused, int64_t count,
                         int64_t trial0, int64_t p0max, int64_t m_rows, const ScoreWidths& wd, float excl_frac,
                         ffa_record* d_rec, cudaStream_t st) {
    if (count <= 0) return FFA_OK;
    const int wmax = wd.w[wd.n - 1];
    if (!fits<CBig>(p0max, wmax)) return fail(FFA_ERR_UNSUPPORTED, "score: profile longer than 32768 bins");
    if (precision == FFA_FOLD_F32)
        return fused ? launch_alg2_t<float, true>(d_prof, sg, count, trial0, p0max, m_rows, wd, excl_frac, d_rec, st)
                     : launch_alg2_t<float, false>(d_prof, sg, count, trial0, p0max, m_rows, wd, excl_frac, d_rec, st);
    return fused ? launch_alg2_t<int32_t, true>(d_prof, sg, count, trial0, p0max, m_rows, wd, excl_frac, d_rec, st)
                 : launch_alg2_t<int32_t, false>(d_prof, sg, count, trial0, p0max, m_rows, wd, excl_frac, d_rec, st);
}

}  // namespace

ffa_status launch_score_alg2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                             int64_t trial0, int64_t p0, int64_t ld, int64_t m_rows, const ScoreWidths& wd,
                             float excl_frac, ffa_record* d_rec, cudaStream_t st) {
    return alg2_dispatch(d_prof, single(p0, ld, count, d_rec), precision, fused, count, trial0, p0, m_rows, wd, excl_frac,
                         d_rec, st);
}

ffa_status launch_score_alg2_group(const void* d_plane, int32_t precision, int n, const int64_t* p0,
                                   const int64_t* off, int64_t m_rows, const ScoreWidths& wd, float excl_frac,
                                   ffa_record* const* recs, cudaStream_t st) {
    if (n < 1 || n > FOLD_GROUP_MAX) return fail(FFA_ERR_ARG, "score group: 1..FOLD_GROUP_MAX base periods");
    ScoreGroup sg;
    sg.n = n;
    int64_t p0max = 0;
    for (int i = 0; i < n; ++i) {
        sg.t0[i] = (int64_t)i * m_rows;
        sg.p0[i] = (int32_t)p0[i];
        sg.off[i] = off[i];
        sg.ld[i] = plane_pitch(p0[i]);
        sg.rec[i] = recs[i];
        p0max = p0[i] > p0max ? p0[i] : p0max;
    }
    sg.t0[n] = (int64_t)n * m_rows;
    return alg2_dispatch(d_plane, sg, precision, true, (int64_t)n * m_rows, 0, p0max, m_rows, wd, excl_frac,
                         recs[0], st);
}

}  // namespace ffa
