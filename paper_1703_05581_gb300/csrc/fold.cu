// The FFA fold on the GPU (Section 2.1).
//
// Recursion: output trial k of a block of 2^s rows is head[k>>1] plus
// tail[k>>1] read ceil(k/2) bins further on (cyclic).  Unrolled, row r of a
// 2^m-row block enters trial k with the cyclic shift
//     shift(r, k) = sum_l bit_(m-1-l)(r) * ceil((k >> l) / 2).
//
// Multi-stage passes.  After s stages the plane holds, for every group g of
// 2^s consecutive input rows, its 2^s partial trials at row g*2^s + kappa.
// A pass of q further stages combines blocks of 2^q groups.  For a fixed
// input trial kappa, output trial kappa*2^q + v of a block takes group u's
// partial trial kappa at the shift  kappa*u + shift_q(u, v)  where shift_q
// is the shift table of a 2^q-row block (because ceil((kappa*2^(q-l) +
// (v>>l))/2) = kappa*2^(q-l-1) + ceil((v>>l)/2) for l < q).  So each pass is
// a plain 2^q-row FFA whose input row u starts at column kappa*u: the same
// adds in the same tree as the recursion, hence bit-identical results.
//
// A CTA owns (block, kappa, column tile): it stages 2^q rows of B + 2^q - 1
// columns (the halo covers the local shifts) in shared memory, runs the q
// local stages in registers (two register-blocked sub-passes) and writes 2^q
// rows of B columns.  Planes inside a search have a row pitch padded to a
// multiple of 4 elements, so rows are 16-byte aligned for the staging copies
// and the 128-bit output stores.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace ffa {


// Base periods folded by one launch: entry i has p0[i] bins, m_data[i] data
// rows (all share m_rows), its plane at element offset off[i] of the plane
// buffers with row pitch ld[i] (>= p0[i]; a multiple of 4 makes every row
// 16-byte aligned), and owns the launch's CTAs [unit0[i], unit0[i + 1]).  A
// single base period is a group of one.  The first pass reads the series
// itself: row g of entry i is src[i][g * p0[i] ...], densely packed (entries
// of a batch read their own series).
struct FoldGroup {
    int32_t n;
    const void* src[FOLD_GROUP_MAX];
    int64_t p0[FOLD_GROUP_MAX];
    int64_t m_data[FOLD_GROUP_MAX];
    int64_t off[FOLD_GROUP_MAX];
    int64_t ld[FOLD_GROUP_MAX];
    int64_t unit0[FOLD_GROUP_MAX + 1];
};

// this CTA's entry and its unit within the entry
__device__ __forceinline__ int group_entry(const FoldGroup& g, int64_t unit) {
    int lo = 0, hi = g.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g.unit0[mid] <= unit) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <class T>
struct FoldIn;
template <>
struct FoldIn<float> { using type = float; };
template <>
struct FoldIn<int32_t> { using type = int8_t; };

// Asynchronous global -> shared copies (cp.async): a lane issues all of its
// copies for a tile without waiting, then waits once (cp_async_wait).  The
// 16-byte form bypasses L1 (each element is read by one tile only, apart from
// the halo, which the next tile finds in L2).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage `wt` cyclic columns of a row starting at column `base` (< p0) into
// shared memory (one warp per row); returns the element offset (0..3) of
// logical column 0 in rowp (16-byte aligned).  A segment that does not wrap
// is copied as whole 16-byte chunks from its aligned-down start, so the
// offset is its misalignment; the chunk holding the segment's last element
// ends within that element's 16-byte block, so nothing outside it is read.
// A wrapping segment (or a row shorter than the segment) is copied element
// by element at offset 0, int8 rows are widened to int32 through registers
// (whole 4-byte words when the segment does not wrap), and rows at or beyond
// m_data (live == false) are zero.
template <class T, class S>
__device__ __forceinline__ int stage_row(T* __restrict__ rowp, const S* __restrict__ src, int64_t base,
                                         int64_t p0, int wt, bool live, int lane) {
    if (!live) {
        for (int x = 4 * lane; x < wt; x += 128) *reinterpret_cast<int4*>(rowp + x) = make_int4(0, 0, 0, 0);
        return 0;
    }
    if constexpr (sizeof(T) == sizeof(S)) {
        if (base + wt <= p0) {
            const S* g = src + base;
            const int a = (int)(((uintptr_t)g >> 2) & 3);
            const S* g0 = g - a;
            const int nc = (wt + a + 3) >> 2;
            for (int k = lane; k < nc; k += 32) cp_async16(rowp + 4 * k, g0 + 4 * k);
            return a;
        }
        if (wt <= p0) {
            const int n1 = (int)(p0 - base);  // columns before the wrap
            const S* a = src + base;
            for (int x = lane; x < n1; x += 32) cp_async4(rowp + x, a + x);
            for (int x = n1 + lane; x < wt; x += 32) cp_async4(rowp + x, src + (x - n1));
            return 0;
        }
        int64_t col = base + lane;
        while (col >= p0) col -= p0;
        for (int x = lane; x < wt; x += 32) {
            cp_async4(rowp + x, src + col);
            col += 32;
            while (col >= p0) col -= p0;
        }
        return 0;
    } else {
        if (base + wt <= p0) {
            // int8 series widened to int32: whole aligned 4-byte words of the
            // segment, one load per lane per word, each byte sign-extended into
            // one 128-bit shared store; logical column 0 sits at the segment's
            // misalignment, as for the copied rows (little-endian bytes)
            const S* g = src + base;
            const int a = (int)((uintptr_t)g & 3);
            const uint32_t* w0 = reinterpret_cast<const uint32_t*>(g - a);
            const int nw = (wt + a + 3) >> 2;
            for (int k = lane; k < nw; k += 32) {
                const uint32_t v = __ldg(w0 + k);
                *reinterpret_cast<int4*>(rowp + 4 * k) =
                    make_int4((int)(v << 24) >> 24, (int)(v << 16) >> 24, (int)(v << 8) >> 24, (int)v >> 24);
            }
            return a;
        }
        int64_t col = base + lane;
        while (col >= p0) col -= p0;
        for (int x = lane; x < wt; x += 32) {
            rowp[x] = (T)src[col];
            col += 32;
            while (col >= p0) col -= p0;
        }
        return 0;
    }
}

// ---------------------------------------------------------------------------
// The FFA of R = 2^QQ rows on W = 4 + R - 1 consecutive columns held in
// registers (compile-time shifts): out[v][0..3] is trial v at the first four
// columns.  load() reads a row's W values starting at element offset `off`
// (0..3) of a 16-byte aligned pointer: 128-bit loads, then two branch-free
// selects per value (a warp-uniform branch on the offset measured slower).
// ---------------------------------------------------------------------------
template <class T, int QQ>
struct RegFFA {
    static constexpr int R = 1 << QQ;
    static constexpr int W = 4 + R - 1;
    static constexpr int NV = (W + 6) / 4;  // 128-bit loads covering W values at any offset
    static __device__ __forceinline__ void load(const T* p, int off, T (&a)[W]) {
        T r[4 * NV];
#pragma unroll
        for (int k = 0; k < NV; ++k)
            *reinterpret_cast<int4*>(&r[4 * k]) = *reinterpret_cast<const int4*>(p + 4 * k);
        const bool b0 = (off & 1) != 0, b1 = (off & 2) != 0;
        T t[W + 2];
#pragma unroll
        for (int k = 0; k < W + 2; ++k) t[k] = b0 ? r[k + 1] : r[k];
#pragma unroll
        for (int k = 0; k < W; ++k) a[k] = b1 ? t[k + 2] : t[k];
    }
    static __device__ __forceinline__ void run(T (&a)[R][W], T (&out)[R][4]) {
#pragma unroll
        for (int t = 1; t <= QQ; ++t) {
            const int g = 1 << t, half = g >> 1;
            T b[R][W];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int gb = r & ~(g - 1), v = r - gb;
                const int hr = gb + (v >> 1), tr = gb + half + (v >> 1), sf = (v + 1) >> 1;
#pragma unroll
                for (int x = 0; x < W; ++x)
                    if (x + g - 1 < W) b[r][x] = a[hr][x] + a[tr][x + sf];
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int x = 0; x < W; ++x) a[r][x] = b[r][x];
        }
#pragma unroll
        for (int v = 0; v < R; ++v)
#pragma unroll
            for (int x = 0; x < 4; ++x) out[v][x] = a[v][x];
    }
};

template <class T>
__device__ __forceinline__ int as_bits(T v) {
    if constexpr (sizeof(T) == 4 && !std::is_integral<T>::value) return __float_as_int(v);
    else return (int)v;
}

// Four consecutive outputs to global memory: one 128-bit store when the row
// is 16-byte aligned (vec), else element stores up to `left` columns.
template <class T>
__device__ __forceinline__ void store4(T* d, const T (&v)[4], int64_t left, bool vec) {
    if (vec) {
        *reinterpret_cast<int4*>(d) = make_int4(as_bits(v[0]), as_bits(v[1]), as_bits(v[2]), as_bits(v[3]));
    } else {
#pragma unroll
        for (int x = 0; x < 4; ++x)
            if (x < left) d[x] = v[x];
    }
}

// ---------------------------------------------------------------------------
// One pass of q = Q1 + Q2 <= 6 stages.  A CTA owns (block, kappa, column
// tile of B columns): it stages 2^q input rows of B + 2^q - 1 columns, row u
// starting at column c + kappa*u (cyclically), in shared memory.  Sub-pass 1:
// each thread takes 4 consecutive columns of a group of 2^Q1 rows, applies
// Q1 stages in registers and stores the group's 2^Q1 partial trials,
// unshifted, with 128-bit stores.  Sub-pass 2: for trial k1 of sub-pass 1,
// input row u2 of the last Q2 stages is read at column offset k1*u2 (the
// shift that the unrolled recursion assigns it), Q2 stages in registers, and
// the tile's output rows go to global memory (128-bit stores on a padded
// pitch).  Tiles are B = 256 columns up to 5 stages and 128 for 6 (64 rows),
// so two CTAs fit an SM.
// ---------------------------------------------------------------------------
constexpr int FK_THREADS = 256;
__host__ __device__ constexpr int fk_r4(int x) { return (x + 3) & ~3; }
__host__ __device__ constexpr int fk_max(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int fk_wt(int q, int b) { return b + (1 << q) - 1; }                  // staged columns
__host__ __device__ constexpr int fk_w1(int q, int q1, int b) { return b + (1 << q) - (1 << q1); }  // valid after sub-pass 1
// Row widths (elements) of the two shared buffers: room for the staging
// copies and for every 128-bit load of the two sub-passes.
__host__ __device__ constexpr int fk_wa(int q, int q1, int b) {
    return fk_max(fk_r4(fk_wt(q, b) + 3), 4 * ((fk_w1(q, q1, b) + 3) / 4 - 1) + 4 * ((4 + (1 << q1) - 1 + 6) / 4));
}
__host__ __device__ constexpr int fk_wb(int q, int q1, int b) {
    return fk_max(fk_r4(fk_w1(q, q1, b)), (b - 4) + 4 * ((((1 << q1) - 1) * ((1 << (q - q1)) - 1)) / 4) +
                                              4 * ((4 + (1 << (q - q1)) - 1 + 6) / 4));
}

template <class T, bool FIRST, int Q1, int Q2, int B>
__global__ void __launch_bounds__(FK_THREADS, 2) k_fold(const void* __restrict__ src_v, T* __restrict__ dst_all,
                                                       const FoldGroup fg, int s) {
    constexpr int q = Q1 + Q2;
    constexpr int rows = 1 << q;
    constexpr int R1 = 1 << Q1, R2 = 1 << Q2;
    constexpr int WT = fk_wt(q, B), W1 = fk_w1(q, Q1, B);
    constexpr int WA = fk_wa(q, Q1, B), WB = fk_wb(q, Q1, B);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int off_a[rows];
    T* bufA = reinterpret_cast<T*>(smem_raw);
    T* bufB = bufA + rows * WA;

    const int ei = group_entry(fg, blockIdx.x);
    const int64_t p0 = fg.p0[ei], m_data = fg.m_data[ei], ld = fg.ld[ei];
    const int64_t n_ct = (p0 + B - 1) / B;
    T* __restrict__ dst = dst_all + fg.off[ei];
    const int64_t unit = blockIdx.x - fg.unit0[ei];
    const int64_t ct = unit % n_ct;
    const int64_t rest = unit / n_ct;
    const int64_t kappa = rest & ((1ll << s) - 1);
    const int64_t blk = rest >> s;
    const int64_t c = ct * B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = FK_THREADS / 32;

    const int64_t kmod = kappa % p0;
    auto row_base = [&](int u) -> int64_t {
        int64_t base = c + (kmod * (u % p0)) % p0;
        return base >= p0 ? base - p0 : base;
    };
    if constexpr (FIRST && sizeof(typename FoldIn<T>::type) == 1) {
        // int8 series: the plain loads of all of this warp's rows are issued
        // before any is widened and stored, so that their DRAM latencies
        // overlap (cp.async cannot widen).  Rows that wrap or lie beyond the
        // data take stage_row's general path.
        using S = typename FoldIn<T>::type;
        constexpr int RPW = (rows + NW - 1) / NW;     // rows per warp
        constexpr int KPL = ((WT + 6) / 4 + 31) / 32;  // aligned words per lane and row
        const S* srcb = (const S*)fg.src[ei];
        uint32_t wv[RPW][KPL];
        int aw[RPW];
#pragma unroll
        for (int j = 0; j < RPW; ++j) {
            const int u = warp + j * NW;
            aw[j] = -1;
            if (u < rows) {
                const int64_t g = blk * rows + u;
                const int64_t base = row_base(u);
                if (g < m_data && base + WT <= p0) {
                    const S* gp = srcb + g * p0 + base;
                    const int a = (int)((uintptr_t)gp & 3);
                    const uint32_t* w0 = reinterpret_cast<const uint32_t*>(gp - a);
                    const int nw = (WT + a + 3) >> 2;  // the word holding the last element ends the copy
#pragma unroll
                    for (int t = 0; t < KPL; ++t) {
                        const int k = lane + 32 * t;
                        wv[j][t] = k < nw ? __ldg(w0 + k) : 0u;
                    }
                    aw[j] = a;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < RPW; ++j) {
            const int u = warp + j * NW;
            if (u >= rows) continue;
            T* rowp = bufA + u * WA;
            int a = aw[j];
            if (a >= 0) {
                const int nw = (WT + a + 3) >> 2;
#pragma unroll
                for (int t = 0; t < KPL; ++t) {
                    const int k = lane + 32 * t;
                    const uint32_t v = wv[j][t];
                    if (k < nw)
                        *reinterpret_cast<int4*>(rowp + 4 * k) = make_int4(
                            (int)(v << 24) >> 24, (int)(v << 16) >> 24, (int)(v << 8) >> 24, (int)v >> 24);
                }
            } else {
                const int64_t g = blk * rows + u;
                a = stage_row(rowp, srcb + g * p0, row_base(u), p0, WT, g < m_data, lane);
            }
            if (lane == 0) off_a[u] = a;
        }
    } else {
        for (int u = warp; u < rows; u += NW) {
            const int64_t g = blk * rows + u;
            const int64_t base = row_base(u);
            int a;
            if (FIRST)
                a = stage_row(bufA + u * WA, (const typename FoldIn<T>::type*)fg.src[ei] + g * p0, base, p0, WT,
                              g < m_data, lane);
            else
                a = stage_row(bufA + u * WA, (const T*)src_v + fg.off[ei] + ((g << s) + kappa) * ld, base, p0, WT,
                              true, lane);
            if (lane == 0) off_a[u] = a;
        }
    }
    cp_async_wait();
    __syncthreads();
    const int64_t grow0 = (blk << (s + q)) + (kappa << q);
    const int64_t ncols = (c + B <= p0) ? B : p0 - c;
    const bool vec = (ld & 3) == 0 && ((uintptr_t)dst & 15) == 0;

    // sub-pass 1: groups of R1 consecutive rows
    {
        constexpr int W = RegFFA<T, Q1>::W;
        constexpr int nstrips = (W1 + 3) / 4;
        constexpr int items = (rows / R1) * nstrips;
        for (int it = threadIdx.x; it < items; it += FK_THREADS) {
            const int strip = it % nstrips, g = it / nstrips;
            const int x0 = 4 * strip;
            T a[R1][W];
#pragma unroll
            for (int u = 0; u < R1; ++u) RegFFA<T, Q1>::load(bufA + (g * R1 + u) * WA + x0, off_a[g * R1 + u], a[u]);
            T out[R1][4];
            RegFFA<T, Q1>::run(a, out);
            if (Q2 == 0) {
                if (x0 < ncols) {
#pragma unroll
                    for (int v = 0; v < R1; ++v) store4(dst + (grow0 + v) * ld + c + x0, out[v], ncols - x0, vec);
                }
            } else {
                // group g is input row u2 = g of sub-pass 2
#pragma unroll
                for (int v = 0; v < R1; ++v)
                    *reinterpret_cast<int4*>(bufB + (v * R2 + g) * WB + x0) =
                        make_int4(as_bits(out[v][0]), as_bits(out[v][1]), as_bits(out[v][2]), as_bits(out[v][3]));
            }
        }
    }
    if (Q2 > 0) {
        __syncthreads();
        constexpr int W = RegFFA<T, Q2>::W;
        constexpr int nstrips = B / 4;
        constexpr int items = R1 * nstrips;
        for (int it = threadIdx.x; it < items; it += FK_THREADS) {
            const int strip = it % nstrips, k1 = it / nstrips;
            const int x0 = 4 * strip;
            T a[R2][W];
#pragma unroll
            for (int u = 0; u < R2; ++u) {
                const int sh = k1 * u;
                RegFFA<T, Q2>::load(bufB + (k1 * R2 + u) * WB + x0 + (sh & ~3), sh & 3, a[u]);
            }
            T out[R2][4];
            RegFFA<T, Q2>::run(a, out);
            if (x0 < ncols) {
#pragma unroll
                for (int v = 0; v < R2; ++v)
                    store4(dst + (grow0 + k1 * R2 + v) * ld + c + x0, out[v], ncols - x0, vec);
            }
        }
    }
}

// Split m stages into passes of at most `qmax`, as evenly as possible.
static int split_passes(int m, int qmax, int* qs) {
    if (m == 0) return 0;
    int np = (m + qmax - 1) / qmax;
    for (int i = 0; i < np; ++i) qs[i] = m / np + (i < m % np ? 1 : 0);
    return np;
}

// Fill the group's CTA ranges for a pass whose CTAs cover `rows` output rows
// and `tile` columns; returns the launch's CTA count.
static int64_t group_units(FoldGroup& fg, int64_t m_rows, int rows, int tile) {
    int64_t u = 0;
    for (int i = 0; i < fg.n; ++i) {
        fg.unit0[i] = u;
        u += (m_rows / rows) * ((fg.p0[i] + tile - 1) / tile);
    }
    fg.unit0[fg.n] = u;
    return u;
}

template <class T, bool FIRST, int Q1, int Q2, int B>
static ffa_status launch_k(const void* src, T* dst, FoldGroup& fg, int64_t m_rows, int s, cudaStream_t st) {
    constexpr int q = Q1 + Q2;
    constexpr int rows = 1 << q;
    const size_t smem =
        sizeof(T) * ((size_t)rows * fk_wa(q, Q1, B) + (Q2 > 0 ? (size_t)rows * fk_wb(q, Q1, B) : 0));
    ffa_status es = ensure_smem((const void*)k_fold<T, FIRST, Q1, Q2, B>, smem);
    if (es != FFA_OK) return es;
    const int64_t units = group_units(fg, m_rows, rows, B);
    if (units <= 0) return FFA_OK;
    if (units > INT32_MAX) return fail(FFA_ERR_UNSUPPORTED, "fold: plane too large for one launch");
    k_fold<T, FIRST, Q1, Q2, B><<<(unsigned)units, FK_THREADS, smem, st>>>(src, dst, fg, s);
    FFA_LAUNCH_CHECK("k_fold");
    count_launch();
    return FFA_OK;
}

// Tile width of a pass: `wide` != 0 takes 256 columns, else 128.
template <class T, bool FIRST, int Q1, int Q2>
static ffa_status launch_kb(bool wide, const void* src, T* dst, FoldGroup& fg, int64_t m_rows, int s,
                            cudaStream_t st) {
    return wide ? launch_k<T, FIRST, Q1, Q2, 256>(src, dst, fg, m_rows, s, st)
                : launch_k<T, FIRST, Q1, Q2, 128>(src, dst, fg, m_rows, s, st);
}

template <class T, bool FIRST>
static ffa_status pass_q(int q, bool wide, const void* src, T* dst, FoldGroup& fg, int64_t m_rows, int s,
                         cudaStream_t st) {
    switch (q) {
        case 0: return launch_kb<T, FIRST, 0, 0>(wide, src, dst, fg, m_rows, s, st);
        case 1: return launch_kb<T, FIRST, 1, 0>(wide, src, dst, fg, m_rows, s, st);
        case 2: return launch_kb<T, FIRST, 2, 0>(wide, src, dst, fg, m_rows, s, st);
        case 3: return launch_kb<T, FIRST, 3, 0>(wide, src, dst, fg, m_rows, s, st);
        case 4: return launch_kb<T, FIRST, 2, 2>(wide, src, dst, fg, m_rows, s, st);
        case 5: return launch_kb<T, FIRST, 3, 2>(wide, src, dst, fg, m_rows, s, st);
        case 6: return launch_kb<T, FIRST, 3, 3>(wide, src, dst, fg, m_rows, s, st);
        default: break;
    }
    return fail(FFA_ERR_ARG, "fold: at most 6 stages per pass");
}

// The fold's launch shape: at most `qmax` stages per pass, tiles of `tile`
// columns (0: 256 below six stages, 128 at six, so that two CTAs fit an SM).
struct FoldShape {
    int qmax;
    int tile;
};

template <class T>
static ffa_status fold_impl(const void* d_z, FoldGroup& fg, int64_t m_rows, int stages, T* d_plane, T* d_tmp,
                            cudaStream_t st, FoldShape fs) {
    int qs[64];
    int np = split_passes(stages, fs.qmax, qs);
    if (np == 0) {
        // no stage to run: copy the (zero-padded) rows
        np = 1;
        qs[0] = 0;
    }
    // ping-pong so that the last pass lands in d_plane
    T* bufs[2] = {d_plane, d_tmp};
    int s = 0;
    for (int pi = 0; pi < np; ++pi) {
        T* dst = bufs[(np - 1 - pi) & 1];
        const void* src = pi == 0 ? d_z : (const void*)bufs[(np - pi) & 1];
        const bool wide = fs.tile == 256 || (fs.tile == 0 && qs[pi] < 6);
        ffa_status e = pi == 0 ? pass_q<T, true>(qs[pi], wide, src, dst, fg, m_rows, s, st)
                               : pass_q<T, false>(qs[pi], wide, src, dst, fg, m_rows, s, st);
        if (e != FFA_OK) return e;
        s += qs[pi];
    }
    return FFA_OK;
}

// ---------------------------------------------------------------------------
// Stages per pass and tile width, tuned.  Any split of the stages into passes,
// and any tile width, gives the same add tree (bit-identical planes); only the
// time differs.  The cache maps (device, precision, stages, floor(log2 p0)) to
// the fastest shape measured by tune_fold; untuned shapes use six stages per
// pass with the default widths.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, FoldShape> g_tune;
constexpr FoldShape SHAPE_DEFAULT = {6, 0};

int log2i(int64_t v) {
    int r = 0;
    while ((int64_t)2 << r <= v) ++r;
    return r;
}

FoldShape tuned_shape(int precision, int stages, int64_t p0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SHAPE_DEFAULT;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, precision, stages, log2i(p0)));
    return it == g_tune.end() ? SHAPE_DEFAULT : it->second;
}
}  // namespace

static ffa_status fold_group(const void* d_z, int32_t precision, FoldGroup& fg, int64_t m_rows, int stages,
                             void* d_plane, void* d_tmp, cudaStream_t st, FoldShape fs) {
    if (precision == FFA_FOLD_F32)
        return fold_impl<float>(d_z, fg, m_rows, stages, (float*)d_plane, (float*)d_tmp, st, fs);
    return fold_impl<int32_t>(d_z, fg, m_rows, stages, (int32_t*)d_plane, (int32_t*)d_tmp, st, fs);
}

static ffa_status fold_with(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                            int stages, int64_t ld, void* d_plane, void* d_tmp, cudaStream_t st, FoldShape fs) {
    FoldGroup fg;
    fg.n = 1;
    fg.p0[0] = p0;
    fg.m_data[0] = m_data;
    fg.off[0] = 0;
    fg.ld[0] = ld;
    fg.src[0] = d_z;
    return fold_group(d_z, precision, fg, m_rows, stages, d_plane, d_tmp, st, fs);
}

// Time each maximum pass depth 3..6 with each tile width (128 and 256
// columns) on one shape (CUDA events, best of 2 after a warm-up) and cache
// the fastest.  The planes are scratch.
ffa_status tune_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                     int stages, int64_t ld, void* d_plane, void* d_tmp, cudaStream_t st, int* best_q) {
    cudaEvent_t e0, e1;
    FFA_CUDA_TRY(cudaEventCreate(&e0));
    FFA_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    FoldShape bs = SHAPE_DEFAULT;
    ffa_status s = FFA_OK;
    for (int q = 3; q <= 6 && s == FFA_OK; ++q) {
        for (int tile : {128, 256}) {
            const FoldShape fs = {q, tile};
            s = fold_with(d_z, precision, p0, m_data, m_rows, stages, ld, d_plane, d_tmp, st, fs);  // warm-up
            float t_q = 1e30f;
            for (int rep = 0; rep < 2 && s == FFA_OK; ++rep) {
                cudaEventRecord(e0, st);
                s = fold_with(d_z, precision, p0, m_data, m_rows, stages, ld, d_plane, d_tmp, st, fs);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "tune_fold");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                t_q = ms < t_q ? ms : t_q;
            }
            if (s != FFA_OK) break;
            if (t_q < best) {
                best = t_q;
                bs = fs;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != FFA_OK) return s;
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple(dev, precision, stages, log2i(p0))] = bs;
    }
    if (best_q) *best_q = bs.qmax * 1000 + bs.tile;
    return FFA_OK;
}

ffa_status launch_fold_group(const void* d_z, int32_t precision, int n, const int64_t* p0, const int64_t* m_data,
                             const int64_t* off, int64_t m_rows, int stages, void* d_plane, void* d_tmp,
                             cudaStream_t st, const void* const* z) {
    if (n < 1 || n > FOLD_GROUP_MAX) return fail(FFA_ERR_ARG, "fold group: 1..FOLD_GROUP_MAX base periods");
    FoldGroup fg;
    fg.n = n;
    for (int i = 0; i < n; ++i) {
        fg.p0[i] = p0[i];
        fg.m_data[i] = m_data[i];
        fg.off[i] = off[i];
        fg.ld[i] = plane_pitch(p0[i]);
        fg.src[i] = z ? z[i] : d_z;
    }
    return fold_group(d_z, precision, fg, m_rows, stages, d_plane, d_tmp, st,
                      tuned_shape(precision, stages, p0[n - 1]));
}

// Run the first `stages` FFA stages (all of them when stages < 0).  With
// fewer stages the plane holds, per group of 2^stages rows, its partial
// trials (row g * 2^stages + kappa); zero stages copy the (zero-padded) rows.
ffa_status launch_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                       int64_t m_rows, int stages, int64_t ld, void* d_plane, void* d_tmp, cudaStream_t st) {
    int m = 0;
    while ((1ll << m) < m_rows) ++m;
    if (stages < 0 || stages > m) stages = m;
    return fold_with(d_z, precision, p0, m_data, m_rows, stages, ld, d_plane, d_tmp, st,
                     tuned_shape(precision, stages, p0));
}

}  // namespace ffa

// ---------------------------------------------------------------------------
// Fold without any allocation (see ffa_fold_noalloc in include/ffa.h).
// ---------------------------------------------------------------------------
namespace {
// Scratch plane shared by every ffa_fold_noalloc call on a device; it lives
// in the module image, so every GPU that loads the library holds it.
static __device__ __align__(256) float g_fold_scratch[FFA_NOALLOC_FOLD_MAX_ELEMS];

// The array's device address is looked up once per device and context: a
// cudaDeviceReset (or any re-creation of the primary context) reloads the
// module, so the address is looked up again when the current context's
// unique id changes.  The driver calls come through the runtime's entry
// point query, so the library still links only against the runtime.
typedef CUresult (*ctx_get_current_t)(CUcontext*);
typedef CUresult (*ctx_get_id_t)(CUcontext, unsigned long long*);

std::mutex g_scratch_mu;
struct ScratchSlot {
    void* ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool has_id = false;
};
ScratchSlot g_scratch[64];

// Unique id of the calling thread's current context; false if none is
// current yet or the driver does not offer the query.
bool current_ctx_id(unsigned long long* id) {
    static ctx_get_current_t get_cur = nullptr;
    static ctx_get_id_t get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            get_cur = (ctx_get_current_t)f1;
            get_id = (ctx_get_id_t)f2;
        }
    }
    if (!get_cur || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}
}  // namespace

extern "C" ffa_status ffa_fold_noalloc(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                                       int64_t m_rows, void* d_plane, void* stream) {
    using namespace ffa;
    if (p0 < 1 || m_data < 0 || m_rows < 1 || (m_rows & (m_rows - 1)) != 0 || m_data > m_rows)
        return fail(FFA_ERR_ARG, "fold_noalloc: need p0 >= 1, m_rows a power of two >= m_data");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8)
        return fail(FFA_ERR_ARG, "fold_noalloc: bad precision");
    if (!d_z || !d_plane) return fail(FFA_ERR_ARG, "fold_noalloc: null buffer");
    // m_rows >= 1 here; the division form cannot overflow
    if (p0 > (int64_t)FFA_NOALLOC_FOLD_MAX_ELEMS / m_rows)
        return fail(FFA_ERR_UNSUPPORTED,
                    "fold_noalloc: m_rows * p0 exceeds FFA_NOALLOC_FOLD_MAX_ELEMS (the fixed scratch)");
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FFA_ERR_UNSUPPORTED, "fold_noalloc: device index >= 64");
    void* scratch;
    {
        // set-up once per device and context, with that device current: the
        // device address of the array (its host-side name is only a stand-in,
        // not a device address)
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        ScratchSlot& sl = g_scratch[dev];
        unsigned long long id = 0;
        const bool has_id = current_ctx_id(&id);
        if (!sl.ptr || !has_id || !sl.has_id || id != sl.ctx_id) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_fold_scratch);
            if (e != cudaSuccess || !ptr) return cuda_fail(e, "fold_noalloc: cudaGetSymbolAddress");
            sl.ptr = ptr;
            // the lookup makes the primary context current if none was
            sl.has_id = current_ctx_id(&sl.ctx_id);
        }
        scratch = sl.ptr;
    }
    return launch_fold(d_z, precision, p0, m_data, m_rows, -1, p0, d_plane, scratch, as_stream(stream));
}
