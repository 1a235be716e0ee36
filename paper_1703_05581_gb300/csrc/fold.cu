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
// local stages there (ping-pong buffers) and writes 2^q rows of B columns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "internal.h"

namespace ffa {


// Base periods folded by one launch: entry i has p0[i] bins, m_data[i] data
// rows (all share m_rows), its plane at element offset off[i] of the plane
// buffers, and owns the launch's CTAs [unit0[i], unit0[i + 1]).  A single
// base period is a group of one.
struct FoldGroup {
    int32_t n;
    int64_t p0[FOLD_GROUP_MAX];
    int64_t m_data[FOLD_GROUP_MAX];
    int64_t off[FOLD_GROUP_MAX];
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

// Asynchronous 4-byte global -> shared copy (cp.async): a lane issues all of
// its copies for a tile without waiting, then waits once (cp_async_wait).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class T, class S>
__device__ __forceinline__ void put_async(T* dst, const S* src) {
    if constexpr (sizeof(T) == sizeof(S)) cp_async4(dst, src);
    else *dst = (T)*src;  // int8 series into int32 rows: converted through registers
}

// Stage `wt` cyclic columns of a row starting at column `base` (< p0) into
// shared memory: at most one wrap when wt <= p0, so the segment is two
// contiguous runs.  Same-width rows are copied with cp.async (the caller
// waits with cp_async_wait before its barrier), so every row of a tile is in
// flight at once.
template <class T, class S>
__device__ __forceinline__ void stage_row(T* __restrict__ rowp, const S* __restrict__ src, int64_t base,
                                          int64_t p0, int wt, bool live, int lane) {
    if (!live) {
        for (int x = lane; x < wt; x += 32) rowp[x] = (T)0;
        return;
    }
    if (wt <= p0) {
        const int n1 = (int)((p0 - base) < wt ? (p0 - base) : wt);  // columns before the wrap
        const S* a = src + base;
#pragma unroll 4
        for (int x = lane; x < n1; x += 32) put_async(rowp + x, a + x);
#pragma unroll 4
        for (int x = n1 + lane; x < wt; x += 32) put_async(rowp + x, src + (x - n1));
    } else {
        int64_t col = base + lane;
        while (col >= p0) col -= p0;
        for (int x = lane; x < wt; x += 32) {
            put_async(rowp + x, src + col);
            col += 32;
            while (col >= p0) col -= p0;
        }
    }
}

// ---------------------------------------------------------------------------
// One pass of q <= 5 stages.  A CTA owns (block, kappa, column tile): it
// stages 2^q rows of B + 2^q - 1 columns in shared memory (row u starting at
// column c + kappa*u, cyclically), runs the q local stages with one warp per
// row (ping-pong buffers, conflict-free contiguous accesses) and writes 2^q
// rows of B columns.
// ---------------------------------------------------------------------------
constexpr int FP_THREADS = 256;
constexpr int FP_B = 256;

template <class T, bool FIRST>
__global__ void __launch_bounds__(FP_THREADS) k_fold_pass(const void* __restrict__ src_v,
                                                          T* __restrict__ dst_all, const FoldGroup fg,
                                                          int s, int q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rows = 1 << q;
    const int wt = FP_B + rows - 1;
    T* buf0 = reinterpret_cast<T*>(smem_raw);
    T* buf1 = buf0 + rows * wt;
    const int ei = group_entry(fg, blockIdx.x);
    const int64_t p0 = fg.p0[ei], m_data = fg.m_data[ei];
    const int64_t n_ct = (p0 + FP_B - 1) / FP_B;
    T* __restrict__ dst = dst_all + fg.off[ei];
    if (!FIRST) src_v = (const T*)src_v + fg.off[ei];
    const int64_t unit = blockIdx.x - fg.unit0[ei];
    const int64_t ct = unit % n_ct;
    const int64_t rest = unit / n_ct;
    const int64_t kappa = rest & ((1ll << s) - 1);
    const int64_t blk = rest >> s;
    const int64_t c = ct * FP_B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = FP_THREADS / 32;

    const int64_t kmod = kappa % p0;
    for (int u = warp; u < rows; u += NW) {
        const int64_t g = blk * rows + u;  // group index at level s
        int64_t base = c + (kmod * (u % p0)) % p0;
        if (base >= p0) base -= p0;
        if (FIRST)
            stage_row(buf0 + u * wt, (const typename FoldIn<T>::type*)src_v + g * p0, base, p0, wt,
                      g < m_data, lane);
        else
            stage_row(buf0 + u * wt, (const T*)src_v + ((g << s) + kappa) * p0, base, p0, wt, true, lane);
    }
    cp_async_wait();
    __syncthreads();
    T* in = buf0;
    T* out = buf1;
    for (int t = 1; t <= q; ++t) {
        const int half = 1 << (t - 1);
        const int width = wt - ((1 << t) - 1);
        for (int r = warp; r < rows; r += NW) {
            const int gb = r & ~((1 << t) - 1);
            const int v = r - gb;
            const T* h = in + (gb + (v >> 1)) * wt;
            const T* tl = in + (gb + half + (v >> 1)) * wt + ((v + 1) >> 1);
            T* o = out + r * wt;
            for (int x = lane; x < width; x += 32) o[x] = h[x] + tl[x];
        }
        __syncthreads();
        T* tmp = in;
        in = out;
        out = tmp;
    }
    const int64_t out_row0 = (blk << (s + q)) + (kappa << q);
    const int64_t ncols = (c + FP_B <= p0) ? FP_B : p0 - c;
    for (int v = warp; v < rows; v += NW) {
        T* d = dst + (out_row0 + v) * p0 + c;
        const T* sv = in + v * wt;
        for (int x = lane; x < ncols; x += 32) d[x] = sv[x];
    }
}

// Split m stages into passes of at most `qmax`, as evenly as possible.
static int split_passes(int m, int qmax, int* qs) {
    if (m == 0) return 0;
    int np = (m + qmax - 1) / qmax;
    for (int i = 0; i < np; ++i) qs[i] = m / np + (i < m % np ? 1 : 0);
    return np;
}

// ---------------------------------------------------------------------------
// Register-blocked pass (q = Q1 + Q2 <= 5 stages).  After staging the tile
// as above, each thread takes 4 consecutive columns of one group of 2^Q1 rows,
// loads them with aligned 128-bit shared-memory reads, applies Q1 stages in
// registers (compile-time shifts) and stores its 2^Q1 partial trials already
// shifted left by kappa1*u2, the column offset at which the second sub-pass
// reads them; the second sub-pass then reads 128-bit aligned as well, applies
// the remaining Q2 stages and writes the tile's output rows to global memory.
// Neighbouring threads take neighbouring columns: conflict-free 16-byte reads.
// ---------------------------------------------------------------------------
template <class T, int QQ>
struct RegStages {
    static constexpr int R = 1 << QQ;
    static constexpr int W = 4 + R - 1;      // columns needed for 4 outputs
    static constexpr int NV = (W + 3) / 4;   // 128-bit loads per row
    // rows: R pointers (16-byte aligned) into shared memory; out[v][0..3]
    static __device__ __forceinline__ void run(const T* const* rowp, T (&out)[R][4]) {
        T a[R][NV * 4];
#pragma unroll
        for (int u = 0; u < R; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k)
                *reinterpret_cast<int4*>(&a[u][4 * k]) = *reinterpret_cast<const int4*>(rowp[u] + 4 * k);
#pragma unroll
        for (int t = 1; t <= QQ; ++t) {
            const int g = 1 << t, half = g >> 1;
            T b[R][NV * 4];
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

constexpr int F4_THREADS = 256;
constexpr int F4_B = 256;
__host__ __device__ constexpr int f4_wa(int q) { return ((F4_B + (1 << q) - 1 + 3) & ~3) + 8; }
__host__ __device__ constexpr int f4_wb(int q, int q1) { return ((F4_B + (1 << q) - (1 << q1) + 3) & ~3) + 8; }

template <class T, bool FIRST, int Q1, int Q2>
__global__ void __launch_bounds__(F4_THREADS, 2) k_fold_reg(const void* __restrict__ src_v,
                                                           T* __restrict__ dst_all, const FoldGroup fg,
                                                           int s) {
    constexpr int q = Q1 + Q2;
    constexpr int rows = 1 << q;
    constexpr int R1 = 1 << Q1, R2 = 1 << Q2;
    constexpr int WA = f4_wa(q), WB = f4_wb(q, Q1);
    constexpr int W1 = F4_B + rows - R1;  // valid columns after the first sub-pass
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* bufA = reinterpret_cast<T*>(smem_raw);
    T* bufB = bufA + rows * WA;

    const int ei = group_entry(fg, blockIdx.x);
    const int64_t p0 = fg.p0[ei], m_data = fg.m_data[ei];
    const int64_t n_ct = (p0 + F4_B - 1) / F4_B;
    T* __restrict__ dst = dst_all + fg.off[ei];
    if (!FIRST) src_v = (const T*)src_v + fg.off[ei];
    const int64_t unit = blockIdx.x - fg.unit0[ei];
    const int64_t ct = unit % n_ct;
    const int64_t rest = unit / n_ct;
    const int64_t kappa = rest & ((1ll << s) - 1);
    const int64_t blk = rest >> s;
    const int64_t c = ct * F4_B;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = F4_THREADS / 32;
    constexpr int WT = F4_B + rows - 1;  // staged columns

    const int64_t kmod = kappa % p0;
    for (int u = warp; u < rows; u += NW) {
        const int64_t g = blk * rows + u;
        int64_t base = c + (kmod * (u % p0)) % p0;
        if (base >= p0) base -= p0;
        if (FIRST)
            stage_row(bufA + u * WA, (const typename FoldIn<T>::type*)src_v + g * p0, base, p0, WT,
                      g < m_data, lane);
        else
            stage_row(bufA + u * WA, (const T*)src_v + ((g << s) + kappa) * p0, base, p0, WT, true, lane);
    }
    cp_async_wait();
    __syncthreads();
    const int64_t grow0 = (blk << (s + q)) + (kappa << q);
    const int64_t ncols = (c + F4_B <= p0) ? F4_B : p0 - c;

    // first sub-pass: groups of R1 consecutive rows
    {
        constexpr int nstrips = (W1 + 3) / 4;
        constexpr int items = (rows / R1) * nstrips;
        for (int it = threadIdx.x; it < items; it += F4_THREADS) {
            const int strip = it % nstrips, g = it / nstrips;
            const int x0 = 4 * strip;
            const T* rp[R1];
#pragma unroll
            for (int u = 0; u < R1; ++u) rp[u] = bufA + (g * R1 + u) * WA + x0;
            T out[R1][4];
            RegStages<T, Q1>::run(rp, out);
            if (Q2 == 0) {
#pragma unroll
                for (int v = 0; v < R1; ++v) {
                    T* d = dst + (grow0 + v) * p0 + c + x0;
#pragma unroll
                    for (int x = 0; x < 4; ++x)
                        if (x0 + x < ncols) d[x] = out[v][x];
                }
            } else {
                // group g is input row u2 = g of the second sub-pass; trial v of it is
                // read at column offset v*u2: store it shifted left by that much
                const int u2 = g;
#pragma unroll
                for (int v = 0; v < R1; ++v) {
                    T* d = bufB + (v * R2 + u2) * WB;
                    const int sh = v * u2;
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        const int xx = x0 + x - sh;
                        if (xx >= 0 && x0 + x < W1) d[xx] = out[v][x];
                    }
                }
            }
        }
    }
    if (Q2 > 0) {
        __syncthreads();
        constexpr int nstrips = F4_B / 4;
        constexpr int items = R1 * nstrips;
        for (int it = threadIdx.x; it < items; it += F4_THREADS) {
            const int strip = it % nstrips, k1 = it / nstrips;
            const int x0 = 4 * strip;
            const T* rp[R2];
#pragma unroll
            for (int u = 0; u < R2; ++u) rp[u] = bufB + (k1 * R2 + u) * WB + x0;
            T out[R2][4];
            RegStages<T, Q2>::run(rp, out);
#pragma unroll
            for (int v = 0; v < R2; ++v) {
                T* d = dst + (grow0 + k1 * R2 + v) * p0 + c + x0;
#pragma unroll
                for (int x = 0; x < 4; ++x)
                    if (x0 + x < ncols) d[x] = out[v][x];
            }
        }
    }
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

template <class T, bool FIRST, int Q1, int Q2>
static ffa_status launch_reg(const void* src, T* dst, FoldGroup& fg, int64_t m_rows, int s, cudaStream_t st) {
    constexpr int q = Q1 + Q2;
    constexpr int rows = 1 << q;
    const size_t smem = sizeof(T) * ((size_t)rows * f4_wa(q) + (Q2 > 0 ? (size_t)rows * f4_wb(q, Q1) : 0));
    ffa_status es = ensure_smem((const void*)k_fold_reg<T, FIRST, Q1, Q2>, smem);
    if (es != FFA_OK) return es;
    const int64_t units = group_units(fg, m_rows, rows, F4_B);
    if (units <= 0) return FFA_OK;
    k_fold_reg<T, FIRST, Q1, Q2><<<(unsigned)units, F4_THREADS, smem, st>>>(src, dst, fg, s);
    FFA_LAUNCH_CHECK("k_fold_reg");
    count_launch();
    return FFA_OK;
}

template <class T, bool FIRST>
static ffa_status pass_q(int q, const void* src, T* dst, FoldGroup& fg, int64_t m_rows, int s,
                         cudaStream_t st) {
    switch (q) {
        case 1: return launch_reg<T, FIRST, 1, 0>(src, dst, fg, m_rows, s, st);
        case 2: return launch_reg<T, FIRST, 2, 0>(src, dst, fg, m_rows, s, st);
        case 3: return launch_reg<T, FIRST, 3, 0>(src, dst, fg, m_rows, s, st);
        case 4: return launch_reg<T, FIRST, 2, 2>(src, dst, fg, m_rows, s, st);
        case 5: return launch_reg<T, FIRST, 3, 2>(src, dst, fg, m_rows, s, st);
        default: break;
    }
    const int rows = 1 << q;
    const size_t smem = 2 * sizeof(T) * (size_t)rows * (FP_B + rows - 1);
    ffa_status es = ensure_smem((const void*)k_fold_pass<T, FIRST>, smem);
    if (es != FFA_OK) return es;
    const int64_t units = group_units(fg, m_rows, rows, FP_B);
    if (units <= 0) return FFA_OK;
    k_fold_pass<T, FIRST><<<(unsigned)units, FP_THREADS, smem, st>>>(src, dst, fg, s, q);
    FFA_LAUNCH_CHECK("k_fold_pass");
    count_launch();
    return FFA_OK;
}

template <class T>
static ffa_status fold_impl(const void* d_z, FoldGroup& fg, int64_t m_rows, int stages, T* d_plane, T* d_tmp,
                            cudaStream_t st, int qmax) {
    int qs[64];
    int np = split_passes(stages, qmax, qs);
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
        ffa_status e = pi == 0 ? pass_q<T, true>(qs[pi], src, dst, fg, m_rows, s, st)
                               : pass_q<T, false>(qs[pi], src, dst, fg, m_rows, s, st);
        if (e != FFA_OK) return e;
        s += qs[pi];
    }
    return FFA_OK;
}

// ---------------------------------------------------------------------------
// Stages per pass, tuned.  Any split of the stages into passes gives the
// same add tree (bit-identical planes); only the time differs.  The cache
// maps (device, precision, stages, floor(log2 p0)) to the fastest maximum
// pass depth measured by tune_fold; untuned shapes use 5.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tune;
constexpr int QMAX_DEFAULT = 5;

int log2i(int64_t v) {
    int r = 0;
    while ((int64_t)2 << r <= v) ++r;
    return r;
}

int tuned_qmax(int precision, int stages, int64_t p0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return QMAX_DEFAULT;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(dev, precision, stages, log2i(p0)));
    return it == g_tune.end() ? QMAX_DEFAULT : it->second;
}
}  // namespace

static ffa_status fold_group(const void* d_z, int32_t precision, FoldGroup& fg, int64_t m_rows, int stages,
                             void* d_plane, void* d_tmp, cudaStream_t st, int qmax) {
    if (precision == FFA_FOLD_F32)
        return fold_impl<float>(d_z, fg, m_rows, stages, (float*)d_plane, (float*)d_tmp, st, qmax);
    return fold_impl<int32_t>(d_z, fg, m_rows, stages, (int32_t*)d_plane, (int32_t*)d_tmp, st, qmax);
}

ffa_status fold_with(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                     int stages, void* d_plane, void* d_tmp, cudaStream_t st, int qmax) {
    FoldGroup fg;
    fg.n = 1;
    fg.p0[0] = p0;
    fg.m_data[0] = m_data;
    fg.off[0] = 0;
    return fold_group(d_z, precision, fg, m_rows, stages, d_plane, d_tmp, st, qmax);
}

// Time each maximum pass depth 3..5 on one shape (CUDA events, best of 2
// after a warm-up) and cache the fastest.  The planes are scratch.
ffa_status tune_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                     int stages, void* d_plane, void* d_tmp, cudaStream_t st, int* best_q) {
    cudaEvent_t e0, e1;
    FFA_CUDA_TRY(cudaEventCreate(&e0));
    FFA_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bq = QMAX_DEFAULT;
    ffa_status s = FFA_OK;
    for (int q = 3; q <= 5 && s == FFA_OK; ++q) {
        s = fold_with(d_z, precision, p0, m_data, m_rows, stages, d_plane, d_tmp, st, q);  // warm-up
        float t_q = 1e30f;
        for (int rep = 0; rep < 2 && s == FFA_OK; ++rep) {
            cudaEventRecord(e0, st);
            s = fold_with(d_z, precision, p0, m_data, m_rows, stages, d_plane, d_tmp, st, q);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) s = cuda_fail(cudaGetLastError(), "tune_fold");
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            t_q = ms < t_q ? ms : t_q;
        }
        if (t_q < best) {
            best = t_q;
            bq = q;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != FFA_OK) return s;
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[std::make_tuple(dev, precision, stages, log2i(p0))] = bq;
    }
    if (best_q) *best_q = bq;
    return FFA_OK;
}

ffa_status launch_fold_group(const void* d_z, int32_t precision, int n, const int64_t* p0, const int64_t* m_data,
                             const int64_t* off, int64_t m_rows, int stages, void* d_plane, void* d_tmp,
                             cudaStream_t st) {
    if (n < 1 || n > FOLD_GROUP_MAX) return fail(FFA_ERR_ARG, "fold group: 1..FOLD_GROUP_MAX base periods");
    FoldGroup fg;
    fg.n = n;
    for (int i = 0; i < n; ++i) {
        fg.p0[i] = p0[i];
        fg.m_data[i] = m_data[i];
        fg.off[i] = off[i];
    }
    return fold_group(d_z, precision, fg, m_rows, stages, d_plane, d_tmp, st,
                      tuned_qmax(precision, stages, p0[n - 1]));
}

// Run the first `stages` FFA stages (all of them when stages < 0).  With
// fewer stages the plane holds, per group of 2^stages rows, its partial
// trials (row g * 2^stages + kappa); zero stages copy the (zero-padded) rows.
ffa_status launch_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                       int64_t m_rows, int stages, void* d_plane, void* d_tmp, cudaStream_t st) {
    int m = 0;
    while ((1ll << m) < m_rows) ++m;
    if (stages < 0 || stages > m) stages = m;
    return fold_with(d_z, precision, p0, m_data, m_rows, stages, d_plane, d_tmp, st,
                     tuned_qmax(precision, stages, p0));
}

}  // namespace ffa

// ---------------------------------------------------------------------------
// Fold without any allocation (see ffa_fold_noalloc in include/ffa.h).
// ---------------------------------------------------------------------------
namespace {
// Scratch plane shared by every ffa_fold_noalloc call on a device; it lives
// in the module image, so every GPU that loads the library holds it.
static __device__ __align__(256) float g_fold_scratch[FFA_NOALLOC_FOLD_MAX_ELEMS];

std::mutex g_scratch_mu;
void* g_scratch_ptr[64] = {};
}  // namespace

extern "C" ffa_status ffa_fold_noalloc(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                                       int64_t m_rows, void* d_plane, void* stream) {
    using namespace ffa;
    if (p0 < 1 || m_data < 0 || m_rows < 1 || (m_rows & (m_rows - 1)) != 0 || m_data > m_rows)
        return fail(FFA_ERR_ARG, "fold_noalloc: need p0 >= 1, m_rows a power of two >= m_data");
    if (precision != FFA_FOLD_F32 && precision != FFA_FOLD_I8)
        return fail(FFA_ERR_ARG, "fold_noalloc: bad precision");
    if (!d_z || !d_plane) return fail(FFA_ERR_ARG, "fold_noalloc: null buffer");
    if (m_rows * p0 > (int64_t)FFA_NOALLOC_FOLD_MAX_ELEMS)
        return fail(FFA_ERR_UNSUPPORTED,
                    "fold_noalloc: m_rows * p0 exceeds FFA_NOALLOC_FOLD_MAX_ELEMS (the fixed scratch)");
    int dev = 0;
    FFA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(FFA_ERR_UNSUPPORTED, "fold_noalloc: device index >= 64");
    void* scratch;
    {
        // set-up once per device, with that device current: the device address of
        // the array (its host-side name is only a stand-in, not a device address)
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_fold_scratch);
            if (e != cudaSuccess || !ptr) return cuda_fail(e, "fold_noalloc: cudaGetSymbolAddress");
            g_scratch_ptr[dev] = ptr;
        }
        scratch = g_scratch_ptr[dev];
    }
    return launch_fold(d_z, precision, p0, m_data, m_rows, -1, d_plane, scratch, as_stream(stream));
}
