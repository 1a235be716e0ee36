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

#include "common.cuh"
#include "internal.h"

namespace ffa {

constexpr int FOLD_THREADS = 256;

template <class T>
struct FoldIn;
template <>
struct FoldIn<float> { using type = float; };
template <>
struct FoldIn<int32_t> { using type = int8_t; };

// One pass of q stages.  first: read the series (rows >= m_data are zero)
// instead of the previous plane.
template <class T, bool FIRST>
__global__ void __launch_bounds__(FOLD_THREADS) k_fold_pass(
    const void* __restrict__ src_v, T* __restrict__ dst, int64_t p0, int64_t m_rows,
    int64_t m_data, int s, int q, int bw, int64_t n_ct) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int rows = 1 << q;
    const int wt = bw + rows - 1;  // staged width incl. halo
    T* buf0 = reinterpret_cast<T*>(smem_raw);
    T* buf1 = buf0 + rows * wt;

    const int64_t unit = blockIdx.x;
    const int64_t ct = unit % n_ct;
    const int64_t rest = unit / n_ct;
    const int64_t kappa = rest & ((1ll << s) - 1);
    const int64_t blk = rest >> s;
    const int64_t c = ct * bw;

    // stage the 2^q input rows
    for (int u = threadIdx.x / 32; u < rows; u += FOLD_THREADS / 32) {
        const int64_t g = blk * rows + u;  // group index at level s
        int64_t base = (c + (kappa % p0) * (u % p0)) % p0;
        T* rowp = buf0 + u * wt;
        if (FIRST) {
            const typename FoldIn<T>::type* z = (const typename FoldIn<T>::type*)src_v;
            bool live = g < m_data;
            const typename FoldIn<T>::type* zr = z + g * p0;
            for (int x = threadIdx.x & 31; x < wt; x += 32) {
                int64_t col = (base + x) % p0;
                rowp[x] = live ? (T)zr[col] : (T)0;
            }
        } else {
            const T* pl = (const T*)src_v + ((g << s) + kappa) * p0;
            for (int x = threadIdx.x & 31; x < wt; x += 32) {
                int64_t col = (base + x) % p0;
                rowp[x] = pl[col];
            }
        }
    }
    __syncthreads();

    // q local stages
    T* in = buf0;
    T* out = buf1;
    for (int t = 1; t <= q; ++t) {
        const int half = 1 << (t - 1);
        const int width = wt - ((1 << t) - 1);
        for (int r = threadIdx.x / 32; r < rows; r += FOLD_THREADS / 32) {
            const int gb = r & ~((1 << t) - 1);
            const int v = r - gb;
            const T* h = in + (gb + (v >> 1)) * wt;
            const T* tl = in + (gb + half + (v >> 1)) * wt + ((v + 1) >> 1);
            T* o = out + r * wt;
            for (int x = threadIdx.x & 31; x < width; x += 32) o[x] = h[x] + tl[x];
        }
        __syncthreads();
        T* tmp = in;
        in = out;
        out = tmp;
    }

    // write 2^q output rows of the tile
    const int64_t out_row0 = (blk << (s + q)) + (kappa << q);
    const int64_t ncols = (c + bw <= p0) ? bw : p0 - c;
    for (int v = threadIdx.x / 32; v < rows; v += FOLD_THREADS / 32) {
        T* d = dst + (out_row0 + v) * p0 + c;
        const T* sv = in + v * wt;
        for (int x = threadIdx.x & 31; x < ncols; x += 32) d[x] = sv[x];
    }
}

// Split m stages into passes of at most `qmax`, as evenly as possible.
static int split_passes(int m, int qmax, int* qs) {
    if (m == 0) return 0;
    int np = (m + qmax - 1) / qmax;
    for (int i = 0; i < np; ++i) qs[i] = m / np + (i < m % np ? 1 : 0);
    return np;
}

template <class T>
static ffa_status fold_impl(const void* d_z, int64_t p0, int64_t m_data, int64_t m_rows,
                            T* d_plane, T* d_tmp, cudaStream_t st) {
    int m = 0;
    while ((1ll << m) < m_rows) ++m;
    const int qmax = 5;
    const int bw = p0 < 256 ? (int)p0 : 256;
    const int64_t n_ct = (p0 + bw - 1) / bw;
    int qs[64];
    int np = split_passes(m, qmax, qs);
    if (np == 0) {
        // a single row: the fold is the row itself
        np = 1;
        qs[0] = 0;
    }
    // ping-pong so that the last pass lands in d_plane
    T* bufs[2] = {d_plane, d_tmp};
    int s = 0;
    for (int pi = 0; pi < np; ++pi) {
        int q = qs[pi];
        T* dst = bufs[(np - 1 - pi) & 1];
        const void* src = pi == 0 ? d_z : (const void*)bufs[(np - pi) & 1];
        int rows = 1 << q;
        size_t smem = 2 * (size_t)rows * (bw + rows - 1) * sizeof(T);
        int64_t units = (m_rows >> q) * n_ct;
        if (pi == 0) {
            ffa_status es = ensure_smem((const void*)k_fold_pass<T, true>, smem);
            if (es != FFA_OK) return es;
            k_fold_pass<T, true><<<(unsigned)units, FOLD_THREADS, smem, st>>>(
                src, dst, p0, m_rows, m_data, s, q, bw, n_ct);
        } else {
            ffa_status es = ensure_smem((const void*)k_fold_pass<T, false>, smem);
            if (es != FFA_OK) return es;
            k_fold_pass<T, false><<<(unsigned)units, FOLD_THREADS, smem, st>>>(
                src, dst, p0, m_rows, m_data, s, q, bw, n_ct);
        }
        FFA_LAUNCH_CHECK("k_fold_pass");
        count_launch();
        s += q;
    }
    return FFA_OK;
}

ffa_status launch_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                       int64_t m_rows, void* d_plane, void* d_tmp, cudaStream_t st) {
    if (precision == FFA_FOLD_F32)
        return fold_impl<float>(d_z, p0, m_data, m_rows, (float*)d_plane, (float*)d_tmp, st);
    return fold_impl<int32_t>(d_z, p0, m_data, m_rows, (int32_t*)d_plane, (int32_t*)d_tmp, st);
}

}  // namespace ffa
