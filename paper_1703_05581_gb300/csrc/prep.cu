// Series preparation on the GPU (Section 2.3 of the paper):
//   * pre-downsampling by D0 and per-octave downsampling by 2 (FP64 sums);
//   * the dynamic running-median dereddening, exact;
//   * FP64 normalisation to FP32 z, or to the int8 code q = clip(rint(16 z)).
//
// Running median design (exact, tiled).  A CTA owns T consecutive outputs
// a..l.  Their windows all contain the core C = [s_l, e_a]; window i is C
// plus |F_i| <= T-1 fringe samples.  The rank-r element of window i lies
// between C's order statistics (r - |F_i|) and r, so with
//   rho_lo = min_i (r1_i - |F_i|),  rho_hi = max_i r2_i
// every median of the tile lies in [C_(rho_lo), C_(rho_hi)].  Two histogram
// passes over C (on the top 12 and next 12 bits of an order-preserving
// 64-bit key) find the 24-bit key prefixes P_lo, P_hi of those two order
// statistics.  The samples of the tile's union whose prefix lies in
// [P_lo, P_hi] are the only possible medians (about T of them); they are
// sorted in shared memory and each thread walks the sorted list counting the
// ones inside its own window, starting from the exact number of window
// samples below P_lo.  T <= (W+1)/4 keeps rho_lo >= 0 and rho_hi < |C|.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace ffa {

// ---------------------------------------------------------------------------
// downsampling
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_downsample(const T* __restrict__ x, int64_t m, int64_t f,
                             double* __restrict__ y) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const T* p = x + f * i;
        double s = 0.0;
        for (int64_t j = 0; j < f; ++j) s += (double)p[j];
        y[i] = s;
    }
}

__global__ void k_downsample2(const double* __restrict__ x, int64_t m, double* __restrict__ y) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        double2 v = reinterpret_cast<const double2*>(x)[i];
        y[i] = (0.0 + v.x) + v.y;
    }
}

static int grid_for(int64_t m, int block) {
    int64_t g = (m + block - 1) / block;
    int64_t cap = (int64_t)sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

ffa_status launch_downsample(const void* d_in, int32_t in_type, int64_t n, int64_t f,
                             double* d_out, cudaStream_t st) {
    int64_t m = n / f;
    if (m <= 0) return FFA_OK;
    if (in_type == FFA_IN_F64 && f == 2 && ((uintptr_t)d_in % 16) == 0) {
        k_downsample2<<<grid_for(m, 256), 256, 0, st>>>((const double*)d_in, m, d_out);
    } else if (in_type == FFA_IN_F32) {
        k_downsample<float><<<grid_for(m, 256), 256, 0, st>>>((const float*)d_in, m, f, d_out);
    } else if (in_type == FFA_IN_U8) {
        k_downsample<uint8_t><<<grid_for(m, 256), 256, 0, st>>>((const uint8_t*)d_in, m, f, d_out);
    } else if (in_type == FFA_IN_F64) {
        k_downsample<double><<<grid_for(m, 256), 256, 0, st>>>((const double*)d_in, m, f, d_out);
    } else {
        return fail(FFA_ERR_ARG, "downsample: bad input type");
    }
    FFA_LAUNCH_CHECK("k_downsample");
    count_launch();
    return FFA_OK;
}

// ---------------------------------------------------------------------------
// block-wide helpers
// ---------------------------------------------------------------------------
template <class V>
__device__ V block_reduce_min(V v, V* s_tmp) {
    for (int o = 16; o > 0; o >>= 1) {
        V u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_tmp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        v = lane < nw ? s_tmp[lane] : s_tmp[0];
        for (int o = 16; o > 0; o >>= 1) {
            V u = __shfl_xor_sync(0xffffffffu, v, o);
            v = u < v ? u : v;
        }
        if (lane == 0) s_tmp[0] = v;
    }
    __syncthreads();
    V r = s_tmp[0];
    __syncthreads();
    return r;
}

template <class V>
__device__ V block_reduce_max(V v, V* s_tmp) {
    for (int o = 16; o > 0; o >>= 1) {
        V u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) s_tmp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        v = lane < nw ? s_tmp[lane] : s_tmp[0];
        for (int o = 16; o > 0; o >>= 1) {
            V u = __shfl_xor_sync(0xffffffffu, v, o);
            v = u > v ? u : v;
        }
        if (lane == 0) s_tmp[0] = v;
    }
    __syncthreads();
    V r = s_tmp[0];
    __syncthreads();
    return r;
}

// Exclusive prefix sum over the block of one uint32 per thread.
__device__ uint32_t block_exscan(uint32_t v, uint32_t* s_tmp, uint32_t* total) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += u;
    }
    __syncthreads();
    if (lane == 31) s_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        uint32_t y = lane < nw ? s_tmp[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += u;
        }
        if (lane < nw) s_tmp[lane] = y;  // inclusive warp totals
    }
    __syncthreads();
    uint32_t base = warp > 0 ? s_tmp[warp - 1] : 0u;
    if (total) *total = s_tmp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

// Find the bin of a histogram (nbins a multiple of blockDim) that holds the
// element of 0-based rank `rank`; returns it via *bin and the count of
// elements in lower bins via *below.  Requires rank < total.
__device__ void block_find_rank(const uint32_t* hist, int nbins, uint32_t rank, uint32_t* s_tmp,
                                int* s_bin, uint32_t* s_below) {
    int per = nbins / blockDim.x;
    int b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (int t = 0; t < per; ++t) sum += hist[b0 + t];
    uint32_t ex = block_exscan(sum, s_tmp, nullptr);
    if (rank >= ex && rank < ex + sum) {
        uint32_t c = ex;
        for (int t = 0; t < per; ++t) {
            uint32_t hcount = hist[b0 + t];
            if (rank < c + hcount) {
                *s_bin = b0 + t;
                *s_below = c;
                break;
            }
            c += hcount;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// small windows (W <= 127): direct rank counting per output
// ---------------------------------------------------------------------------
__global__ void k_runmed_small(const double* __restrict__ x, int64_t n, int64_t w,
                               double* __restrict__ resid) {
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t h = w / 2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        int64_t s = i - h < 0 ? 0 : i - h;
        int64_t e = i + h > n - 1 ? n - 1 : i + h;
        int64_t cnt = e - s + 1;
        int64_t r1 = (cnt - 1) / 2, r2 = cnt / 2;
        double v1 = 0.0, v2 = 0.0;
        for (int64_t j = s; j <= e; ++j) {
            double v = x[j];
            int64_t lt = 0, le = 0;
            for (int64_t t = s; t <= e; ++t) {
                double u = x[t];
                lt += (u < v);
                le += (u <= v);
            }
            if (lt <= r1 && r1 < le) v1 = v;
            if (lt <= r2 && r2 < le) v2 = v;
        }
        double med = (r1 == r2) ? v1 : (v1 + v2) / 2;
        resid[i] = x[i] - med;
    }
}

// ---------------------------------------------------------------------------
// tiled exact running median
// ---------------------------------------------------------------------------
constexpr int RM_CAP = 4096;    // candidate capacity (power of two)
constexpr int RM_MAXT = 1024;   // largest tile

struct RmShared {
    uint32_t hist1[4096];
    uint32_t hist2a[4096];
    uint32_t hist2b[4096];
    uint64_t ckey[RM_CAP];
    uint32_t coff[RM_CAP];
    uint32_t lflag[RM_MAXT + 1];
    uint32_t rflag[RM_MAXT + 1];
    uint32_t tmp[64];
    int64_t tmp64[64];
    unsigned long long kmin, kmax;
    uint32_t ccount;
    int bin_a, bin_b;
    uint32_t below_a, below_b;
};

// Exact rank-`rank` key of x[s..e] by an 8-pass, 8-bit radix select over the
// whole CTA (slow path for tiles whose candidate set overflows).
__device__ uint64_t cta_select_key(const double* __restrict__ x, int64_t s, int64_t e, uint32_t rank,
                                   RmShared& sh) {
    uint64_t prefix = 0, mask = 0;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < 256; b += blockDim.x) sh.hist1[b] = 0;
        __syncthreads();
        for (int64_t p = s + threadIdx.x; p <= e; p += blockDim.x) {
            uint64_t k = dkey(x[p]);
            if ((k & mask) == prefix) atomicAdd(&sh.hist1[(k >> shift) & 0xff], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t c = 0;
            for (int b = 0; b < 256; ++b) {
                if (rank < c + sh.hist1[b]) {
                    sh.bin_a = b;
                    sh.below_a = c;
                    break;
                }
                c += sh.hist1[b];
            }
        }
        __syncthreads();
        rank -= sh.below_a;
        prefix |= (uint64_t)sh.bin_a << shift;
        mask |= (uint64_t)0xff << shift;
        __syncthreads();
    }
    return prefix;
}

__global__ void __launch_bounds__(1024) k_runmed_tile(const double* __restrict__ x, int64_t n,
                                                      int64_t w, double* __restrict__ resid,
                                                      int32_t* d_status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    RmShared& sh = *reinterpret_cast<RmShared*>(smem_raw);
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int64_t h = w / 2;
    const int64_t a = (int64_t)blockIdx.x * T;
    const int64_t l = (a + T < n ? a + T : n) - 1;
    const int64_t i = a + tid;
    const bool active = i <= l;
    auto win_s = [&](int64_t q) { return q - h < 0 ? (int64_t)0 : q - h; };
    auto win_e = [&](int64_t q) { return q + h > n - 1 ? n - 1 : q + h; };
    const int64_t s_a = win_s(a), e_a = win_e(a), s_l = win_s(l), e_l = win_e(l);
    const int64_t c0 = s_l, c1 = e_a;
    const int64_t csize = c1 - c0 + 1;
    const int64_t s_i = win_s(active ? i : l), e_i = win_e(active ? i : l);
    const int64_t n_i = e_i - s_i + 1;
    const int64_t f_i = n_i - csize;
    const int64_t r1 = (n_i - 1) / 2, r2 = n_i / 2;

    int64_t lo_need = block_reduce_min<int64_t>(active ? r1 - f_i : INT64_MAX, sh.tmp64);
    int64_t hi_need = block_reduce_max<int64_t>(active ? r2 : INT64_MIN, sh.tmp64);
    bool bracket_ok = csize > 0 && lo_need >= 0 && hi_need < csize;

    bool fast = false;
    if (bracket_ok) {
        const uint32_t rho_lo = (uint32_t)lo_need, rho_hi = (uint32_t)hi_need;
        // pass 1: top 12 key bits over the core
        for (int b = tid; b < 4096; b += T) {
            sh.hist1[b] = 0;
            sh.hist2a[b] = 0;
            sh.hist2b[b] = 0;
        }
        __syncthreads();
        for (int64_t p = c0 + tid; p <= c1; p += T) atomicAdd(&sh.hist1[dkey(x[p]) >> 52], 1u);
        __syncthreads();
        block_find_rank(sh.hist1, 4096, rho_lo, sh.tmp, &sh.bin_a, &sh.below_a);
        block_find_rank(sh.hist1, 4096, rho_hi, sh.tmp, &sh.bin_b, &sh.below_b);
        const uint32_t b1_lo = sh.bin_a, b1_hi = sh.bin_b;
        const uint32_t below1_lo = sh.below_a, below1_hi = sh.below_b;
        __syncthreads();
        // pass 2: next 12 bits inside the two selected top buckets
        for (int64_t p = c0 + tid; p <= c1; p += T) {
            uint64_t k = dkey(x[p]);
            uint32_t top = (uint32_t)(k >> 52), sub = (uint32_t)(k >> 40) & 0xfff;
            if (top == b1_lo) atomicAdd(&sh.hist2a[sub], 1u);
            if (top == b1_hi && b1_hi != b1_lo) atomicAdd(&sh.hist2b[sub], 1u);
        }
        __syncthreads();
        block_find_rank(sh.hist2a, 4096, rho_lo - below1_lo, sh.tmp, &sh.bin_a, &sh.below_a);
        const uint32_t b2_lo = sh.bin_a, below2_lo = sh.below_a;
        __syncthreads();
        block_find_rank(b1_hi == b1_lo ? sh.hist2a : sh.hist2b, 4096, rho_hi - below1_hi, sh.tmp,
                        &sh.bin_b, &sh.below_b);
        const uint32_t b2_hi = sh.bin_b;
        const uint64_t p_lo = ((uint64_t)b1_lo << 12) | b2_lo;
        const uint64_t p_hi = ((uint64_t)b1_hi << 12) | b2_hi;
        const uint32_t c_below = below1_lo + below2_lo;  // core samples with prefix < p_lo
        // gather candidates from the union [s_a, e_l]; flag fringe samples below p_lo
        if (tid == 0) {
            sh.ccount = 0;
            sh.kmin = ~0ull;
            sh.kmax = 0ull;
        }
        for (int t = tid; t <= RM_MAXT; t += T) {
            sh.lflag[t] = 0;
            sh.rflag[t] = 0;
        }
        __syncthreads();
        for (int64_t p = s_a + tid; p <= e_l; p += T) {
            uint64_t k = dkey(x[p]);
            uint64_t pre = k >> 40;
            if (pre >= p_lo && pre <= p_hi) {
                uint32_t slot = atomicAdd(&sh.ccount, 1u);
                if (slot < RM_CAP) {
                    sh.ckey[slot] = k;
                    sh.coff[slot] = (uint32_t)(p - s_a);
                }
                atomicMin(&sh.kmin, (unsigned long long)k);
                atomicMax(&sh.kmax, (unsigned long long)k);
            }
            if (p < s_l) sh.lflag[p - s_a] = pre < p_lo;
            if (p > e_a) sh.rflag[p - e_a - 1] = pre < p_lo;
        }
        __syncthreads();
        const uint32_t cc = sh.ccount;
        if (cc > RM_CAP && sh.kmin == sh.kmax) {
            // every possible median has the same value
            if (active) resid[i] = x[i] - dkey_inv(sh.kmin);
            return;
        }
        if (cc <= RM_CAP) {
            fast = true;
            // fringe counts: left suffix sums, right prefix sums
            uint32_t lsz = (uint32_t)(s_l - s_a), rsz = (uint32_t)(e_l - e_a);
            uint32_t lv = (uint32_t)tid < lsz ? sh.lflag[tid] : 0u;
            uint32_t rv = (uint32_t)tid < rsz ? sh.rflag[tid] : 0u;
            uint32_t ltot, rtot;
            uint32_t lex = block_exscan(lv, sh.tmp, &ltot);
            uint32_t rex = block_exscan(rv, sh.tmp, &rtot);
            // lflag[t] <- number flagged in [t, lsz); rflag[t] <- number flagged in [0, t]
            __syncthreads();
            if ((uint32_t)tid < lsz) sh.lflag[tid] = ltot - lex;
            if ((uint32_t)tid == lsz) sh.lflag[tid] = 0;
            if ((uint32_t)tid < rsz) sh.rflag[tid] = rex + rv;
            // bitonic sort of the candidates by key
            uint32_t np2 = 1;
            while (np2 < cc) np2 <<= 1;
            for (uint32_t t = cc + tid; t < np2; t += T) {
                sh.ckey[t] = ~0ull;
                sh.coff[t] = 0xffffffffu;
            }
            __syncthreads();
            for (uint32_t kk = 2; kk <= np2; kk <<= 1) {
                for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
                    for (uint32_t t = tid; t < np2; t += T) {
                        uint32_t u = t ^ jj;
                        if (u > t) {
                            bool up = (t & kk) == 0;
                            uint64_t kt = sh.ckey[t], ku = sh.ckey[u];
                            if ((kt > ku) == up) {
                                sh.ckey[t] = ku;
                                sh.ckey[u] = kt;
                                uint32_t o = sh.coff[t];
                                sh.coff[t] = sh.coff[u];
                                sh.coff[u] = o;
                            }
                        }
                    }
                    __syncthreads();
                }
            }
            if (active) {
                uint32_t lcnt = (s_i < s_l) ? sh.lflag[(uint32_t)(s_i - s_a)] : 0u;
                uint32_t rcnt = (e_i > e_a) ? sh.rflag[(uint32_t)(e_i - e_a - 1)] : 0u;
                int64_t below = (int64_t)c_below + lcnt + rcnt;
                int64_t t1 = r1 - below, t2 = r2 - below;
                uint32_t so = (uint32_t)(s_i - s_a), eo = (uint32_t)(e_i - s_a);
                int64_t c = 0;
                uint64_t k1 = 0, k2 = 0;
                bool got2 = false;
                if (t1 >= 0) {
                    for (uint32_t j = 0; j < cc; ++j) {
                        uint32_t off = sh.coff[j];
                        if (off >= so && off <= eo) {
                            if (c == t1) k1 = sh.ckey[j];
                            if (c == t2) {
                                k2 = sh.ckey[j];
                                got2 = true;
                                break;
                            }
                            ++c;
                        }
                    }
                }
                if (!got2) {
                    dev_fail(d_status, FFA_ERR_DEVICE);
                    resid[i] = __longlong_as_double(0x7ff8000000000000ll);
                } else {
                    double v1 = dkey_inv(k1), v2 = dkey_inv(k2);
                    double med = (t1 == t2) ? v1 : (v1 + v2) / 2;
                    resid[i] = x[i] - med;
                }
            }
            return;
        }
    }
    if (!fast) {
        if (!bracket_ok) dev_fail(d_status, FFA_ERR_DEVICE);
        // slow exact path: per output, radix select over its own window
        for (int64_t q = a; q <= l; ++q) {
            int64_t s = win_s(q), e = win_e(q);
            int64_t cnt = e - s + 1;
            uint64_t k1 = cta_select_key(x, s, e, (uint32_t)((cnt - 1) / 2), sh);
            uint64_t k2 = (cnt % 2 == 1) ? k1 : cta_select_key(x, s, e, (uint32_t)(cnt / 2), sh);
            if (tid == 0) {
                double v1 = dkey_inv(k1), v2 = dkey_inv(k2);
                double med = (cnt % 2 == 1) ? v1 : (v1 + v2) / 2;
                resid[q] = x[q] - med;
            }
            __syncthreads();
        }
    }
}

ffa_status launch_detrend(const double* d_raw, int64_t n, int32_t window, double* d_resid,
                          int32_t* d_status, cudaStream_t st) {
    if (n <= 0) return FFA_OK;
    int64_t w = window | 1;
    if (w <= 127) {
        k_runmed_small<<<grid_for(n, 256), 256, 0, st>>>(d_raw, n, w, d_resid);
        FFA_LAUNCH_CHECK("k_runmed_small");
        count_launch();
        return FFA_OK;
    }
    int T = 32;
    while (T * 2 <= RM_MAXT && T * 2 <= (w + 1) / 4) T *= 2;
    size_t smem = sizeof(RmShared);
    ffa_status es = ensure_smem((const void*)k_runmed_tile, smem);
    if (es != FFA_OK) return es;
    int64_t tiles = (n + T - 1) / T;
    k_runmed_tile<<<(unsigned)tiles, T, smem, st>>>(d_raw, n, w, d_resid, d_status);
    FFA_LAUNCH_CHECK("k_runmed_tile");
    count_launch();
    return FFA_OK;
}

// ---------------------------------------------------------------------------
// normalisation: FP64 mean and population std (fixed reduction tree)
// ---------------------------------------------------------------------------
constexpr int NRM_BLOCKS = 1024;
constexpr int NRM_THREADS = 256;

__device__ double block_sum_d(double v, double* s) {
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] = s[threadIdx.x] + s[threadIdx.x + o];
        __syncthreads();
    }
    double r = s[0];
    __syncthreads();
    return r;
}

// mode 0: partial sums of r; mode 1: partial sums of (r - mean)^2
__global__ void __launch_bounds__(NRM_THREADS) k_stats_partial(const double* __restrict__ r,
                                                               int64_t n, const double* stats,
                                                               int mode, double* partial) {
    __shared__ double s[NRM_THREADS];
    int64_t chunk = (n + NRM_BLOCKS - 1) / NRM_BLOCKS;
    int64_t b0 = (int64_t)blockIdx.x * chunk;
    int64_t b1 = b0 + chunk < n ? b0 + chunk : n;
    double mean = mode ? stats[0] : 0.0;
    double acc = 0.0;
    for (int64_t p = b0 + threadIdx.x; p < b1; p += NRM_THREADS) {
        double v = r[p];
        if (mode) {
            double d = v - mean;
            acc = acc + __dmul_rn(d, d);
        } else {
            acc = acc + v;
        }
    }
    double t = block_sum_d(acc, s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NRM_BLOCKS) k_stats_final(int64_t n, int mode, double* stats,
                                                            const double* partial) {
    __shared__ double s[NRM_BLOCKS];
    double t = block_sum_d(partial[threadIdx.x], s);
    if (threadIdx.x == 0) {
        if (mode == 0) stats[0] = n > 0 ? t / (double)n : 0.0;
        else stats[1] = n > 0 ? sqrt(t / (double)n) : 0.0;
    }
}

// z = (r - mean) / sd in FP64 (0 for a constant series); bits[i] = z > cutoff
// (uncapped) when bits is given; then the cap z = min(max(z, -clip), clip)
// (clip = +inf when off) before the FP32 rounding or the int8 code.
__global__ void k_normalise_f32(const double* __restrict__ r, int64_t n, const double* stats,
                                double clip, double cutoff, int8_t* __restrict__ bits,
                                float* __restrict__ z) {
    double mean = stats[0], sd = stats[1];
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = sd > 0.0 ? __ddiv_rn(r[i] - mean, sd) : 0.0;
        if (bits) bits[i] = v > cutoff ? 1 : 0;
        v = fmin(fmax(v, -clip), clip);
        z[i] = __double2float_rn(v);
    }
}

__global__ void k_normalise_i8(const double* __restrict__ r, int64_t n, const double* stats,
                               double clip, double cutoff, int8_t* __restrict__ bits,
                               int8_t* __restrict__ q) {
    double mean = stats[0], sd = stats[1];
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double v = sd > 0.0 ? __ddiv_rn(r[i] - mean, sd) : 0.0;
        if (bits) bits[i] = v > cutoff ? 1 : 0;
        v = fmin(fmax(v, -clip), clip);
        double c = rint(16.0 * v);
        c = c > 127.0 ? 127.0 : (c < -127.0 ? -127.0 : c);
        q[i] = (int8_t)(int)c;
    }
}

ffa_status launch_normalise(const double* d_resid, int64_t n, int32_t precision, void* d_out,
                            double* d_stats, cudaStream_t st, float clip, float cutoff,
                            int8_t* d_bits) {
    if (n <= 0) return FFA_OK;
    const double cl = clip > 0.0f ? (double)clip : INFINITY;
    double* partial = d_stats + 2;
    k_stats_partial<<<NRM_BLOCKS, NRM_THREADS, 0, st>>>(d_resid, n, d_stats, 0, partial);
    k_stats_final<<<1, NRM_BLOCKS, 0, st>>>(n, 0, d_stats, partial);
    k_stats_partial<<<NRM_BLOCKS, NRM_THREADS, 0, st>>>(d_resid, n, d_stats, 1, partial);
    k_stats_final<<<1, NRM_BLOCKS, 0, st>>>(n, 1, d_stats, partial);
    if (precision == FFA_FOLD_F32)
        k_normalise_f32<<<grid_for(n, 256), 256, 0, st>>>(d_resid, n, d_stats, cl, (double)cutoff,
                                                          d_bits, (float*)d_out);
    else
        k_normalise_i8<<<grid_for(n, 256), 256, 0, st>>>(d_resid, n, d_stats, cl, (double)cutoff,
                                                         d_bits, (int8_t*)d_out);
    FFA_LAUNCH_CHECK("k_normalise");
    count_launch(5);
    return FFA_OK;
}

}  // namespace ffa
