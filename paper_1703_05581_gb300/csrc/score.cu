// Algorithm 1 of Section 2.2.1 on the GPU: median / MAD normalisation
// (Eq. 3-4) and power-of-two boxcar matched filters, each box sum divided by
// sqrt(width); the score is the best over widths and phases.
//
// One CTA scores one profile held in shared memory.
//   * Median: exact radix select (12 + 12 + 8 key bits) over order-preserving
//     keys of the values; an even count takes the mean of the two middle
//     values in FP64.
//   * MAD (float profiles): the FP32 deviations |x - fl(med)| differ from the
//     exact FP64 deviations |x - med| by at most E = max|x| * 2^-20, and so
//     do their order statistics.  Radix-selecting the FP32 deviations gives
//     brackets [v - E, v + E] for the exact order statistics; only the few
//     samples whose FP32 deviation falls within 3E of the bracket are
//     re-evaluated in FP64 and sorted, which yields the exact MAD.
//   * MAD (int profiles): |2x - (a+b)| is an exact integer; selected directly.
//   * Boxcars: box_2w[j] = box_w[j] + box_w[j+w] (cyclic), the running box
//     values held in registers; max and first argmax per listed width.
//   * S/N_w = (B_w - w*med) / (K*MAD*sqrt(w)) in FP64 with round-to-nearest
//     intrinsics (no fused multiply-add), best = max (ties: smaller width).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace ffa {

constexpr int SC_THREADS = 1024;
constexpr int SC_MAXV = 32;          // values per thread: p0 <= 32768
constexpr int SC_CAP = 1024;         // exact-MAD candidate capacity
constexpr double K_MAD = 1.4826;     // printed after Eq. 4

struct ScShared {
    uint32_t hist[4096];
    double cand[SC_CAP];
    uint32_t tmp[64];
    float ftmp[64];
    int itmp[64];
    double bw_val[16];
    int bw_idx[16];
    uint32_t ccount, cbelow;
    int bin;
    uint32_t below;
};

__device__ __forceinline__ uint32_t vkey(float v) { return fkey(v); }
__device__ __forceinline__ uint32_t vkey(int32_t v) { return ikey(v); }
__device__ __forceinline__ float vfrom(uint32_t k, float*) { return fkey_inv(k); }
__device__ __forceinline__ int32_t vfrom(uint32_t k, int32_t*) { return (int32_t)(k ^ 0x80000000u); }

// exclusive block scan (one value per thread), blockDim multiple of 32
__device__ uint32_t sc_exscan(uint32_t v, uint32_t* s_tmp) {
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
        if (lane < nw) s_tmp[lane] = y;
    }
    __syncthreads();
    uint32_t r = (warp > 0 ? s_tmp[warp - 1] : 0u) + x - v;
    __syncthreads();
    return r;
}

__device__ void sc_find_rank(ScShared& sh, uint32_t rank) {
    const int per = 4096 / SC_THREADS;
    int b0 = threadIdx.x * per;
    uint32_t sum = 0;
    for (int t = 0; t < per; ++t) sum += sh.hist[b0 + t];
    uint32_t ex = sc_exscan(sum, sh.tmp);
    if (rank >= ex && rank < ex + sum) {
        uint32_t c = ex;
        for (int t = 0; t < per; ++t) {
            uint32_t hc = sh.hist[b0 + t];
            if (rank < c + hc) {
                sh.bin = b0 + t;
                sh.below = c;
                break;
            }
            c += hc;
        }
    }
    __syncthreads();
}

// Exact key of the rank-th smallest of keyf(j), j < n.
template <class KeyF>
__device__ uint32_t sc_select(ScShared& sh, int n, uint32_t rank, KeyF keyf) {
    uint32_t prefix = 0, mask = 0;
    const int shifts[3] = {20, 8, 0};
    const uint32_t masks[3] = {0xfffu, 0xfffu, 0xffu};
    for (int pass = 0; pass < 3; ++pass) {
        for (int b = threadIdx.x; b < 4096; b += SC_THREADS) sh.hist[b] = 0;
        __syncthreads();
        const int sh_ = shifts[pass];
        const uint32_t mk = masks[pass];
        for (int j = threadIdx.x; j < n; j += SC_THREADS) {
            uint32_t k = keyf(j);
            if ((k & mask) == prefix) atomicAdd(&sh.hist[(k >> sh_) & mk], 1u);
        }
        __syncthreads();
        sc_find_rank(sh, rank);
        rank -= sh.below;
        prefix |= (uint32_t)sh.bin << sh_;
        mask |= mk << sh_;
        __syncthreads();
    }
    return prefix;
}

__device__ float sc_block_max(float v, ScShared& sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh.ftmp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (SC_THREADS >> 5) ? sh.ftmp[lane] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh.ftmp[0] = v;
    }
    __syncthreads();
    float r = sh.ftmp[0];
    __syncthreads();
    return r;
}

// (max value, smallest index) over the block; result valid in thread 0.
template <class T>
__device__ void sc_block_argmax(T v, int j, ScShared& sh, T* out_v, int* out_j) {
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(0xffffffffu, v, o);
        int k = __shfl_xor_sync(0xffffffffu, j, o);
        if (u > v || (u == v && k < j)) {
            v = u;
            j = k;
        }
    }
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T* vt = reinterpret_cast<T*>(sh.ftmp);
    if (lane == 0) {
        vt[warp] = v;
        sh.itmp[warp] = j;
    }
    __syncthreads();
    if (warp == 0) {
        v = vt[lane];
        j = sh.itmp[lane];
        for (int o = 16; o > 0; o >>= 1) {
            T u = __shfl_xor_sync(0xffffffffu, v, o);
            int k = __shfl_xor_sync(0xffffffffu, j, o);
            if (u > v || (u == v && k < j)) {
                v = u;
                j = k;
            }
        }
        if (lane == 0) {
            *out_v = v;
            *out_j = j;
        }
    }
    __syncthreads();
}

// bitonic sort of sh.cand[0..n) ascending (n <= SC_CAP)
__device__ void sc_sort_cand(ScShared& sh, uint32_t n) {
    uint32_t np2 = 1;
    while (np2 < n) np2 <<= 1;
    for (uint32_t t = n + threadIdx.x; t < np2; t += SC_THREADS) sh.cand[t] = INFINITY;
    __syncthreads();
    for (uint32_t kk = 2; kk <= np2; kk <<= 1) {
        for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
            for (uint32_t t = threadIdx.x; t < np2; t += SC_THREADS) {
                uint32_t u = t ^ jj;
                if (u > t) {
                    bool up = (t & kk) == 0;
                    double a = sh.cand[t], b = sh.cand[u];
                    if ((a > b) == up) {
                        sh.cand[t] = b;
                        sh.cand[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// slow exact path for the float MAD: 64-bit radix select over FP64 deviations
__device__ double sc_select_dev64(ScShared& sh, const float* vals, int n, double med, uint32_t rank) {
    uint64_t prefix = 0, mask = 0;
    for (int pass = 0; pass < 8; ++pass) {
        int shift = 56 - 8 * pass;
        for (int b = threadIdx.x; b < 4096; b += SC_THREADS) sh.hist[b] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += SC_THREADS) {
            uint64_t k = dkey(fabs((double)vals[j] - med));
            if ((k & mask) == prefix) atomicAdd(&sh.hist[(k >> shift) & 0xff], 1u);
        }
        __syncthreads();
        sc_find_rank(sh, rank);
        rank -= sh.below;
        prefix |= (uint64_t)sh.bin << shift;
        mask |= (uint64_t)0xff << shift;
        __syncthreads();
    }
    return dkey_inv(prefix);
}

template <class T>
__global__ void __launch_bounds__(SC_THREADS) k_score(const T* __restrict__ prof, int64_t p0,
                                                      ScoreWidths wd, ffa_record* __restrict__ rec,
                                                      int32_t* d_status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScShared& sh = *reinterpret_cast<ScShared*>(smem_raw);
    T* vals = reinterpret_cast<T*>(smem_raw + sizeof(ScShared));
    const int n = (int)p0;
    const T* src = prof + (int64_t)blockIdx.x * p0;
    for (int j = threadIdx.x; j < n; j += SC_THREADS) vals[j] = src[j];
    __syncthreads();

    const uint32_t r1 = (uint32_t)((n - 1) / 2), r2 = (uint32_t)(n / 2);
    // ---- median (Eq. 3 inner median) ----
    auto key_val = [&](int j) { return vkey(vals[j]); };
    uint32_t ka = sc_select(sh, n, r1, key_val);
    uint32_t kb = (r1 == r2) ? ka : sc_select(sh, n, r2, key_val);
    const T va = vfrom(ka, (T*)nullptr), vb = vfrom(kb, (T*)nullptr);
    const double med = (r1 == r2) ? (double)va : ((double)va + (double)vb) / 2;

    // ---- MAD (Eq. 3) ----
    double mad;
    if constexpr (std::is_floating_point<T>::value) {
        // float profile
        float amax = 0.0f;
        for (int j = threadIdx.x; j < n; j += SC_THREADS) amax = fmaxf(amax, fabsf((float)vals[j]));
        amax = sc_block_max(amax, sh);
        const float m32 = __double2float_rn(med);
        const float E = ldexpf(amax, -20);
        auto key_dev = [&](int j) { return fkey(fabsf((float)vals[j] - m32)); };
        float v1 = fkey_inv(sc_select(sh, n, r1, key_dev));
        float v2 = (r1 == r2) ? v1 : fkey_inv(sc_select(sh, n, r2, key_dev));
        const float lo_w = v1 - 3.0f * E, hi_w = v2 + 3.0f * E;
        if (threadIdx.x == 0) {
            sh.ccount = 0;
            sh.cbelow = 0;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += SC_THREADS) {
            float dt = fabsf((float)vals[j] - m32);
            if (dt < lo_w) {
                atomicAdd(&sh.cbelow, 1u);
            } else if (dt <= hi_w) {
                uint32_t slot = atomicAdd(&sh.ccount, 1u);
                if (slot < SC_CAP) sh.cand[slot] = fabs((double)vals[j] - med);
            }
        }
        __syncthreads();
        const uint32_t cc = sh.ccount, cb = sh.cbelow;
        if (cc <= SC_CAP && cb <= r1 && r2 - cb < cc) {
            sc_sort_cand(sh, cc);
            double d1 = sh.cand[r1 - cb], d2 = sh.cand[r2 - cb];
            mad = (r1 == r2) ? d1 : (d1 + d2) / 2;
        } else {
            if (cc <= SC_CAP) dev_fail(d_status, FFA_ERR_DEVICE);  // bracket invariant broken
            double d1 = sc_select_dev64(sh, (const float*)vals, n, med, r1);
            double d2 = (r1 == r2) ? d1 : sc_select_dev64(sh, (const float*)vals, n, med, r2);
            mad = (r1 == r2) ? d1 : (d1 + d2) / 2;
        }
        __syncthreads();
    } else {
        // int profile: e = |2x - (a + b)| is an exact integer, d = e / 2
        const int64_t s2 = (r1 == r2) ? 2 * (int64_t)va : (int64_t)va + (int64_t)vb;
        auto key_e = [&](int j) {
            int64_t e = 2 * (int64_t)vals[j] - s2;
            return (uint32_t)(e < 0 ? -e : e);
        };
        uint32_t e1 = sc_select(sh, n, r1, key_e);
        uint32_t e2 = (r1 == r2) ? e1 : sc_select(sh, n, r2, key_e);
        mad = (r1 == r2) ? (double)e1 / 2 : ((double)e1 + (double)e2) / 4;
    }

    // ---- boxcars (Section 2.2.1) ----
    T v[SC_MAXV];
#pragma unroll
    for (int t = 0; t < SC_MAXV; ++t) {
        int j = threadIdx.x + t * SC_THREADS;
        v[t] = j < n ? vals[j] : (T)0;
    }
    int wi = 0;
    for (int w = 1; w <= wd.w[wd.n - 1]; w <<= 1) {
        if (w == wd.w[wi]) {
            T best = (T)0;
            int bj = 0x7fffffff;
            bool have = false;
#pragma unroll
            for (int t = 0; t < SC_MAXV; ++t) {
                int j = threadIdx.x + t * SC_THREADS;
                if (j < n && (!have || v[t] > best)) {
                    best = v[t];
                    bj = j;
                    have = true;
                }
            }
            if (!have) {
                if constexpr (std::is_floating_point<T>::value) best = -INFINITY;
                else best = INT32_MIN;
            }
            T bv;
            int bjj;
            sc_block_argmax<T>(best, bj, sh, &bv, &bjj);
            if (threadIdx.x == 0) {
                sh.bw_val[wi] = (double)bv;
                sh.bw_idx[wi] = bjj;
            }
            ++wi;
        }
        if (2 * w > wd.w[wd.n - 1]) break;
        // box_2w[j] = box_w[j] + box_w[(j + w) mod p0]
        __syncthreads();
#pragma unroll
        for (int t = 0; t < SC_MAXV; ++t) {
            int j = threadIdx.x + t * SC_THREADS;
            if (j < n) vals[j] = v[t];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < SC_MAXV; ++t) {
            int j = threadIdx.x + t * SC_THREADS;
            if (j < n) {
                int jj = j + w;
                jj = jj % n;
                v[t] = v[t] + vals[jj];
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        ffa_record r;
        if (!(mad > 0.0)) {
            r.snr = 0.0f;
            r.width = wd.w[0];
            r.phase = 0;
            r.flags = 1;
        } else {
            double best = -INFINITY;
            int bw = wd.w[0], bj = 0;
            const double kmad = __dmul_rn(K_MAD, mad);
            for (int t = 0; t < wd.n; ++t) {
                double w = (double)wd.w[t];
                double num = __dsub_rn(sh.bw_val[t], __dmul_rn(w, med));
                double den = __dmul_rn(kmad, __dsqrt_rn(w));
                double snr = __ddiv_rn(num, den);
                if (snr > best) {
                    best = snr;
                    bw = wd.w[t];
                    bj = sh.bw_idx[t];
                }
            }
            r.snr = __double2float_rn(best);
            r.width = bw;
            r.phase = bj;
            r.flags = 0;
        }
        rec[blockIdx.x] = r;
    }
}

size_t score_smem_bytes(int64_t p0) { return sizeof(ScShared) + (size_t)p0 * 4; }

ffa_status launch_score(const void* d_prof, int32_t precision, int64_t count, int64_t p0,
                        const ScoreWidths& wd, ffa_record* d_rec, int32_t* d_status,
                        cudaStream_t st) {
    if (count <= 0) return FFA_OK;
    if (p0 < 1 || p0 > SC_THREADS * SC_MAXV) return fail(FFA_ERR_UNSUPPORTED, "score: p0 > 32768");
    size_t smem = score_smem_bytes(p0);
    if (precision == FFA_FOLD_F32) {
        ffa_status es = ensure_smem((const void*)k_score<float>, smem);
        if (es != FFA_OK) return es;
        k_score<float><<<(unsigned)count, SC_THREADS, smem, st>>>((const float*)d_prof, p0, wd, d_rec,
                                                                   d_status);
    } else {
        ffa_status es = ensure_smem((const void*)k_score<int32_t>, smem);
        if (es != FFA_OK) return es;
        k_score<int32_t><<<(unsigned)count, SC_THREADS, smem, st>>>((const int32_t*)d_prof, p0, wd,
                                                                     d_rec, d_status);
    }
    FFA_LAUNCH_CHECK("k_score");
    count_launch();
    return FFA_OK;
}

}  // namespace ffa
