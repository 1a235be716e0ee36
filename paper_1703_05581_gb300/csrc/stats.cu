// Periodogram statistics for false-alarm analysis (Section 4.3): the S/N
// histogram of a search's records, accumulated on the device across searches,
// and the mapping of a histogram's tail probabilities to Gaussian-equivalent
// sigma (each S/N's probability put through the normal quantile function).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ffa {
namespace {

constexpr int HIST_MAX_BINS = 4096;
constexpr int HIST_THREADS = 512;

struct Edges {
    float e[HIST_MAX_BINS + 1];
};

// counts[0]: S/N < edges[0]; counts[1 + b]: edges[b] <= S/N < edges[b + 1];
// counts[n_bins + 1]: S/N >= edges[n_bins].  Per-CTA shared counters, then
// one 64-bit atomic per non-empty bin.
__global__ void __launch_bounds__(HIST_THREADS) k_snr_hist(const ffa_record* __restrict__ rec,
                                                           int64_t n, const Edges edges, int n_bins,
                                                           unsigned long long* __restrict__ counts) {
    __shared__ float e[HIST_MAX_BINS + 1];
    __shared__ uint32_t h[HIST_MAX_BINS + 2];
    for (int b = threadIdx.x; b <= n_bins; b += HIST_THREADS) e[b] = edges.e[b];
    for (int b = threadIdx.x; b < n_bins + 2; b += HIST_THREADS) h[b] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * HIST_THREADS;
    for (int64_t i = (int64_t)blockIdx.x * HIST_THREADS + threadIdx.x; i < n; i += stride) {
        const float s = rec[i].snr;
        // number of edges <= s
        int lo = 0, hi = n_bins + 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (e[mid] <= s) lo = mid + 1;
            else hi = mid;
        }
        atomicAdd(&h[lo], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins + 2; b += HIST_THREADS)
        if (h[b]) atomicAdd(&counts[b], (unsigned long long)h[b]);
}

// Upper-tail normal quantile: the z with Q(z) = erfc(z / sqrt 2) / 2 = p, by
// bisection on the decreasing Q until the bracket stops shrinking (binary64
// resolution).
double upper_normal_quantile(double p) {
    if (!(p > 0.0)) return INFINITY;
    if (p >= 1.0) return -INFINITY;
    const double rs2 = 0.70710678118654752440;  // 1 / sqrt 2
    double a = -40.0, b = 40.0;
    for (int it = 0; it < 2000; ++it) {
        const double m = 0.5 * (a + b);
        if (m <= a || m >= b) break;
        if (0.5 * std::erfc(m * rs2) > p) a = m;
        else b = m;
    }
    return 0.5 * (a + b);
}

}  // namespace
}  // namespace ffa

using namespace ffa;

extern "C" ffa_status ffa_snr_histogram(const ffa_record* d_records, int64_t n, const float* edges,
                                        int32_t n_bins, uint64_t* d_counts, void* stream) {
    if (n < 0) return fail(FFA_ERR_ARG, "snr_histogram: negative count");
    if (n_bins < 1 || n_bins > HIST_MAX_BINS)
        return fail(FFA_ERR_ARG, "snr_histogram: n_bins must be in [1, 4096]");
    if (!edges || !d_counts) return fail(FFA_ERR_ARG, "snr_histogram: null argument");
    for (int b = 0; b < n_bins; ++b)
        if (!(edges[b] < edges[b + 1])) return fail(FFA_ERR_ARG, "snr_histogram: edges must increase");
    if (n == 0) return FFA_OK;
    if (!d_records) return fail(FFA_ERR_ARG, "snr_histogram: null records");
    cudaStream_t st = as_stream(stream);
    Edges e;  // by value: no device allocation
    for (int b = 0; b <= n_bins; ++b) e.e[b] = edges[b];
    const int64_t want = (n + HIST_THREADS - 1) / HIST_THREADS;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count() * 4);
    k_snr_hist<<<grid, HIST_THREADS, 0, st>>>(d_records, n, e, n_bins, (unsigned long long*)d_counts);
    FFA_LAUNCH_CHECK("snr histogram");
    count_launch(1);
    return FFA_OK;
}

extern "C" ffa_status ffa_sigma_gauss(const uint64_t* counts, int32_t n_bins, double* sigma) {
    if (n_bins < 1 || !counts || !sigma) return fail(FFA_ERR_ARG, "sigma_gauss: bad argument");
    uint64_t total = 0;
    for (int b = 0; b < n_bins + 2; ++b) total += counts[b];
    if (total == 0) return fail(FFA_ERR_ARG, "sigma_gauss: empty histogram");
    // tail = trials with S/N >= edges[b] = counts[1 + b] + ... + counts[n_bins + 1]
    uint64_t tail = counts[n_bins + 1];
    std::vector<double> out((size_t)n_bins + 1);
    out[(size_t)n_bins] = upper_normal_quantile((double)tail / (double)total);
    for (int b = n_bins - 1; b >= 0; --b) {
        tail += counts[1 + b];
        out[(size_t)b] = upper_normal_quantile((double)tail / (double)total);
    }
    for (int b = 0; b <= n_bins; ++b) sigma[b] = out[(size_t)b];
    return FFA_OK;
}
