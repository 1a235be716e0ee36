// Internal launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ffa.h"

namespace ffa {

struct ScoreWidths {
    int32_t n;
    int32_t w[16];
};

// Process-wide count of kernel launches made by the library.
void count_launch(int64_t n = 1);

// Raise a kernel's dynamic shared memory limit once per (kernel, device).
ffa_status ensure_smem(const void* func, size_t bytes);

ffa_status launch_downsample(const void* d_in, int32_t in_type, int64_t n, int64_t f,
                             double* d_out, cudaStream_t st);
ffa_status launch_detrend(const double* d_raw, int64_t n, int32_t window, double* d_resid,
                          int32_t* d_status, cudaStream_t st);
ffa_status launch_normalise(const double* d_resid, int64_t n, int32_t precision, void* d_out,
                            double* d_stats, cudaStream_t st);
ffa_status launch_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                       int64_t m_rows, int stages, void* d_plane, void* d_tmp, cudaStream_t st);
// Algorithm 1 on `count` trials starting at trial0.  fused: d_prof is the
// plane after all but the last FFA stage (m_rows rows); the kernel applies the
// last stage while loading.  Otherwise d_prof holds ready profiles.
ffa_status launch_score2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                         int64_t trial0, int64_t p0, int64_t m_rows, const ScoreWidths& wd,
                         ffa_record* d_rec, int32_t* d_status, cudaStream_t st);
// Algorithm 2 (Section 2.2.2) with the same fused/unfused inputs.
ffa_status launch_score_alg2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                             int64_t trial0, int64_t p0, int64_t m_rows, const ScoreWidths& wd,
                             float excl_frac, ffa_record* d_rec, cudaStream_t st);

constexpr int STATS_DOUBLES = 2 + 1024;  // {mean, std} + reduction partials

}  // namespace ffa
