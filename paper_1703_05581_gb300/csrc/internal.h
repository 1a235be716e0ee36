// Internal launchers shared between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ffa.h"

// The search plan (host only): base periods in periodogram order, per-octave
// bookkeeping and the byte offsets of the workspace regions.
struct ffa_plan {
    ffa_search_config cfg;
    int64_t n = 0;       // input samples
    int64_t n0 = 0;      // after pre-downsampling
    int32_t window = 1;  // odd running-median window (1 = off)
    int32_t n_octaves = 0;
    int64_t n_trials = 0;
    int64_t max_plane = 0;  // largest m_rows * p0
    int64_t plane_elems = 0;  // elements of each plane buffer (>= max_plane; room for grouped planes)
    std::vector<ffa_plan_entry> entries;
    std::vector<int64_t> oct_first, oct_count, oct_n;
    // workspace layout (bytes)
    size_t off_raw_a = 0, off_raw_b = 0, off_resid = 0, off_z = 0, off_stats = 0, off_plane0 = 0,
           off_plane1 = 0, off_cand = 0, off_best = 0, off_bits = 0, ws_bytes = 0;
};


namespace ffa {

struct ScoreWidths {
    int32_t n;
    int32_t w[16];
};

// Process-wide count of kernel launches made by the library.
void count_launch(int64_t n = 1);

// Streaming multiprocessors of the current device (queried once per device;
// 1 if the query fails).  Grid sizes are multiples of it.
int sm_count();

// Raise a kernel's dynamic shared memory limit once per (kernel, device).
ffa_status ensure_smem(const void* func, size_t bytes);

ffa_status launch_downsample(const void* d_in, int32_t in_type, int64_t n, int64_t f,
                             double* d_out, cudaStream_t st);
ffa_status launch_detrend(const double* d_raw, int64_t n, int32_t window, double* d_resid,
                          int32_t* d_status, cudaStream_t st);
// clip > 0 caps the normalised series at +-clip; d_bits (optional) receives
// z > cutoff per sample (1/0, before the cap).
ffa_status launch_normalise(const double* d_resid, int64_t n, int32_t precision, void* d_out,
                            double* d_stats, cudaStream_t st, float clip = 0.0f,
                            float cutoff = 0.0f, int8_t* d_bits = nullptr);
// Persistence (Section 5) of `count` trials: d_bplane is the folded 0/1
// series after all but the last FFA stage (m_rows rows of p0, int32); each
// trial's sum over its record's best window, last stage applied on the fly.
ffa_status launch_persist(const int32_t* d_bplane, int64_t m_rows, int64_t p0, int64_t ld,
                          const ffa_record* d_rec, uint32_t* d_persist, cudaStream_t st);
// Row pitch (elements) of a fold plane inside a search: P0 rounded up to a
// multiple of 4, so every row starts on a 16-byte boundary.  Columns
// [p0, pitch) are padding that no reader uses.
inline int64_t plane_pitch(int64_t p0) { return (p0 + 3) & ~(int64_t)3; }

// Base periods per grouped launch (fold, score): small planes are folded
// and scored together so that a launch fills the GPU.
constexpr int FOLD_GROUP_MAX = 32;
// Fold n base periods sharing m_rows (and their tuned pass depth) in one set
// of launches: entry i has p0[i] bins, m_data[i] rows of the series z[i]
// (host array of device pointers, or null: every entry reads d_z), its plane
// at element offset off[i] of d_plane / d_tmp, rows plane_pitch(p0[i]) apart.
ffa_status launch_fold_group(const void* d_z, int32_t precision, int n, const int64_t* p0, const int64_t* m_data,
                             const int64_t* off, int64_t m_rows, int stages, void* d_plane, void* d_tmp,
                             cudaStream_t st, const void* const* z = nullptr);
// One base period; the plane's rows are `ld` elements apart (ld >= p0).
ffa_status launch_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                       int64_t m_rows, int stages, int64_t ld, void* d_plane, void* d_tmp, cudaStream_t st);
// Time pass depths 3..6 with tiles of 128 and 256 columns for one fold shape
// and cache the fastest (used by every later launch_fold of that precision,
// stage count and log2 p0); *best_q = depth * 1000 + tile width.
ffa_status tune_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data, int64_t m_rows,
                     int stages, int64_t ld, void* d_plane, void* d_tmp, cudaStream_t st, int* best_q);
// Algorithm 1 on `count` trials starting at trial0.  fused: d_prof is the
// plane after all but the last FFA stage (m_rows rows); the kernel applies the
// last stage while loading.  Otherwise d_prof holds ready profiles.  Rows
// (profiles) are `ld` elements apart.
ffa_status launch_score2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                         int64_t trial0, int64_t p0, int64_t ld, int64_t m_rows, const ScoreWidths& wd,
                         ffa_record* d_rec, int32_t* d_status, cudaStream_t st);
// The fused scorers over a group of n base periods sharing m_rows and the
// widths: planes at element offsets off[i] of d_plane (rows
// plane_pitch(p0[i]) apart), the m_rows records of entry i at recs[i] (host
// array of device pointers; entries may belong to different series).
ffa_status launch_score2_group(const void* d_plane, int32_t precision, int n, const int64_t* p0, const int64_t* off,
                               int64_t m_rows, const ScoreWidths& wd, ffa_record* const* recs, int32_t* d_status,
                               cudaStream_t st);
ffa_status launch_score_alg2_group(const void* d_plane, int32_t precision, int n, const int64_t* p0,
                                   const int64_t* off, int64_t m_rows, const ScoreWidths& wd, float excl_frac,
                                   ffa_record* const* recs, cudaStream_t st);
// Algorithm 2 (Section 2.2.2) with the same fused/unfused inputs.
ffa_status launch_score_alg2(const void* d_prof, int32_t precision, bool fused, int64_t count,
                             int64_t trial0, int64_t p0, int64_t ld, int64_t m_rows, const ScoreWidths& wd,
                             float excl_frac, ffa_record* d_rec, cudaStream_t st);

// The scorer's CTA shape (0..3) for profiles of p0 bins and widths up to wmax.
int score_shape(int64_t p0, int wmax);

// ffa2best on a plan's records (defined in best.cu); workspace bytes it needs.
size_t best_workspace_bytes(int64_t n_entries, int64_t n_trials);

constexpr int STATS_DOUBLES = 2 + 1024;  // {mean, std} + reduction partials

}  // namespace ffa
