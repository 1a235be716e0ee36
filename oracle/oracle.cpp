// Plain CPU oracle for the Fast Folding Algorithm period search of
// Cameron et al. 2017, "An investigation of pulsar searching techniques with
// the Fast Folding Algorithm".
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the package's smoke check and the CPU
// baseline leg of the benchmark do.  It shares no code, header, table or
// constant with the CUDA library.
//
// Everything is written to be checked by eye against the paper:
//   * downsampling, pre-downsampling and the dynamic running-median
//     dereddening of Section 2.3 (ffancy);
//   * the FFA recursion of Section 2.1 (Eq. 1-2 and the padding rule that
//     follows them), literally, as a recursive head/tail split;
//   * Algorithm 1 of Section 2.2.1 (Eq. 3-4): median / MAD normalisation and
//     power-of-two boxcar matched filters divided by sqrt(width).
// Floating point is FP64 unless stated; the fold is also instantiated for
// float (the GPU's FP32 adds, same add tree) and int64 (the int8 path).
// Compile with -ffp-contract=off so that no multiply-add is fused.
//
// Readings of points the paper leaves open (each restated where it is used):
//   R1 shift convention: output trial k of a 2^s-row group is
//      head[k>>1] + tail[k>>1] rolled left by ceil(k/2) bins;
//   R2 M_data = floor(N/P0) data rows, zero rows up to the next power of two;
//   R3 trial k <-> period P0 + k/(M-1) samples (Eq. 2 with the padded N);
//   R4 boxcars are cyclic over the profile, phase = first bin of the window;
//   R5 widths 1,2,4,... up to and including the first width > duty*P0;
//   R6 median of an even count = mean of the two middle values; MAD = 0 gives
//      S/N = 0 and a flag;
//   R7 K = 1.4826 as printed after Eq. 4;
//   R8 S/N_w = (max box sum - w*median) / (K * MAD * sqrt(w));
//   R9 downsampling sums adjacent samples, dropping an odd tail;
//   R10 each octave dereddens the downsampled raw series with a window that
//      is fixed in current samples (so it doubles in initial samples);
//   R11 the dereddened series is normalised by its FP64 mean and population
//      standard deviation;
//   R12 int8 path: q = clip(rint(16 z), -127, 127), round half to even;
//   R13 ties: within a trial max S/N, then smallest width, then smallest
//      phase; across trials the first in (octave, P0, trial) order;
//   R14 a base period with fewer than min_rows data rows is skipped;
//   R15 Algorithm 2 filters first: b_w[j] = sum_{i<w} x[(j+i) mod p0], not
//      normalised; I_max = its maximum (first position j* on ties);
//   R16 the Algorithm 2 exclusion window ("20 % of the profile width",
//      centred on the position of I_max) is the 2h+1 profile bins within
//      cyclic distance h = floor(excl_frac * p0 / 2) of the box's centre
//      c = (j* + floor(w/2)) mod p0; I_av and sigma are the FP64 mean and
//      population standard deviation (two-pass) of the other, unfiltered,
//      profile bins ("the average value and standard deviation of the
//      profile ... based on the remaining 80 %");
//   R17 the matched filter keeps unit noise by dividing by sqrt(w), as in
//      Algorithm 1, so with the off-pulse level scaled the same way
//      A_w = (I_max - w I_av) / (sigma sqrt(w)); score = max over widths with
//      the R13 tie-breaks; sigma = 0 or fewer than 2 off-window bins gives
//      score 0 and flag bit 0.  (Reading the statistics off the filtered
//      bins instead puts white noise's 5 sigma_gauss at S/N 12.2, against
//      the 7.1 printed in Section 4.3; this reading gives about 7.)
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <set>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------------------
// Section 2.3: downsampling (R9).  y[i] = sum_{j<f} x[f*i + j].
// ---------------------------------------------------------------------------
template <class T>
void downsample(const T* x, int64_t n, int64_t f, double* y) {
    int64_t m = n / f;
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < f; ++j) s += (double)x[f * i + j];
        y[i] = s;
    }
}

// Median of a list of values (R6): the middle value, or the mean of the two
// middle values for an even count.  Uses std::nth_element as the selection
// primitive.
double median_of(std::vector<double> v) {
    size_t n = v.size();
    size_t hi = n / 2;
    std::nth_element(v.begin(), v.begin() + hi, v.end());
    double b = v[hi];
    if (n % 2 == 1) return b;
    double a = *std::max_element(v.begin(), v.begin() + hi);
    return (a + b) / 2;
}

// The window of the centred running median at sample i (Section 2.3): width
// w (odd), truncated at both ends of the series.
inline void window_of(int64_t i, int64_t n, int64_t w, int64_t* s, int64_t* e) {
    int64_t h = w / 2;
    *s = std::max<int64_t>(0, i - h);
    *e = std::min<int64_t>(n - 1, i + h);
}

// ---------------------------------------------------------------------------
// Section 2.1: the FFA recursion (R1).  `src` holds m power-of-two rows of p0
// bins; `dst` receives the m folded trials.  `tmp` is scratch of the same
// size.  The two halves are folded independently, then trial k of the whole
// set is head[k>>1] plus tail[k>>1] read ceil(k/2) bins further on (cyclic).
// ---------------------------------------------------------------------------
template <class T>
void fold_rec(const T* src, int64_t m, int64_t p0, T* dst, T* tmp) {
    if (m == 1) {
        std::memcpy(dst, src, sizeof(T) * p0);
        return;
    }
    int64_t h = m / 2;
    // the halves are folded into tmp, using dst as their scratch
    fold_rec(src, h, p0, tmp, dst);
    fold_rec(src + h * p0, h, p0, tmp + h * p0, dst + h * p0);
    const T* head = tmp;
    const T* tail = tmp + h * p0;
    for (int64_t k = 0; k < m; ++k) {
        int64_t i = k >> 1;
        int64_t shift = (k + 1) >> 1;  // ceil(k/2)
        for (int64_t j = 0; j < p0; ++j)
            dst[k * p0 + j] = head[i * p0 + j] + tail[i * p0 + (j + shift) % p0];
    }
}

// One output trial of the same recursion, evaluated alone: the recursion is
// followed down both halves for trial k>>1 only.  Same add tree as fold_rec.
template <class T>
void fold_one(const T* src, int64_t m, int64_t p0, int64_t k, T* out) {
    if (m == 1) {
        std::memcpy(out, src, sizeof(T) * p0);
        return;
    }
    int64_t h = m / 2;
    std::vector<T> head(p0), tail(p0);
    fold_one(src, h, p0, k >> 1, head.data());
    fold_one(src + h * p0, h, p0, k >> 1, tail.data());
    int64_t shift = (k + 1) >> 1;
    for (int64_t j = 0; j < p0; ++j) out[j] = head[j] + tail[(j + shift) % p0];
}

// Pack the first m_data*p0 samples as rows, zero rows up to m (R2).
template <class T>
std::vector<T> make_rows(const T* z, int64_t p0, int64_t m_data, int64_t m) {
    std::vector<T> rows((size_t)(m * p0), T(0));
    std::memcpy(rows.data(), z, sizeof(T) * (size_t)(m_data * p0));
    return rows;
}

const double K_MAD = 1.4826;  // R7

}  // namespace

extern "C" {

// Per-trial record of the oracle.
typedef struct {
    double snr;
    double median;
    double mad;
    int32_t width;
    int32_t phase;
    int32_t flags;  // bit 0: MAD == 0
    int32_t pad;
} oracle_score;

// Search configuration (periods in seconds, as in ffancy's interface).
typedef struct {
    double tsamp;
    double period_min;
    double period_max;
    double duty;             // R5 width rule (used when n_widths_fixed == 0)
    int32_t downsample0;     // D0 >= 1 (pre-downsampling, Section 2.3)
    int32_t detrend_window;  // 0: min(2 Pmax, 4 Pmin); < 0: no dereddening
    int32_t min_rows;        // R14
    int32_t fold_type;       // 0: FP64 fold of FP64 z; 1: FP32 fold of FP32 z; 2: int8 q, int64 fold
    int32_t n_widths_fixed;
    int32_t widths_fixed[16];
} oracle_cfg;

// One base period of the plan.
typedef struct {
    int32_t octave;
    int32_t p0;
    int32_t m_data;
    int32_t m_rows;
    int32_t n_widths;
    int32_t widths[16];
    int32_t pad;
    int64_t n_octave;     // samples in this octave's series
    int64_t first_trial;  // index of trial 0 in the periodogram
} oracle_plan_row;

// --- Section 2.3 downsampling -------------------------------------------
void oracle_downsample_f32(const float* x, int64_t n, int64_t f, double* y) { downsample(x, n, f, y); }
void oracle_downsample_u8(const uint8_t* x, int64_t n, int64_t f, double* y) { downsample(x, n, f, y); }
void oracle_downsample_f64(const double* x, int64_t n, int64_t f, double* y) { downsample(x, n, f, y); }

// --- Section 2.3 dereddening ----------------------------------------------
// Definition: the running median at the listed samples, each by selection
// over its own window.
void oracle_running_median_at(const double* x, int64_t n, int64_t w, const int64_t* idx,
                              int64_t n_idx, double* out) {
    for (int64_t t = 0; t < n_idx; ++t) {
        int64_t s, e;
        window_of(idx[t], n, w, &s, &e);
        out[t] = median_of(std::vector<double>(x + s, x + e + 1));
    }
}

// The same running median for every sample, by sliding two sorted halves
// (lower half `lo`, upper half `hi`) along the series.
void oracle_running_median(const double* x, int64_t n, int64_t w, double* out) {
    if (n <= 0) return;
    std::multiset<double> lo, hi;
    auto rebalance = [&]() {
        while (lo.size() > hi.size() + 1) {
            auto it = std::prev(lo.end());
            hi.insert(*it);
            lo.erase(it);
        }
        while (lo.size() < hi.size()) {
            auto it = hi.begin();
            lo.insert(*it);
            hi.erase(it);
        }
    };
    auto insert = [&](double v) {
        if (lo.empty() || v <= *std::prev(lo.end())) lo.insert(v);
        else hi.insert(v);
        rebalance();
    };
    auto erase = [&](double v) {
        if (v <= *std::prev(lo.end())) lo.erase(lo.find(v));
        else hi.erase(hi.find(v));
        rebalance();
    };
    int64_t s, e;
    window_of(0, n, w, &s, &e);
    for (int64_t j = s; j <= e; ++j) insert(x[j]);
    for (int64_t i = 0; i < n; ++i) {
        int64_t s2, e2;
        window_of(i, n, w, &s2, &e2);
        for (int64_t j = e + 1; j <= e2; ++j) insert(x[j]);
        for (int64_t j = s; j < s2; ++j) erase(x[j]);
        s = s2;
        e = e2;
        double b = *std::prev(lo.end());
        out[i] = (lo.size() > hi.size()) ? b : (b + *hi.begin()) / 2;
    }
}

// --- normalisation (R11) and int8 quantisation (R12) ----------------------
// z = (r - mean) / std with FP64 mean and population std.  Writes the FP64
// z, its FP32 rounding and/or the int8 code when the pointers are non-null.
// Returns 1 if the standard deviation is zero (then every output is 0).
int oracle_normalise(const double* r, int64_t n, double* z64, float* z32, int8_t* q,
                     double* mean_std) {
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) sum += r[i];
    double mean = n > 0 ? sum / (double)n : 0.0;
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = r[i] - mean;
        ss += d * d;
    }
    double sd = n > 0 ? std::sqrt(ss / (double)n) : 0.0;
    if (mean_std) {
        mean_std[0] = mean;
        mean_std[1] = sd;
    }
    for (int64_t i = 0; i < n; ++i) {
        double z = sd > 0.0 ? (r[i] - mean) / sd : 0.0;
        if (z64) z64[i] = z;
        if (z32) z32[i] = (float)z;
        if (q) {
            double v = std::nearbyint(16.0 * z);
            v = std::min(127.0, std::max(-127.0, v));
            q[i] = (int8_t)v;
        }
    }
    return sd > 0.0 ? 0 : 1;
}

// --- Section 2.1 FFA --------------------------------------------------------
// rows: m (power of two) rows of p0 bins, row-major; out: m trials.
void oracle_fold_f64(const double* rows, int64_t m, int64_t p0, double* out) {
    std::vector<double> tmp((size_t)(m * p0));
    fold_rec(rows, m, p0, out, tmp.data());
}
void oracle_fold_f32(const float* rows, int64_t m, int64_t p0, float* out) {
    std::vector<float> tmp((size_t)(m * p0));
    fold_rec(rows, m, p0, out, tmp.data());
}
void oracle_fold_i64(const int64_t* rows, int64_t m, int64_t p0, int64_t* out) {
    std::vector<int64_t> tmp((size_t)(m * p0));
    fold_rec(rows, m, p0, out, tmp.data());
}
// One trial k of the fold of the series z packed as m_data rows of p0 bins
// plus zero rows up to m (R2).
void oracle_trial_f64(const double* z, int64_t p0, int64_t m_data, int64_t m, int64_t k, double* out) {
    auto rows = make_rows(z, p0, m_data, m);
    fold_one(rows.data(), m, p0, k, out);
}
void oracle_trial_f32(const float* z, int64_t p0, int64_t m_data, int64_t m, int64_t k, float* out) {
    auto rows = make_rows(z, p0, m_data, m);
    fold_one(rows.data(), m, p0, k, out);
}
void oracle_trial_i64(const int64_t* z, int64_t p0, int64_t m_data, int64_t m, int64_t k, int64_t* out) {
    auto rows = make_rows(z, p0, m_data, m);
    fold_one(rows.data(), m, p0, k, out);
}

// --- Section 2.2.1 Algorithm 1 ---------------------------------------------
// Median and MAD normalisation (Eq. 3-4), then boxcars of the listed widths,
// each box sum divided by sqrt(width) (R4, R8); score = best over widths
// and phases with the R13 tie-breaks.  Box sums come from a cyclic prefix
// sum: sum_{i<w} x[(j+i) mod p0] = C[j+w] - C[j].
void oracle_score_alg1_f64(const double* x, int64_t p0, const int32_t* widths, int32_t nw,
                           oracle_score* out) {
    std::vector<double> v(x, x + p0);
    double med = median_of(v);
    for (int64_t i = 0; i < p0; ++i) v[i] = std::fabs(x[i] - med);
    double mad = median_of(v);
    out->median = med;
    out->mad = mad;
    out->flags = 0;
    out->pad = 0;
    if (!(mad > 0.0)) {
        out->snr = 0.0;
        out->width = widths[0];
        out->phase = 0;
        out->flags = 1;
        return;
    }
    int64_t wmax = 0;
    for (int32_t t = 0; t < nw; ++t) wmax = std::max<int64_t>(wmax, widths[t]);
    std::vector<double> c((size_t)(p0 + wmax + 1));
    c[0] = 0.0;
    for (int64_t t = 0; t < p0 + wmax; ++t) c[t + 1] = c[t] + x[t % p0];
    double best = -std::numeric_limits<double>::infinity();
    int32_t best_w = widths[0], best_j = 0;
    for (int32_t t = 0; t < nw; ++t) {
        int64_t w = widths[t];
        double bmax = -std::numeric_limits<double>::infinity();
        int64_t jmax = 0;
        for (int64_t j = 0; j < p0; ++j) {
            double b = c[j + w] - c[j];
            if (b > bmax) {
                bmax = b;
                jmax = j;
            }
        }
        double num = bmax - (double)w * med;
        double den = (K_MAD * mad) * std::sqrt((double)w);
        double snr = num / den;
        if (snr > best) {
            best = snr;
            best_w = (int32_t)w;
            best_j = (int32_t)jmax;
        }
    }
    out->snr = best;
    out->width = best_w;
    out->phase = best_j;
}

// The same scorer on an exact integer profile (int8 path): the median, MAD
// and box sums are exact; the S/N is evaluated with the same FP64 steps.
void oracle_score_alg1_i64(const int64_t* x, int64_t p0, const int32_t* widths, int32_t nw,
                           oracle_score* out) {
    std::vector<double> v(x, x + p0);
    double med = median_of(v);
    for (int64_t i = 0; i < p0; ++i) v[i] = std::fabs((double)x[i] - med);
    double mad = median_of(v);
    out->median = med;
    out->mad = mad;
    out->flags = 0;
    out->pad = 0;
    if (!(mad > 0.0)) {
        out->snr = 0.0;
        out->width = widths[0];
        out->phase = 0;
        out->flags = 1;
        return;
    }
    int64_t wmax = 0;
    for (int32_t t = 0; t < nw; ++t) wmax = std::max<int64_t>(wmax, widths[t]);
    std::vector<int64_t> c((size_t)(p0 + wmax + 1));
    c[0] = 0;
    for (int64_t t = 0; t < p0 + wmax; ++t) c[t + 1] = c[t] + x[t % p0];
    double best = -std::numeric_limits<double>::infinity();
    int32_t best_w = widths[0], best_j = 0;
    for (int32_t t = 0; t < nw; ++t) {
        int64_t w = widths[t];
        int64_t bmax = std::numeric_limits<int64_t>::min();
        int64_t jmax = 0;
        for (int64_t j = 0; j < p0; ++j) {
            int64_t b = c[j + w] - c[j];
            if (b > bmax) {
                bmax = b;
                jmax = j;
            }
        }
        double num = (double)bmax - (double)w * med;
        double den = (K_MAD * mad) * std::sqrt((double)w);
        double snr = num / den;
        if (snr > best) {
            best = snr;
            best_w = (int32_t)w;
            best_j = (int32_t)jmax;
        }
    }
    out->snr = best;
    out->width = best_w;
    out->phase = best_j;
}

// --- Section 2.2.2 Algorithm 2 ---------------------------------------------
// Boxcar filter first (R15), then per width the maximum I_max at j*, an
// exclusion window of about excl_frac of the profile centred on that box
// (R16), and the S/N of Eq. 5 against the mean and standard deviation of the
// remaining profile bins (R17).  median/mad of the record are set to I_av and
// sigma of the winning width.
void oracle_score_alg2_f64(const double* x, int64_t p0, const int32_t* widths, int32_t nw,
                           double excl_frac, oracle_score* out) {
    int64_t wmax = 0;
    for (int32_t t = 0; t < nw; ++t) wmax = std::max<int64_t>(wmax, widths[t]);
    std::vector<double> c((size_t)(p0 + wmax + 1));
    c[0] = 0.0;
    for (int64_t t = 0; t < p0 + wmax; ++t) c[t + 1] = c[t] + x[t % p0];
    const int64_t h = (int64_t)std::floor(excl_frac * (double)p0 / 2.0);
    const int64_t n_off = p0 - std::min<int64_t>(p0, 2 * h + 1);
    double best = -std::numeric_limits<double>::infinity();
    int32_t best_w = widths[0], best_j = 0;
    double best_av = 0.0, best_sd = 0.0;
    bool any = false;
    for (int32_t t = 0; t < nw; ++t) {
        const int64_t w = widths[t];
        int64_t jmax = 0;
        double bmax = c[w] - c[0];
        for (int64_t j = 1; j < p0; ++j) {
            const double b = c[j + w] - c[j];
            if (b > bmax) {
                bmax = b;
                jmax = j;
            }
        }
        if (n_off < 2) continue;
        const int64_t centre = (jmax + w / 2) % p0;
        auto off = [&](int64_t j) {
            int64_t d = ((j - centre) % p0 + p0) % p0;  // cyclic distance from the centre
            d = std::min(d, p0 - d);
            return d > h;
        };
        double sum = 0.0;
        for (int64_t j = 0; j < p0; ++j)
            if (off(j)) sum += x[j];
        const double av = sum / (double)n_off;
        double ss = 0.0;
        for (int64_t j = 0; j < p0; ++j)
            if (off(j)) ss += (x[j] - av) * (x[j] - av);
        const double sd = std::sqrt(ss / (double)n_off);
        if (!(sd > 0.0)) continue;
        const double a = (bmax - (double)w * av) / (sd * std::sqrt((double)w));
        any = true;
        if (a > best) {
            best = a;
            best_w = (int32_t)w;
            best_j = (int32_t)jmax;
            best_av = av;
            best_sd = sd;
        }
    }
    out->pad = 0;
    if (!any) {
        out->snr = 0.0;
        out->width = widths[0];
        out->phase = 0;
        out->flags = 1;
        out->median = 0.0;
        out->mad = 0.0;
        return;
    }
    out->snr = best;
    out->width = best_w;
    out->phase = best_j;
    out->flags = 0;
    out->median = best_av;
    out->mad = best_sd;
}

// --- Section 2.3 search plan -------------------------------------------------
// Period range in samples of the D0-downsampled series; octave o searches
// P0 in [Pmin, min(2 Pmin, ceil(Pmax / 2^o))) on the series downsampled 2^o
// times.  Returns the number of base periods; fills at most `cap` rows.
int64_t oracle_plan(const oracle_cfg* cfg, int64_t n, oracle_plan_row* rows, int64_t cap,
                    int64_t* n_trials, int32_t* window) {
    int64_t d0 = cfg->downsample0 >= 1 ? cfg->downsample0 : 1;
    double pmin = cfg->period_min / (cfg->tsamp * (double)d0);
    double pmax = cfg->period_max / (cfg->tsamp * (double)d0);
    int64_t p_min = (int64_t)std::ceil(pmin - 1e-9);
    int64_t p_max = (int64_t)std::ceil(pmax - 1e-9);
    if (p_min < 1) p_min = 1;
    int64_t w = cfg->detrend_window > 0 ? cfg->detrend_window : std::min(2 * p_max, 4 * p_min);
    if (cfg->detrend_window < 0) w = 1;
    w |= 1;
    if (window) *window = (int32_t)w;
    int64_t count = 0, trials = 0;
    int64_t n_o = n / d0;
    for (int32_t o = 0;; ++o) {
        if (o > 0) n_o /= 2;
        double hi_real = pmax / std::ldexp(1.0, o);
        int64_t hi = std::min<int64_t>(2 * p_min, (int64_t)std::ceil(hi_real - 1e-9));
        if (hi <= p_min || n_o <= 0) break;
        for (int64_t p0 = p_min; p0 < hi; ++p0) {
            int64_t m_data = n_o / p0;
            int64_t min_rows = cfg->min_rows > 0 ? cfg->min_rows : 2;
            if (m_data < min_rows) continue;
            int64_t m = 1;
            while (m < m_data) m *= 2;
            if (count < cap) {
                oracle_plan_row& r = rows[count];
                std::memset(&r, 0, sizeof(r));
                r.octave = o;
                r.p0 = (int32_t)p0;
                r.m_data = (int32_t)m_data;
                r.m_rows = (int32_t)m;
                r.n_octave = n_o;
                r.first_trial = trials;
                if (cfg->n_widths_fixed > 0) {
                    r.n_widths = cfg->n_widths_fixed;
                    for (int t = 0; t < cfg->n_widths_fixed; ++t) r.widths[t] = cfg->widths_fixed[t];
                } else {
                    int nw = 0;
                    for (int64_t wd = 1;; wd *= 2) {
                        r.widths[nw++] = (int32_t)wd;
                        if ((double)wd > cfg->duty * (double)p0 || nw == 16) break;
                    }
                    r.n_widths = nw;
                }
            }
            ++count;
            trials += m;
        }
    }
    if (n_trials) *n_trials = trials;
    return count;
}

// The dereddened, normalised series of every octave, concatenated, as the
// search folds it (fold_type 0: FP64 z, 1: FP32 z, 2: int8 q; only the
// matching output pointer is written).  `offsets[o]` receives the start of
// octave o.  Returns the number of octaves.
int oracle_octave_series(const oracle_cfg* cfg, const void* series, int64_t n, int in_type,
                         double* z64_out, float* z32_out, int8_t* q_out, int64_t* offsets,
                         int max_oct) {
    int64_t n_trials;
    int32_t w;
    int64_t np = oracle_plan(cfg, n, nullptr, 0, &n_trials, &w);
    (void)np;
    int64_t d0 = cfg->downsample0 >= 1 ? cfg->downsample0 : 1;
    int64_t n_o = n / d0;
    std::vector<double> raw((size_t)std::max<int64_t>(n_o, 1));
    if (in_type == 0) downsample((const float*)series, n, d0, raw.data());
    else downsample((const uint8_t*)series, n, d0, raw.data());
    double pmin = cfg->period_min / (cfg->tsamp * (double)d0);
    double pmax = cfg->period_max / (cfg->tsamp * (double)d0);
    int64_t p_min = std::max<int64_t>(1, (int64_t)std::ceil(pmin - 1e-9));
    int64_t pos = 0;
    int o = 0;
    for (;; ++o) {
        if (o > 0) {
            std::vector<double> nxt((size_t)std::max<int64_t>(n_o / 2, 1));
            downsample(raw.data(), n_o, 2, nxt.data());
            n_o /= 2;
            raw.swap(nxt);
        }
        int64_t hi = std::min<int64_t>(2 * p_min, (int64_t)std::ceil(pmax / std::ldexp(1.0, o) - 1e-9));
        if (hi <= p_min || n_o <= 0 || o >= max_oct) break;
        std::vector<double> r((size_t)n_o);
        if (w > 1) {
            std::vector<double> med((size_t)n_o);
            oracle_running_median(raw.data(), n_o, w, med.data());
            for (int64_t i = 0; i < n_o; ++i) r[i] = raw[i] - med[i];
        } else {
            r.assign(raw.begin(), raw.begin() + n_o);
        }
        offsets[o] = pos;
        oracle_normalise(r.data(), n_o, z64_out ? z64_out + pos : nullptr,
                         z32_out ? z32_out + pos : nullptr, q_out ? q_out + pos : nullptr,
                         nullptr);
        pos += n_o;
    }
    offsets[o] = pos;
    return o;
}

// Fold and score the listed base periods (the inner loop of the search):
// z holds every octave's series (offsets[o] = start of octave o) as FP64
// (fold_type 0), FP32 (1) or int8 (2); records receive each row's trials at
// row.first_trial.  Base periods run in parallel over `nthreads` threads.
void oracle_fold_score_rows(int fold_type, const void* z, const int64_t* offsets,
                            const oracle_plan_row* plan, int64_t np, oracle_score* records,
                            int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < np; ++t) {
        const oracle_plan_row& r = plan[t];
        int64_t p0 = r.p0, m = r.m_rows, md = r.m_data;
        int64_t off = offsets[r.octave];
        if (fold_type == 0) {
            auto rows = make_rows((const double*)z + off, p0, md, m);
            std::vector<double> out((size_t)(m * p0));
            oracle_fold_f64(rows.data(), m, p0, out.data());
            for (int64_t k = 0; k < m; ++k)
                oracle_score_alg1_f64(out.data() + k * p0, p0, r.widths, r.n_widths,
                                      &records[r.first_trial + k]);
        } else if (fold_type == 1) {
            auto rows = make_rows((const float*)z + off, p0, md, m);
            std::vector<float> out((size_t)(m * p0));
            oracle_fold_f32(rows.data(), m, p0, out.data());
            std::vector<double> prof((size_t)p0);
            for (int64_t k = 0; k < m; ++k) {
                for (int64_t j = 0; j < p0; ++j) prof[j] = out[k * p0 + j];
                oracle_score_alg1_f64(prof.data(), p0, r.widths, r.n_widths,
                                      &records[r.first_trial + k]);
            }
        } else {
            const int8_t* qz8 = (const int8_t*)z + off;
            std::vector<int64_t> qz((size_t)(md * p0));
            for (int64_t i = 0; i < md * p0; ++i) qz[i] = qz8[i];
            auto rows = make_rows(qz.data(), p0, md, m);
            std::vector<int64_t> out((size_t)(m * p0));
            oracle_fold_i64(rows.data(), m, p0, out.data());
            for (int64_t k = 0; k < m; ++k)
                oracle_score_alg1_i64(out.data() + k * p0, p0, r.widths, r.n_widths,
                                      &records[r.first_trial + k]);
        }
    }
}

// --- the whole search --------------------------------------------------------
// series: n samples (in_type 0: float32, 1: uint8).  records: one per trial,
// in (octave, P0, trial) order.  Base periods are folded in parallel over
// `nthreads` OpenMP threads (each base period is independent).
int oracle_search(const oracle_cfg* cfg, const void* series, int64_t n, int in_type,
                  oracle_score* records, int64_t cap, int nthreads) {
    int64_t n_trials;
    int32_t w;
    int64_t np = oracle_plan(cfg, n, nullptr, 0, &n_trials, &w);
    if (n_trials > cap) return -1;
    std::vector<oracle_plan_row> plan((size_t)np);
    oracle_plan(cfg, n, plan.data(), np, &n_trials, &w);
    int64_t d0 = cfg->downsample0 >= 1 ? cfg->downsample0 : 1;
    // total octave samples
    std::vector<int64_t> offsets(64);
    int64_t total = 0;
    {
        int64_t n_o = n / d0;
        for (int o = 0; o < 63; ++o) {
            total += n_o;
            n_o /= 2;
        }
    }
    std::vector<double> z64;
    std::vector<float> z32;
    std::vector<int8_t> q;
    if (cfg->fold_type == 0) z64.resize((size_t)total + 1);
    if (cfg->fold_type == 1) z32.resize((size_t)total + 1);
    if (cfg->fold_type == 2) q.resize((size_t)total + 1);
    oracle_octave_series(cfg, series, n, in_type, z64.empty() ? nullptr : z64.data(),
                         z32.empty() ? nullptr : z32.data(), q.empty() ? nullptr : q.data(),
                         offsets.data(), 63);
    const void* zs = cfg->fold_type == 0 ? (const void*)z64.data()
                   : cfg->fold_type == 1 ? (const void*)z32.data() : (const void*)q.data();
    oracle_fold_score_rows(cfg->fold_type, zs, offsets.data(), plan.data(), np, records, nthreads);
    return 0;
}

// Best record (R13): maximum S/N, the earliest in periodogram order on ties.
int64_t oracle_best(const oracle_score* records, int64_t n) {
    int64_t best = -1;
    for (int64_t i = 0; i < n; ++i)
        if (best < 0 || records[i].snr > records[best].snr) best = i;
    return best;
}

}  // extern "C"
