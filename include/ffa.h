/*
 * ffa.h -- C ABI of the GB300-native Fast Folding Algorithm period search.
 *
 * The method is the FFA search of Cameron et al. 2017 (MNRAS, "An
 * investigation of pulsar searching techniques with the Fast Folding
 * Algorithm"): a dedispersed time series is optionally pre-downsampled,
 * dereddened with a running median, normalised, folded at every base period
 * P0 by the Staelin FFA (Section 2.1, Eq. 1-2) over octaves of period with
 * downsampling by two per octave (Section 2.3), and every folded profile is
 * scored by Algorithm 1, the MAD-normalised power-of-two boxcar matched
 * filter (Section 2.2.1, Eq. 3-4).
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are device pointers on the current CUDA device;
 *     pointers without the prefix are host pointers.  The caller owns all
 *     memory; the library allocates nothing on the device or the host heap
 *     outside ffa_plan_create (which allocates the opaque plan on the host).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     Device work is enqueued asynchronously on it; inputs must stay valid
 *     and unmodified until that work completes.
 *   - Every call returns an ffa_status and never aborts, prints or exits.
 *     On failure ffa_last_error() returns a message for the calling thread.
 *     Argument errors are detected on the host before any launch.  Checks
 *     that only the device can make (e.g. an internal selection invariant)
 *     set the int32 word *d_status to a non-zero ffa_status; read it after
 *     the stream completes (ffa_wait does this with a bounded wait).
 *   - Layouts are row-major and densely packed (no row pitch).
 *   - Plans are immutable after creation; one plan may be used concurrently
 *     from several host threads on different streams and workspaces.
 */
#ifndef FFA_GB300_H
#define FFA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FFA_OK = 0,
    FFA_ERR_ARG = 1,         /* invalid argument (host check)                      */
    FFA_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed               */
    FFA_ERR_OOM = 3,         /* caller-provided buffer too small                   */
    FFA_ERR_TIMEOUT = 4,     /* a bounded wait expired                             */
    FFA_ERR_CANCELLED = 5,   /* reserved for the serving layer                     */
    FFA_ERR_UNSUPPORTED = 6, /* valid request outside the implemented envelope     */
    FFA_ERR_DEVICE = 7       /* a device-side invariant check failed               */
} ffa_status;

/* Input sample type: 32-bit float (PRESTO-style) or 8-bit unsigned
 * (SIGPROC-style) series, the two formats ffancy reads (Section 2.3). */
typedef enum { FFA_IN_F32 = 0, FFA_IN_U8 = 1, FFA_IN_F64 = 2 } ffa_input_type;

/* Fold precision: FP32 adds of the FP32-rounded normalised series, or exact
 * int32 adds of an int8 code q = clip(rint(16 z), -127, 127). */
typedef enum { FFA_FOLD_F32 = 0, FFA_FOLD_I8 = 1 } ffa_fold_precision;

/* Search configuration (ffancy's interface, Section 2.3; periods in seconds). */
typedef struct {
    double tsamp_s;          /* sampling interval of the input series            */
    double period_min_s;     /* search range [period_min_s, period_max_s)        */
    double period_max_s;
    double duty_max;         /* widths 1,2,4,.. up to the first > duty_max * P0
                                (Section 2.2.1 uses 0.2); ignored if fixed widths */
    int32_t downsample0;     /* pre-downsampling factor D0 >= 1                  */
    int32_t detrend_window;  /* running-median window in samples; 0 = the paper's
                                default min(2 Pmax, 4 Pmin); < 0 = no dereddening;
                                made odd by W |= 1                                */
    int32_t min_rows;        /* skip P0 with fewer data rows (0 -> 2)            */
    int32_t in_type;         /* ffa_input_type                                   */
    int32_t precision;       /* ffa_fold_precision                               */
    int32_t n_widths_fixed;  /* > 0: use widths_fixed[0..n) instead of duty_max  */
    int32_t widths_fixed[16];
    int32_t scorer;          /* ffa_scorer: Algorithm 1 (default) or 2           */
    float alg2_window;       /* Algorithm 2 exclusion window as a fraction of the
                                profile (0 = the paper's 20 %)                     */
    float clip_sigma;        /* > 0: cap the normalised series at +-clip_sigma
                                (Section 5's clipping; the int8 code is taken from
                                the capped value); 0 = off                        */
    float persist_cutoff;    /* persistence: a sample scores 1 when its normalised
                                (uncapped) value exceeds this cutoff (Section 5)  */
    int32_t persistence;     /* nonzero: the plan supports ffa_search_persistence */
} ffa_search_config;

/* Profile scorer (Section 2.2): Algorithm 1, MAD-normalised boxcars; or
 * Algorithm 2, boxcar then S/N against the off-pulse mean and standard
 * deviation outside a window around the maximum (Eq. 5).  Algorithm 2's
 * fixed-width "Ref" form is a single fixed width. */
typedef enum { FFA_SCORE_ALG1 = 0, FFA_SCORE_ALG2 = 1 } ffa_scorer;

/* One periodogram record per trial period (16 bytes).  flags bit 0: the
 * profile's MAD was zero (S/N reported as 0). */
typedef struct {
    float snr;      /* Algorithm 1 score: max over widths and phases             */
    int32_t width;  /* boxcar width (bins) of the best score                     */
    int32_t phase;  /* first bin of the best boxcar window                        */
    uint32_t flags;
} ffa_record;

/* One base period of the plan.  Trial k of this entry (0 <= k < m_rows) is
 * periodogram record first_trial + k and has period
 * (p0 + k / (m_rows - 1)) * tsamp * D0 * 2^octave  (Eq. 2 with N = M * P0). */
typedef struct {
    int32_t octave;
    int32_t p0;          /* bins per folded profile                             */
    int32_t m_data;      /* floor(n_octave / p0) data rows                      */
    int32_t m_rows;      /* next power of two >= m_data; rows beyond are zero   */
    int32_t n_widths;
    int32_t widths[16];
    int32_t pad;
    int64_t n_octave;    /* samples of this octave's series                     */
    int64_t first_trial;
} ffa_plan_entry;

/* A candidate returned by ffa_candidates. */
typedef struct {
    int64_t trial;      /* periodogram index                                     */
    double period_s;
    float snr;
    int32_t octave, p0, k, width, phase;
} ffa_candidate;

typedef struct ffa_plan ffa_plan;

/* ---- plan ---------------------------------------------------------------- */

/* Build the search plan for a series of n input samples (host only, no
 * device work): octaves, base periods, row counts, widths and the workspace
 * size.  Errors: FFA_ERR_ARG for a non-positive tsamp/period range/D0, an
 * empty plan is allowed (zero trials). */
ffa_status ffa_plan_create(const ffa_search_config* cfg, int64_t n, ffa_plan** out);
void ffa_plan_destroy(ffa_plan* plan);

/* Sizes of a plan: base periods, periodogram length, octaves, the odd
 * running-median window and the bytes of device workspace ffa_search needs. */
ffa_status ffa_plan_info(const ffa_plan* plan, int64_t* n_periods, int64_t* n_trials,
                         int32_t* n_octaves, int32_t* window, size_t* workspace_bytes);

/* Copy the first `cap` plan entries (periodogram order) to host memory. */
ffa_status ffa_plan_entries(const ffa_plan* plan, ffa_plan_entry* out, int64_t cap);

/* Trial periods in seconds of periodogram records [trial_begin,
 * trial_begin + count), written to host memory `out`: Eq. 2 with the padded
 * N = M * P0 (Section 2.1), i.e. trial k of a base period of P0 bins and M
 * rows at octave o has period (P0 + k / (M - 1)) * tsamp * D0 * 2^o (P0 for
 * M = 1).  Host only.  FFA_ERR_ARG for a range outside the periodogram. */
ffa_status ffa_plan_periods(const ffa_plan* plan, int64_t trial_begin, int64_t count, double* out);

/* ---- the search ------------------------------------------------------------ */

/* Run the whole search (Section 2.3 pipeline) on the n-sample device series
 * d_series (type cfg.in_type).  Writes n_trials records to d_records.
 * d_workspace: >= workspace_bytes of device memory, 256-byte aligned.
 * d_status: one int32 device word, zeroed by the caller; device-side checks
 * store an ffa_status there.  Asynchronous on `stream`. */
ffa_status ffa_search(const ffa_plan* plan, const void* d_series, void* d_workspace,
                      size_t workspace_bytes, ffa_record* d_records, int32_t* d_status,
                      void* stream);

/* The same pipeline restricted to plan entries [entry_begin, entry_end)
 * (base periods in periodogram order): octaves holding them are prepared,
 * only those base periods are folded and scored, only their records are
 * written.  Independent ranges may run on different devices or processes;
 * their candidate lists merge on the host (the only exchange). */
ffa_status ffa_search_entries(const ffa_plan* plan, const void* d_series, int64_t entry_begin,
                              int64_t entry_end, void* d_workspace, size_t workspace_bytes,
                              ffa_record* d_records, int32_t* d_status, void* stream);

/* Debug outputs of the search, the extra output streams ffancy offers beside
 * the periodogram (Section 2.3: the dereddened copy of the input series and
 * the full suite of folded profiles of an FFA execution).  Both run the
 * search's own preparation of the octave (D0 sums, downsampling chain,
 * dereddening, normalisation) on d_series in the workspace.
 *
 * ffa_search_series: octave `octave`'s series, n_octave samples of it, copied
 * to d_out: what = FFA_DUMP_RESID gives the dereddened series (double,
 * x - running median, before normalisation); FFA_DUMP_Z gives the fold input
 * (float z, or the int8 code for precision FFA_FOLD_I8).
 * ffa_search_plane: every folded profile of plan entry `entry`: all M trials,
 * all FFA stages applied (on the search's own padded-pitch planes), row k =
 * trial k, packed densely as M * P0 elements (float, or int32 for precision
 * FFA_FOLD_I8) into d_plane.
 * Asynchronous on `stream`; FFA_ERR_ARG for an octave or entry outside the
 * plan, FFA_ERR_OOM for a short workspace. */
#define FFA_DUMP_RESID 0
#define FFA_DUMP_Z 1
ffa_status ffa_search_series(const ffa_plan* plan, const void* d_series, int32_t octave, int32_t what,
                             void* d_workspace, size_t workspace_bytes, void* d_out, int32_t* d_status,
                             void* stream);
ffa_status ffa_search_plane(const ffa_plan* plan, const void* d_series, int64_t entry, void* d_workspace,
                            size_t workspace_bytes, void* d_plane, int32_t* d_status, void* stream);

/* ffa_search plus the persistence score of Section 5 for every trial:
 * d_persist[t] (uint32, n_trials of them) = the number of above-cutoff
 * samples (normalised value > cfg.persist_cutoff, 1/0 per sample) that the
 * FFA folds into trial t's best boxcar window (the width and phase of its
 * record): the 0/1 series is folded by the same FFA with integer adds.  A
 * pulsar spreads such samples over many rows, a single burst contributes at
 * most its own length.  Needs a plan made with cfg.persistence != 0
 * (FFA_ERR_ARG otherwise); costs one more integer fold per base period. */
ffa_status ffa_search_persistence(const ffa_plan* plan, const void* d_series, void* d_workspace,
                                  size_t workspace_bytes, ffa_record* d_records, uint32_t* d_persist,
                                  int32_t* d_status, void* stream);

/* Autotuner: for every fold shape of the plan (stage count, floor(log2 P0)),
 * time the FFA with at most 3, 4, 5 and 6 stages per HBM pass, each with
 * column tiles of 128 and 256, on its median base period, and keep the
 * fastest for every later search on this device (process-wide cache).  The
 * pass depth and the tile width never change a result: every split runs the
 * recursion's add tree.  Uses the workspace as scratch; blocks until the
 * timing launches on `stream` finish.  *n_tuned = shapes tuned. */
ffa_status ffa_autotune(const ffa_plan* plan, void* d_workspace, size_t workspace_bytes, void* stream,
                        int32_t* n_tuned);

/* A batch of series (e.g. dedispersion trials of uneven length) with one
 * configuration: plans[i] (all made from the same ffa_search_config, for
 * each series' own length; FFA_ERR_ARG otherwise) searches the device series
 * d_series[i] into d_records[i] (host arrays of `count` pointers).  The
 * batch runs octave by octave: every series' octave is prepared into its own
 * slice of the workspace, then base periods of all series are folded and
 * scored together -- those with the same rows, widths and scorer shape share
 * one set of fold launches and one persistent scorer launch, each reading its
 * own series and writing its own records -- so a batch of short series fills
 * the GPU and takes a fraction of the launches of one search per series.
 * Each record equals the one ffa_search gives for that series alone (same
 * kernels, add tree and scorer shape).  d_workspace: at least
 * ffa_batch_workspace_bytes of device memory, 256-byte aligned (it holds
 * every series' raw and normalised octave series: about 9 bytes per FP32
 * input sample, plus two plane buffers).  Plans with persistence are
 * FFA_ERR_UNSUPPORTED (search them one by one).  Asynchronous on `stream`. */
ffa_status ffa_batch_workspace_bytes(const ffa_plan* const* plans, int32_t count, size_t* bytes);
ffa_status ffa_search_batch(const ffa_plan* const* plans, const void* const* d_series, int32_t count,
                            void* d_workspace, size_t workspace_bytes, ffa_record* const* d_records,
                            int32_t* d_status, void* stream);

/* Candidate extraction (the first step of ffa2best, Section 2.3.3): records
 * with S/N >= snr_min, highest first (ties: lower periodogram index first),
 * at most top_k (<= 4096) of them, written to host memory `out`; *n_out
 * receives the count and *best the globally best record's index (-1 if the
 * periodogram is empty).  Uses the plan's workspace after the records;
 * enqueues device kernels on `stream`, then waits for it with a bounded
 * wait of timeout_ms (FFA_ERR_TIMEOUT on expiry) and copies the result. */
ffa_status ffa_candidates(const ffa_plan* plan, const ffa_record* d_records, double snr_min,
                          int32_t top_k, void* d_workspace, size_t workspace_bytes,
                          ffa_candidate* out, int32_t* n_out, int64_t* best,
                          int32_t* d_status, void* stream, int32_t timeout_ms);

/* ffa_candidates over the trials of plan entries [entry_begin, entry_end)
 * only (d_records is the full periodogram; other records are not read).
 * Trial indices in `out` and *best are periodogram indices. */
ffa_status ffa_candidates_entries(const ffa_plan* plan, int64_t entry_begin, int64_t entry_end,
                                  const ffa_record* d_records, double snr_min, int32_t top_k,
                                  void* d_workspace, size_t workspace_bytes, ffa_candidate* out,
                                  int32_t* n_out, int64_t* best, int32_t* d_status, void* stream,
                                  int32_t timeout_ms);

/* ---- ffa2best: candidate selection (Section 2.3.3) ------------------------ */

/* Thresholds of ffa2best.  Peak separation: walking the periodogram in trial
 * (= period) order, a record with S/N >= snr_min starts a candidate, whose
 * peak is its running maximum; the candidate ends at the first record with
 * S/N below both peak * (1 - drop_frac) and peak - drop_abs, which may start
 * the next one.  Grouping (group != 0): a candidate whose S/N times
 * (1 - group_margin) is at most S * sqrt(d / (d + T |p - q| / q^2)) -- the
 * expected S/N of a stronger kept candidate (S/N S, period q, duty
 * d = width / P0) folded at the wrong period p over the observation length
 * T = n * tsamp, zero once d + T |p - q| / q^2 >= 1 -- is dropped.
 * Harmonics (primes_max >= 2): a candidate of period p within harm_tol * v
 * of v = q * (n/x) or v = q / (n/x), for a stronger kept candidate's period
 * q, a prime x <= primes_max and 0 < n < x, is dropped. */
typedef struct {
    double snr_min;       /* baseline S/N                                   */
    double drop_frac;     /* in [0, 1]                                      */
    double drop_abs;      /* >= 0                                           */
    int32_t group;        /* nonzero: group by the smeared response         */
    int32_t primes_max;   /* 0 or 1: no harmonic matching; at most 97       */
    double harm_tol;      /* relative tolerance, in [0, 0.1]                */
    double group_margin;  /* in [0, 1); 0.16 is the paper's largest measured
                             departure of the algorithms from Eq. 7's law  */
} ffa2best_config;

/* ffa2best on the whole periodogram d_records (n_trials records of `plan`).
 * Peaks are found on the device (however many there are); the strongest 4096
 * of them (all, if fewer) are grouped and harmonic-matched strongest first
 * (ties: lower periodogram index), each candidate compared only with the
 * stronger ones kept, and the first min(cap, kept) kept candidates are
 * written to host `out` (cap in [0, 4096]), strongest first; *n_out receives
 * their count and *n_peaks the number of peaks found.  Uses the plan's
 * workspace; enqueues on `stream`, then waits with a bounded wait of
 * timeout_ms (FFA_ERR_TIMEOUT) and copies the result. */
ffa_status ffa2best(const ffa_plan* plan, const ffa_record* d_records, const ffa2best_config* cfg,
                    void* d_workspace, size_t workspace_bytes, ffa_candidate* out, int32_t cap,
                    int32_t* n_out, int64_t* n_peaks, int32_t* d_status, void* stream,
                    int32_t timeout_ms);

/* ---- periodogram statistics (Section 4.3, false-alarm analysis) ----------- */

/* Add the S/N histogram of n device records to d_counts (n_bins + 2 uint64
 * counters, caller-zeroed before the first call, accumulated across calls):
 * d_counts[0] counts S/N < edges[0], d_counts[1 + b] counts
 * edges[b] <= S/N < edges[b + 1], d_counts[n_bins + 1] counts
 * S/N >= edges[n_bins].  edges: host array of n_bins + 1 strictly
 * increasing floats, 1 <= n_bins <= 4096 (FFA_ERR_ARG otherwise).
 * Asynchronous on `stream`. */
ffa_status ffa_snr_histogram(const ffa_record* d_records, int64_t n, const float* edges,
                             int32_t n_bins, uint64_t* d_counts, void* stream);

/* Gaussian-equivalent sigma of a histogram from ffa_snr_histogram (host
 * counts): sigma[b] = the z with Q(z) = p_b, Q the upper-tail normal
 * probability and p_b the fraction of counted trials with S/N >= edges[b],
 * for b = 0..n_bins (+inf where p_b = 0).  Host only.  FFA_ERR_ARG for an
 * empty histogram. */
ffa_status ffa_sigma_gauss(const uint64_t* counts, int32_t n_bins, double* sigma);

/* Wait for `stream` with a bounded wait (polling), then read *d_status.
 * Returns FFA_ERR_TIMEOUT, FFA_ERR_CUDA, the device status, or FFA_OK. */
ffa_status ffa_wait(void* stream, const int32_t* d_status, int32_t timeout_ms);

/* ---- serving: a request loop with continuous batching --------------------- */

/* A server runs searches submitted from the host as they arrive.  The caller
 * hands it one block of device memory, the HBM admission budget; each
 * request needs ffa_server_request_bytes of it (its series, its periodogram
 * and its search workspace: octave series and fold planes stay on the device
 * while it runs).  n_slots worker threads, each with its own non-blocking
 * stream, admit queued requests first-fit in arrival order as slots and
 * arena memory free up, so requests that arrive while others run overlap on
 * the device (a request passed over 8 times blocks admission until it fits).
 * Results are deterministic: a request's records and candidates are the
 * same alone and in any mix. */
typedef struct ffa_server ffa_server;

typedef struct {
    void* d_arena;        /* caller-owned device memory, 256-byte aligned        */
    size_t arena_bytes;   /* the admission budget                                */
    int32_t n_slots;      /* searches in flight at once, 1..32                    */
    int32_t timeout_ms;   /* bounded wait per search (<= 0: 600 s)                */
} ffa_server_config;

/* Arena bytes one request of n samples with configuration cfg needs. */
ffa_status ffa_server_request_bytes(const ffa_search_config* cfg, int64_t n, size_t* bytes);

/* Start the worker threads (they use the calling thread's current device). */
ffa_status ffa_server_create(const ffa_server_config* cfg, ffa_server** out);

/* Queue a search of the n-sample host series (pinned memory lets its copy
 * overlap other requests' work; it must stay valid until the request
 * completes).  On completion the server keeps the top_k (<= 4096) candidates
 * with S/N >= snr_min, the best trial, and, if host_records is non-null,
 * copies the whole periodogram there (n_trials records).  *ticket identifies
 * the request.  FFA_ERR_OOM if the request needs more than the whole arena. */
ffa_status ffa_server_submit(ffa_server* server, const ffa_search_config* cfg, const void* host_series,
                             int64_t n, double snr_min, int32_t top_k, ffa_record* host_records,
                             int64_t* ticket);

/* Wait up to timeout_ms (< 0: forever) for a request, copy up to cap of its
 * candidates to `out`, its best trial to *best, and times_ms[0..2] = queued,
 * running and total (latency) milliseconds; then forget the ticket.  Returns
 * the request's own status (FFA_ERR_TIMEOUT leaves the ticket valid). */
ffa_status ffa_server_wait(ffa_server* server, int64_t ticket, int32_t timeout_ms, ffa_candidate* out,
                           int32_t cap, int32_t* n_out, int64_t* best, double* times_ms);

/* Requests waiting, requests running, arena bytes in use. */
ffa_status ffa_server_stats(ffa_server* server, int64_t* queued, int64_t* in_flight, size_t* arena_used);

/* Finish every submitted request, stop the workers and free the server. */
void ffa_server_destroy(ffa_server* server);

/* ---- individual steps (for step-level parity checks) ----------------------- */

/* Pre-/octave downsampling (Section 2.3): d_out[i] = sum_{j<factor}
 * d_in[factor*i + j] in FP64 for i < n / factor (odd tail dropped). */
ffa_status ffa_downsample(const void* d_in, int32_t in_type, int64_t n, int64_t factor,
                          double* d_out, void* stream);

/* Dynamic dereddening (Section 2.3): d_resid[i] = d_raw[i] - median of the
 * centred window of `window` (odd) samples truncated at the series ends;
 * an even count takes the mean of its two middle values.  Exact. */
ffa_status ffa_detrend(const double* d_raw, int64_t n, int32_t window, double* d_resid,
                       int32_t* d_status, void* stream);

/* Normalisation: z = (r - mean) / std with the FP64 mean and population
 * standard deviation of d_resid; writes float z (precision F32) or the int8
 * code (precision I8) to d_out, and {mean, std} to d_stats[0..1].  d_stats
 * must hold FFA_STATS_DOUBLES doubles (the rest is reduction scratch). */
#define FFA_STATS_DOUBLES 1026
ffa_status ffa_normalise(const double* d_resid, int64_t n, int32_t precision, void* d_out,
                         double* d_stats, void* stream);

/* The FFA of one base period (Section 2.1): d_z holds >= m_data * p0 samples
 * (float for F32, int8 for I8); rows r >= m_data are zero; m_rows is a power
 * of two >= m_data.  Writes the m_rows folded trials (float or int32) to
 * d_plane (m_rows * p0 elements).  d_tmp: same size, scratch. */
ffa_status ffa_fold(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                    int64_t m_rows, void* d_plane, void* d_tmp, void* stream);

/* Variant of ffa_fold that allocates nothing and takes no scratch argument.
 * The paper has no counterpart: it serves callers that cannot allocate device
 * memory at the point of the call -- for example a real-time pipeline that
 * forbids allocator calls inside its processing loop, or a plug-in that is
 * handed device buffers for its input and output but no allocator.  The
 * scratch plane lives in a fixed file-scope device array of
 * FFA_NOALLOC_FOLD_MAX_ELEMS 32-bit elements (32 MiB) that every GPU loading
 * the library holds until the process exits.  Requires m_rows * p0 <=
 * FFA_NOALLOC_FOLD_MAX_ELEMS, else FFA_ERR_UNSUPPORTED with a message.
 * The first call on a device looks up the array's device address (a
 * cudaGetSymbolAddress, once per device, with that device current); make that
 * first call before any stream capture.  A cudaDeviceReset or any other
 * re-creation of the device's context reloads the array: the next call sees
 * the new context's id and looks the address up again (that call is again a
 * first call).  No cudaMalloc, cudaFree or other allocating routine is
 * called.  All calls share the array and it keeps the last call's contents;
 * nothing in it needs to start at zero because every element read has first
 * been written by the same call.  Calls from streams or host threads of one
 * process that overlap on the GPU race on the array: serialise them.  (Each
 * process has its own copy.)  Results equal ffa_fold's bit for bit.
 * m_rows * p0 is checked without overflow. */
#define FFA_NOALLOC_FOLD_MAX_ELEMS (8 * 1024 * 1024)
ffa_status ffa_fold_noalloc(const void* d_z, int32_t precision, int64_t p0, int64_t m_data,
                            int64_t m_rows, void* d_plane, void* stream);

/* Algorithm 1 (Section 2.2.1) on `count` profiles of p0 bins (float or
 * int32 per precision), widths given on the host; one record per profile. */
ffa_status ffa_score(const void* d_profiles, int32_t precision, int64_t count, int64_t p0,
                     const int32_t* widths, int32_t n_widths, ffa_record* d_records,
                     int32_t* d_status, void* stream);

/* ---- timing (benchmark instrumentation) ---------------------------------------- */

/* When enabled (process-wide), ffa_search records CUDA events on its stream
 * around phases of every octave: 0 = series preparation (downsampling,
 * dereddening, normalisation), 1 = fold + score of all base periods, and,
 * for every 64th base period of the octave (entries first + 64 j), 2 = its
 * fold launches and 3 = its scoring launch; base periods folded and scored
 * in groups (short planes) are timed per group instead, 4 = the group's fold
 * launches and 5 = its scoring launch, for every group holding one of those
 * base periods.  ffa_timing_read waits for the recorded events, writes the
 * summed milliseconds of phase p, octave o to ms[p * 64 + o] and the number
 * of recorded intervals to counts[p * 64 + o] for every p * 64 + o < cap
 * (cap >= 256; 384 covers all six phases), then clears the record.  Off by
 * default. */
ffa_status ffa_timing_enable(int32_t on);

/* Number of kernel launches (and device copies) the library has enqueued in
 * this process so far, all devices and threads together. */
int64_t ffa_launch_count(void);
ffa_status ffa_timing_read(double* ms, int32_t* counts, int32_t cap);

/* Algorithm 2 (Section 2.2.2, Eq. 5) on `count` profiles of p0 bins: per
 * width w the boxcar maximum I_max (first position j*), then I_av and the
 * population standard deviation of the filtered bins farther than
 * floor(excl_frac * p0 / 2) bins (cyclically) from j*, A = (I_max - I_av) /
 * sigma; the record keeps the best width (ties: smaller), its j* and A. */
ffa_status ffa_score_alg2(const void* d_profiles, int32_t precision, int64_t count, int64_t p0,
                          const int32_t* widths, int32_t n_widths, float excl_frac,
                          ffa_record* d_records, void* stream);

/* ---- errors ------------------------------------------------------------------ */
const char* ffa_status_string(ffa_status s);
const char* ffa_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FFA_GB300_H */
