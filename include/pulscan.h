/*
 * pulscan.h -- C ABI of the GB300 boxcar (unmatched-filter) search.
 *
 * The library runs the data-parallel hot path of the Pulscan binary-pulsar
 * search (White et al., arXiv 2406.15186) on one NVIDIA GB300 (sm_103a):
 *
 *   real time series --R2C FFT--> complex spectrum            (§2.2.2)
 *   --per-block median/MAD normalisation, |X|^2 / 2--> power  (§2.2.3, Eq. 8)
 *   --boxcar sums of every width 1..z_max at every bin-->     (§2.2.5)
 *   --per-(segment, width) maximum and chi-square threshold--> (Algorithm 4, Eq. 9)
 *   candidates (series, width, start bin, power, sigma).
 *
 * Conventions used by every entry point:
 *  - Pointers prefixed d_ are DEVICE pointers owned by the caller; h_ are host
 *    pointers owned by the caller.  The plan owns its own scratch (threshold
 *    table, block statistics, per-(segment, width) slots, candidate buffer).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are
 *    asynchronous on that stream unless stated otherwise.
 *  - Every function returns PULSCAN_OK (0) or a negative PULSCAN_ERR_* code;
 *    pulscan_last_error() then returns a message for the calling thread.
 *  - Width w means a boxcar of w bins, w = 1..z_max (the paper's z + 1).
 *  - A series of n real samples has M = n/2 + 1 Fourier bins.  It is cut into
 *    n_seg = max(1, M / segment_len) segments of segment_len bins; the last
 *    segment absorbs the remainder.  The segment is both the normalisation
 *    block (§2.2.3) and the search chunk of Algorithm 4.
 *  - A window is valid only if it lies inside the spectrum: k + w <= M.
 *  - Noise power is Exp(1) after the 1/2 in P = (a^2 + b^2)/2, so a width-w
 *    sum S has 2S ~ chi^2(2w) (Eq. 9); p = Q(w, S), Bonferroni-corrected by
 *    n_trials (default M * z_max per series), sigma = Phi^{-1}(1 - p).
 */
#ifndef PULSCAN_H
#define PULSCAN_H

#include <stdint.h>

#if defined(__GNUC__)
#define PULSCAN_API __attribute__((visibility("default")))
#else
#define PULSCAN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pulscan_stream; /* same type as cudaStream_t */
typedef struct pulscan_plan_s *pulscan_plan;

#define PULSCAN_OK 0
#define PULSCAN_ERR_INVALID_ARG (-1) /* bad argument; nothing was launched      */
#define PULSCAN_ERR_CUDA (-2)        /* a CUDA/cuFFT call failed                */
#define PULSCAN_ERR_NOMEM (-3)       /* device or host allocation failed        */
#define PULSCAN_ERR_CAPACITY (-4)    /* output larger than the given capacity   */
#define PULSCAN_ERR_TIMEOUT (-5)     /* a bounded device wait gave up           */
#define PULSCAN_ERR_UNSUPPORTED (-6) /* valid request this build cannot serve   */

/* One candidate: the maximum boxcar power of one (series, harmonic stage,
 * segment, width) that passes the sigma threshold (Algorithm 4 keeps one per
 * chunk and width).  `bin` is the window's first bin k within its (stage)
 * spectrum (the centre is k + (width - 1)/2); `power` is S_w[k] in FP32;
 * `sigma` is the Bonferroni-corrected Gaussian-equivalent significance
 * (§2.2.3); `harmonics` is the number H of harmonics summed (§2.3; 1 without
 * harmonic summing).  32 bytes. */
typedef struct {
  uint32_t series;
  uint32_t width;
  uint64_t bin;
  float power;
  float sigma;
  uint32_t harmonics;
  uint32_t reserved;
} pulscan_cand;

/* Sizes of the caller-owned buffers of a plan.  All counts are elements. */
typedef struct {
  int64_t n_series;       /* series in the plan                                   */
  int64_t x_floats;       /* time-domain buffer: float[x_floats]                  */
  int64_t spec_floats;    /* spectrum buffer: interleaved (re, im) float pairs    */
  int64_t power_floats;   /* power buffer: float[power_floats]                    */
  int64_t total_segments; /* segments over all series (rows of maxima / stats)    */
  int32_t z_max;
  int32_t segment_len;
  double threshold_sigma;
  int64_t max_candidates; /* capacity of the plan's device candidate buffer       */
} pulscan_plan_info;

/* Create a plan for one series of n real samples.
 * Validation (PULSCAN_ERR_INVALID_ARG, nothing allocated): n >= 2 and even;
 * z_max >= 1; z_max <= segment_len <= M = n/2 + 1 (a window's halo then comes
 * from at most one neighbouring segment); threshold_sigma finite and >= 0.
 * n < 2^33, else PULSCAN_ERR_UNSUPPORTED (start bins are 32-bit in the
 * per-(segment, width) merge keys).
 * The Bonferroni trial count is M * z_max (reading of §2.2.3: every bin times
 * every searched width).  Allocates device scratch on the current device. */
PULSCAN_API int pulscan_plan_create(pulscan_plan *out, int64_t n, int32_t z_max, int32_t segment_len,
                        double threshold_sigma);

/* Create a plan for a batch of series of uneven lengths (DM trials / beams),
 * searched by the same kernels in one pass.  lengths[i] follows the rules of
 * pulscan_plan_create for every i; each series gets its own trial count
 * M_i * z_max.  The buffers hold the series at the offsets returned by
 * pulscan_plan_offsets (series are grouped by length so that each length
 * class is one batched FFT). */
PULSCAN_API int pulscan_plan_create_batch(pulscan_plan *out, const int64_t *h_lengths, int32_t n_series,
                              int32_t z_max, int32_t segment_len, double threshold_sigma);

/* As pulscan_plan_create_batch, plus harmonic summing (§2.3, the GPU
 * decimation listing): for H = 2..numharm the normalised power of every
 * series is decimated by summing adjacent non-overlapping groups of h bins,
 * h = 1..H, aligned at bin 0 and added,
 *   X_H[r] = sum_{h=1}^{H} sum_{j=0}^{h-1} P[h r + j],  r < floor(M / H),
 * which is chi^2 with H(H+1) degrees of freedom per bin for noise; each X_H
 * is searched like the power itself (same widths, segment length and sigma
 * threshold) with a width-w sum distributed as chi^2 with H(H+1) w degrees of
 * freedom, and its own Bonferroni count floor(M / H) x (searched widths).
 * The stage spectra sit in the power buffer after the series' powers
 * (power_floats covers them); the segments of all stages are counted in
 * total_segments (stages after the series, in the same series order);
 * candidates carry H in `harmonics`.  numharm = 1 is pulscan_plan_create_batch.
 * Extra validation (INVALID_ARG): 1 <= numharm <= 8 and
 * segment_len <= floor(M / numharm) for every series.  The logsumexp entry
 * points return PULSCAN_ERR_UNSUPPORTED on such a plan. */
PULSCAN_API int pulscan_plan_create_harmonic(pulscan_plan *out, const int64_t *h_lengths, int32_t n_series,
                                             int32_t z_max, int32_t segment_len, double threshold_sigma,
                                             int32_t numharm);

/* Destroy a plan and free its scratch (after the plan's last stream work). */
PULSCAN_API void pulscan_plan_destroy(pulscan_plan plan);

/* Buffer sizes (see pulscan_plan_info). */
PULSCAN_API int pulscan_plan_get_info(pulscan_plan plan, pulscan_plan_info *h_info);

/* Per-series offsets, each a host array of n_series + 1 int64 written by the
 * call (NULL to skip): h_x_off in floats of the time buffer, h_spec_off in
 * complex bins of the spectrum buffer (float pairs), h_power_off in floats of
 * the power buffer, h_seg_off in segments.  Entry i+1 - entry i is series
 * i's extent (spectrum/power extents include alignment padding). */
PULSCAN_API int pulscan_plan_offsets(pulscan_plan plan, int64_t *h_x_off, int64_t *h_spec_off,
                         int64_t *h_power_off, int64_t *h_seg_off);

/* Where harmonic stage H (1..numharm; 1 = the series' own power) of every
 * series lives: h_power_off[i] (floats of the power buffer), h_seg_off[i]
 * (first global segment) and h_bins[i] (floor(M_i / H) bins) for series i in
 * the caller's order, each a host array of n_series + 1 entries or NULL;
 * entry n_series is the end of the stage (0 for h_bins).  Errors: INVALID_ARG. */
PULSCAN_API int pulscan_plan_stage_offsets(pulscan_plan plan, int32_t harmonics, int64_t *h_power_off,
                                           int64_t *h_seg_off, int64_t *h_bins);

/* Override the Bonferroni trial count of every series (n_trials >= 1; 1 turns
 * the correction off) and recompute the threshold table. Host-synchronous.
 * The count then stays fixed when the searched widths change. */
PULSCAN_API int pulscan_plan_set_trials(pulscan_plan plan, double n_trials);

/* Which widths are searched for candidates (the user-selected step of §2.2.3
 * and Algorithm 4's "z mod z_step = 0" test; the logarithmic z sampling of
 * §4.1.4 that the GPU version searches).  Every width 1..z_max is still
 * summed -- the recursion of §2.2.5 needs them all -- but only searched
 * widths are compared with a threshold and reported; the others get
 * T_w = +inf.  With z = w - 1:
 *   PULSCAN_WIDTHS_ALL  (0): every width (the default);
 *   PULSCAN_WIDTHS_STEP (1): widths with z mod step == 0, i.e. w = 1, 1 + step, ...;
 *   PULSCAN_WIDTHS_LOG2 (2): widths with z a power of two, i.e. w = 2, 3, 5, 9, ...
 * Unless pulscan_plan_set_trials fixed it, the Bonferroni count becomes
 * M x (number of searched widths) per series.  Host-synchronous.
 * Errors: INVALID_ARG (unknown mode, step < 1, or no width searched). */
#define PULSCAN_WIDTHS_ALL 0
#define PULSCAN_WIDTHS_STEP 1
#define PULSCAN_WIDTHS_LOG2 2
PULSCAN_API int pulscan_plan_set_widths(pulscan_plan plan, int32_t mode, int32_t step);

/* Paper-GPU fidelity (§2.5, §2.6 and their appendix listings), for comparing
 * the GPU version's approximations with the exact path:
 *   PULSCAN_FIDELITY_EXACT (0): exact median/MAD and exact chi-square
 *     significance (the default);
 *   PULSCAN_FIDELITY_PAPER_GPU (1): median and MAD of each component by
 *     median of medians over the first segment_len bins of each block (stride-4
 *     groups of local medians, scale 1.4826), and significance by the fitted
 *     polynomial log p(pow = 2 S, dof = 2 a) of §2.6 for every (segment,
 *     width) maximum (the polynomial is not monotone in the power, so every
 *     maximum is evaluated; the search then costs the unthresholded bank).
 * Mode 1 needs segment_len = 4^k <= 16384 (INVALID_ARG / UNSUPPORTED).  The
 * logsumexp entry points return UNSUPPORTED in mode 1. */
#define PULSCAN_FIDELITY_EXACT 0
#define PULSCAN_FIDELITY_PAPER_GPU 1
PULSCAN_API int pulscan_plan_set_fidelity(pulscan_plan plan, int32_t mode);

/* Autotuner of the bank's launch shape: runs the search (bank, deferred
 * blocks, finaliser) on the caller's normalised power d_power three times for
 * each of 1, 2, 3 and 4 warps per CTA, in the scalar form (a warp owns 1056
 * start bins, tile = 1056 x warps) and the packed form (a warp owns two 1056-
 * bin slices and adds them pairwise with add.f32x2, tile = 2112 x warps),
 * each with one CTA per tile and with a persistent grid of per-SM tile
 * ranges, and keeps the fastest; then, on that shape, the deferred blocks'
 * two forms (pulscan_plan_set_defer_form), three runs each.  Segment length,
 * widths and halo are fixed by the search itself, and the two forms perform
 * the same FP32 adds in the same order, so the candidates do not depend on
 * the choice.  Synchronises
 * `stream`, discards the candidates of the trial runs and drops the plan's
 * captured graph.  pulscan_plan_tiling reports the current choice
 * (persistent: -1 automatic, the default; 0 one CTA per tile; 1 persistent;
 * packed: 0 scalar, 1 packed). */
PULSCAN_API int pulscan_plan_autotune(pulscan_plan plan, const float *d_power, pulscan_stream stream);
PULSCAN_API int pulscan_plan_tiling(pulscan_plan plan, int32_t *warps, int32_t *persistent, int32_t *packed);
/* Set the launch shape directly (warps 1 to 4; persistent -1, 0 or 1;
 * packed 0 or 1).  Synchronises the device.  Errors: INVALID_ARG. */
PULSCAN_API int pulscan_plan_set_tiling(pulscan_plan plan, int32_t warps, int32_t persistent, int32_t packed);

/* Pipelined batch search (a schedule of Algorithm 4's search over many
 * series; the results are those of the sequential path).  pulscan_search
 * with use_graph = 1 on a plan of several series splits them into parts of
 * about part_bins bins (consecutive series of one length, in layout order)
 * and captures, per part, its R2C transform and normalisation on a
 * high-priority side stream and its boxcar bank on the capture stream after
 * them, so that the bank of one part overlaps the transform and the
 * normalisation of the next; the deferred blocks and the finaliser follow
 * the last part.  part_bins = 0 (the default) turns it off: the stages run
 * one after another over the whole batch, which measured faster on GB300
 * (the bank's CTAs hold every SM's registers, so the side stream's work
 * cannot run beside it).  Plans with harmonic stages, the paper-GPU fidelity
 * mode or blocks too large for the register normalisation kernel always run
 * the stages in turn.  Builds one
 * cuFFT plan per (length, series count) of the parts, with one shared work
 * area; synchronises the device and drops the plan's captured graph.
 * Errors: INVALID_ARG, NOMEM, CUDA. */
PULSCAN_API int pulscan_plan_set_pipeline(pulscan_plan plan, int64_t part_bins);

/* Fused normalisation and search (§2.2.3 Eq. 8 and §2.2.5 / Algorithm 4 in
 * one pass over the power): with on = 1, pulscan_search (with or without a
 * graph) runs the R2C transform, then only the block statistics of Eq. 8
 * (the exact medians and MADs, kept per segment as (med, 1 / (kappa MAD))
 * pairs), then the boxcar bank, which forms every staged bin's power from
 * the spectrum and its segment's pair as it stages its tile, and the
 * deferred blocks likewise: P never goes to device memory, and d_power is
 * neither read nor written.  The powers formed are bit-identical to
 * pulscan_power_normalise's, so the candidates are those of the separate
 * stages.  on = 0 (the default) restores the separate stages.  Only for the
 * exact mode without harmonic stages and segments of at most 16385 bins
 * (UNSUPPORTED otherwise); overrides the pipelined schedule.  Allocates 16
 * bytes per segment on first use, synchronises the device and drops the
 * plan's captured graph.  Errors: INVALID_ARG, UNSUPPORTED, NOMEM. */
PULSCAN_API int pulscan_plan_set_fused(pulscan_plan plan, int32_t on);

/* Number of parts a captured pulscan_search of the plan is pipelined over
 * (0: it runs sequentially).  Errors: INVALID_ARG. */
PULSCAN_API int pulscan_plan_pipeline_parts(pulscan_plan plan, int64_t *n_parts);

/* A test of the search's bounded-wait path that faults nothing: arms the
 * plan's next boxcar search so that its bank kernel issues no copy into
 * its staging buffer and waits on that copy's barrier for limit_us
 * microseconds (1..1000), then flags the timeout and exits, with nothing in
 * flight; pulscan_candidates of that search returns PULSCAN_ERR_TIMEOUT (and
 * no candidates), and the search after it runs normally.  pulscan_search
 * runs an armed search outside its CUDA graph.  Errors: INVALID_ARG. */
PULSCAN_API int pulscan_plan_test_wait_timeout(pulscan_plan plan, int32_t limit_us);

/* Approximate r-bin output (§2.4, "Pulscan R-Block"): with block_width > 0,
 * pulscan_candidates / pulscan_search_host report in `bin` the block index
 * floor(k / block_width) of each candidate instead of its start bin k (the
 * paper's default block width is 32768); 0 restores exact bins.  The order
 * of the records is unchanged.  Errors: INVALID_ARG (block_width < 0). */
PULSCAN_API int pulscan_plan_set_rblock(pulscan_plan plan, int64_t block_width);

/* Copy the FP32 power threshold T_w of series `series` (w = 1..z_max) to
 * h_thresh[0..z_max-1]: the smallest float S with sigma(S) >= threshold_sigma.
 * Host-synchronous. */
PULSCAN_API int pulscan_plan_thresholds(pulscan_plan plan, int32_t series, float *h_thresh);

/* The same threshold for one width, on the host only (no CUDA call, no plan;
 * §2.2.3 Eq. 9 with the Bonferroni count of §2.2.3): *t_out = the smallest
 * float T with ln Q(shape, T) + ln n_trials <= ln Phi_c(sigma_thr), where
 * Q is the regularised upper incomplete gamma function and shape the gamma
 * shape of the sum (w for a width-w sum of the power, H(H+1)/2 w for the
 * H-harmonic sum of §2.3).  Errors: INVALID_ARG (shape <= 0, n_trials < 1, sigma_thr < 0 or not
 * finite, null t_out). */
PULSCAN_API int pulscan_threshold_power(double shape, double n_trials, double sigma_thr, float *t_out);

/* R2C FFT of every series (cuFFT, unnormalised, e^{-2 pi i k n/N}): d_x
 * float[x_floats] -> d_spec float[spec_floats] as (re, im) pairs. */
PULSCAN_API int pulscan_rfft(pulscan_plan plan, const float *d_x, float *d_spec, pulscan_stream stream);

/* Normalised power (§2.2.3, Eq. 8): per segment and per component, median and
 * MAD (exact order statistics; even counts average the two middle ones; DC
 * bin taken as 0), a = (Re - med)/(kappa MAD), kappa = 1/Phi^{-1}(3/4),
 * P = (a^2 + b^2)/2.  d_spec float[spec_floats] -> d_power float[power_floats].
 * d_stats (nullable) receives float[4 * total_segments]: per segment
 * (med_re, mad_re, med_im, mad_im).  A segment with MAD = 0 gets P = 0.
 * On a harmonic plan the call also writes the stage spectra X_H into
 * d_power (their d_stats rows are left untouched). */
PULSCAN_API int pulscan_power_normalise(pulscan_plan plan, const float *d_spec, float *d_power, float *d_stats,
                            pulscan_stream stream);

/* Boxcar bank + threshold search (§2.2.5, Algorithm 4): for every segment s
 * and width w, the maximum of S_w[k] = sum_{j<w} P[k+j] over the segment's
 * valid start bins (lowest k on ties) becomes a candidate when it is >= T_w.
 * Candidates land in the plan's device buffer; read them with
 * pulscan_candidates.  d_power is read only. */
PULSCAN_API int pulscan_boxcar_search(pulscan_plan plan, const float *d_power, pulscan_stream stream);

/* Copy the candidates of the last pulscan_boxcar_search to h_out, ordered by
 * (series, segment, width).  Synchronises `stream`.  *n_out = the true count;
 * if it exceeds cap (or the plan's buffer), the first cap records are written
 * and PULSCAN_ERR_CAPACITY is returned.  PULSCAN_ERR_TIMEOUT if a device-side
 * bounded wait gave up during the search. */
PULSCAN_API int pulscan_candidates(pulscan_plan plan, pulscan_cand *h_out, int64_t cap, int64_t *n_out,
                       pulscan_stream stream);

/* All per-(segment, width) maxima, thresholded or not (Algorithm 4 without
 * the threshold): d_max float[total_segments * z_max] (row = segment, column
 * = w - 1) and d_argmax uint64[...] (start bin within the series).  Entries
 * with no valid window get NaN and UINT64_MAX. */
PULSCAN_API int pulscan_segment_maxima(pulscan_plan plan, const float *d_power, float *d_max, uint64_t *d_argmax,
                           pulscan_stream stream);

/* pulscan_segment_maxima without allocating: for callers that cannot call
 * cudaMalloc (a real-time pipeline whose device memory all comes from its
 * own pool, where an allocation would synchronise the device; a process under
 * a hard memory cap).  The paper has no counterpart; it is this library's
 * service to such callers.  One series of n samples (validated as in
 * pulscan_plan_create, Bonferroni not involved): d_power float[n/2 + 1] (read
 * only, 16-byte aligned), d_max float[n_seg * z_max] and d_argmax
 * uint64[n_seg * z_max] with the layout of pulscan_segment_maxima.  Scratch
 * is one library-owned static device array of 8 MiB (plus a small header)
 * that each GPU loading the library keeps until exit; the call itself
 * allocates nothing.  Limits: n_seg * z_max <= 2^20, z_max <= 4096 and
 * n < 2^33, else PULSCAN_ERR_UNSUPPORTED; all size checks come before any
 * CUDA call.  The first call on a device sets up (looks up the
 * array's device address, raises the kernel's shared-memory limit): make it
 * before any stream capture.  All calls share the array, so calls that
 * overlap on the GPU race; serialise them. */
PULSCAN_API int pulscan_segment_maxima_noalloc(const float *d_power, int64_t n, int32_t z_max,
                                               int32_t segment_len, float *d_max, uint64_t *d_argmax,
                                               pulscan_stream stream);

/* Whole path (FFT, normalise, search) for a plan: the first call with a given
 * (d_x, d_spec, d_power, stream) captures the kernels into a CUDA graph when
 * use_graph != 0, later calls replay it. */
PULSCAN_API int pulscan_search(pulscan_plan plan, const float *d_x, float *d_spec, float *d_power, int use_graph,
                   pulscan_stream stream);

/* Whole path from HOST memory: copies h_x (float[x_floats], pinned or
 * pageable) into device buffers owned by the plan (allocated on the first
 * call), runs pulscan_search on them and returns the candidates exactly as
 * pulscan_candidates does.  Synchronises `stream`. */
PULSCAN_API int pulscan_search_host(pulscan_plan plan, const float *h_x, pulscan_cand *h_out, int64_t cap,
                                    int64_t *n_out, int use_graph, pulscan_stream stream);

/* The first half of pulscan_search_host, asynchronous: enqueues on `stream`
 * the copy of h_x (float[x_floats]) into the plan's own device buffers and
 * pulscan_search on them, and returns without waiting.  h_x must stay valid
 * and unchanged until the copy has run (pinned memory lets it overlap with
 * other work); collect the candidates with pulscan_candidates on the same
 * stream.  Two plans used in turn on two streams pipeline a stream of series:
 * one series' copy runs while the other's search does.  Errors as
 * pulscan_search; NOMEM for the first call's buffers. */
PULSCAN_API int pulscan_search_host_async(pulscan_plan plan, const float *h_x, int use_graph, pulscan_stream stream);

/* Differentiable extension (a smooth relaxation of Algorithm 4's per-chunk
 * maximum; the paper has no gradient): for every segment s and width w,
 *   Y[s, w] = tau * log sum_{k in s, k <= M - w} exp(S_w[k] / tau),
 * which tends to the segment maximum as tau -> 0.  Runs the R2C FFT and the
 * normalisation (Eq. 8) itself.  d_x float[x_floats] (read only); d_spec
 * float[spec_floats], d_power float[power_floats], d_stats
 * float[4 * total_segments] and d_sel float[8 * total_segments] (the
 * selected order statistics the adjoint needs) are written and must be kept
 * for pulscan_lse_backward; d_y float[total_segments * z_max] (row = segment,
 * column = w - 1) and d_ylo (same layout): Y's FP32 rounding error, so that
 * d_y + d_ylo carries Y well below FP32 resolution (the adjoint's softmax
 * weights exp((S - Y) / tau) amplify an error in Y by 1 / tau); keep it for
 * pulscan_lse_backward.  Terms more than tau ln(2^24 L) below the segment maximum
 * are skipped: they are below FP32 resolution of the sum.  tau > 0.
 * Segments must be at most 4224 bins (else PULSCAN_ERR_UNSUPPORTED). */
PULSCAN_API int pulscan_lse_forward(pulscan_plan plan, const float *d_x, float *d_spec, float *d_power,
                                    float *d_stats, float *d_sel, float *d_y, float *d_ylo, float tau,
                                    pulscan_stream stream);

/* Adjoint of pulscan_lse_forward: given d_gy = dL/dY (same layout as d_y)
 * and the forward's d_spec, d_power, d_stats, d_sel, d_y, d_ylo, writes
 * d_gx = dL/dx float[x_floats].  The chain: softmax weights; the boxcar
 * scatter dL/dP[j] = sum_w sum_{k=j-w+1..j} dL/dS_w[k]; P = (a^2 + b^2)/2;
 * the median / MAD normalisation with its almost-everywhere derivatives at
 * the selected order statistics; the real FFT (DC bin zeroed, so it carries
 * no gradient), via cuFFT C2R.  Uses plan-owned scratch allocated on first
 * use (dL/dP, the segment tails, the C2R input); overlapping backward calls
 * on one plan race. */
PULSCAN_API int pulscan_lse_backward(pulscan_plan plan, const float *d_spec, const float *d_power,
                                     const float *d_stats, const float *d_sel, const float *d_y,
                                     const float *d_ylo, const float *d_gy, float *d_gx, float tau,
                                     pulscan_stream stream);

/* Synthetic signal model of the differentiable workload (§2.1, Eq. 1):
 * d_x = d_noise + amp[i] * d_template for every series i (all
 * float[x_floats] in the plan's layout; d_amp float[n_series] in the
 * caller's series order). */
PULSCAN_API int pulscan_inject(pulscan_plan plan, const float *d_noise, const float *d_template,
                               const float *d_amp, float *d_x, pulscan_stream stream);

/* dL/dA[i] = sum_n dL/dx[n] template[n] over series i (FP64 accumulation),
 * d_gamp float[n_series] in the caller's series order.  The plan allocates
 * 128 bytes per series of partial sums on the first call (16 CTAs per
 * series; the partials are added in a fixed order, so the result is
 * deterministic). */
PULSCAN_API int pulscan_amplitude_grad(pulscan_plan plan, const float *d_gx, const float *d_template,
                                       float *d_gamp, pulscan_stream stream);

/* Per-kernel timing with CUDA events on the launch stream: on = 1 records
 * every stage, on = 2 only the boxcar search kernel (each event between two
 * kernels costs a few microseconds of pipeline drain), 0 disables recording;
 * pulscan_plan_timings then writes the milliseconds of
 * the most recent launch of [rfft, normalise, boxcar search kernel,
 * deferred-block kernel, candidate finalise, segment-maxima kernel, harmonic
 * sums] (-1 where not run) to h_ms[0..min(n,7)-1].  Synchronises the events.
 * With timing on, pulscan_search(use_graph = 1) captures the events into its
 * graph, and every launch of the graph records them again; changing the
 * setting drops the plan's captured graph (the next call captures anew). */
PULSCAN_API int pulscan_plan_enable_timing(pulscan_plan plan, int on);
PULSCAN_API int pulscan_plan_timings(pulscan_plan plan, float *h_ms, int32_t n);

/* Counters of the last pulscan_boxcar_search (host-synchronous):
 * h_out[0..min(n,4)-1] = [blocks deferred to the deferred-block kernel,
 * deferred-block capacity, candidates found, candidate capacity].  A search
 * whose deferred blocks exceed the capacity runs the excess blocks exactly
 * inside the main kernel instead (same results, slower). */
PULSCAN_API int pulscan_plan_counters(pulscan_plan plan, int64_t *h_out, int32_t n);

/* Set the deferred-block list to cap items (0 = every flagged block is run
 * exactly by its own warp; at most 2^24).  A cap above the allocated one
 * reallocates the list (4.2 KB per item; synchronises the device and drops
 * the plan's captured graph).  Errors: INVALID_ARG, NOMEM. */
PULSCAN_API int pulscan_plan_set_defer_capacity(pulscan_plan plan, int64_t cap);

/* How the deferred blocks (the 33-width blocks of Algorithm 4's scan whose
 * exact bound reached the threshold, re-run from their snapshots) are
 * inspected: form 0 = three warps per block (11 bins per thread, merged
 * through shared memory), form 1 = one warp per block (33 bins per lane, a
 * warp max-reduction per width; the block's bin search only for a maximum
 * that reaches T_w).  Same records either way.  Form 1 wins when the blocks
 * fill the GPU several times over, form 0 when few blocks leave one block's
 * chain of steps exposed.  Default: 1 for plans of 2^25 power bins or more,
 * else 0; pulscan_plan_autotune times both on the caller's data and keeps
 * the faster.  Drops the plan's captured graph when the form changes.
 * Errors: INVALID_ARG (null plan, form not 0 or 1). */
PULSCAN_API int pulscan_plan_set_defer_form(pulscan_plan plan, int32_t form);
/* The current form of pulscan_plan_set_defer_form (0 or 1) in *form (host
 * memory, written only on success).  Errors: INVALID_ARG (null plan or
 * form). */
PULSCAN_API int pulscan_plan_defer_form(pulscan_plan plan, int32_t *form);

/* The FP32 add rate of the current GPU, the ceiling of the boxcar bank
 * (§2.2.5: one add per bin and width), measured rather than derived: a
 * kernel of independent adds on every SM (8 CTAs of 256 threads per SM,
 * 32 running sums per thread), timed with CUDA events on `stream`, best of
 * `reps` launches after two untimed ones.  h_out[0] = adds/s with packed
 * pairs (add.rn.f32x2), h_out[1] = adds/s with scalar adds, h_out[2], h_out[3]
 * = the SM clock in MHz during each (clock64 ticks per globaltimer ns of the
 * first CTA); the first min(n, 4) entries are written.  Allocates and frees
 * a small device buffer; synchronises `stream`.  Errors: INVALID_ARG, NOMEM,
 * CUDA. */
PULSCAN_API int pulscan_measure_add_peak(double *h_out, int32_t n, int32_t reps, pulscan_stream stream);

/* Message of the last error on this thread ("" if none). */
PULSCAN_API const char *pulscan_last_error(void);

/* Library version (major * 10000 + minor * 100 + patch). */
PULSCAN_API int pulscan_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PULSCAN_H */
