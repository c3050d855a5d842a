/*
 * fstat.h -- C ABI of the GB300 coherent F-statistic library (libfstat.so).
 *
 * The library computes the multi-detector coherent F-statistic (2F) of a bank
 * of continuous-wave templates (sky position, frequency, spindown) over short
 * Fourier transforms (SFTs), and keeps the top-K candidates.  Its calls follow
 * the paper's statement of the problem: the F-statistic of a frequency band is
 * a loop over frequencies of a sum over detectors of a sum over SFTs
 * (Listing 1, Section "Einstein@Home": ComputeFStatFreqBand / ComputeFStat /
 * ComputeFaFb), fed by flat SFT data arrays with offset arrays instead of a
 * pointer tree (Section "CUDA", version 2 data structure).
 *
 * Per template lambda = (alpha, delta, f, fdot) and SFT alpha of detector d
 * (start t_a, length T, complex bins X_k at absolute bin k):
 *   dtau   = t_m - t_ref + n.r_d(t_m)/c,  tdot = 1 + n.v_d(t_m)/c,  t_m = t_a + T/2
 *   khat   = (f + fdot dtau) tdot T,   k0 = floor(khat),  kappa = khat - k0
 *   Phi    = 2 pi (f dtau + fdot dtau^2 / 2)
 *   z      = (-1)^k0 e^{-i Phi} (sin(pi kappa)/pi) sum_{k=k0-D+1}^{k0+D} X_k/(khat - k)
 *   Fa     = sum a z,  Fb = sum b z  (over all SFTs of all detectors)
 *   2F     = 2 (B|Fa|^2 + A|Fb|^2 - 2C Re(Fa Fb*)) / (AB - C^2),
 *            A = sum a^2, B = sum b^2, C = sum ab.
 * The body of the SFT term is the standard Dirichlet-kernel demodulation that
 * the paper's pseudo-code abbreviates as some_calculations / normalized.
 *
 * Conventions
 *   - Every call returns an fstat_status (0 = FSTAT_OK); nothing throws.  On
 *     error, fstat_last_error(ctx) returns a NUL-terminated message owned by
 *     the context, valid until the next call on it.
 *   - The library copies every input; callers keep ownership of their buffers
 *     and may free them when the call returns.  Outputs go to caller-owned
 *     buffers.  Device memory is owned by the context and released by
 *     fstat_destroy().
 *   - Pointer arguments marked "host or device" are device pointers when the
 *     accompanying `mem` argument is FSTAT_MEM_DEVICE (they must belong to
 *     the context's device) and host pointers otherwise.
 *   - A context is bound to one device and one CUDA stream at a time; it is
 *     not thread-safe.  Separate contexts are independent.
 *   - Template index of (sky s, spindown d, frequency j):
 *       idx = ((s * n_fdot) + d) * n_f + j.
 */
#ifndef FSTAT_H
#define FSTAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fstat_ctx fstat_ctx;

typedef enum {
    FSTAT_OK = 0,
    FSTAT_EINVAL = -1,    /* invalid argument (sizes, non-finite data, D < 1 ...) */
    FSTAT_ENOMEM = -2,    /* device allocation failed */
    FSTAT_ECUDA = -3,     /* a CUDA runtime call failed */
    FSTAT_ESTATE = -4,    /* call out of order (e.g. compute before SFTs/templates) */
    FSTAT_ERANGE = -5,    /* a template's window left the staged SFT range */
    FSTAT_ETIMEOUT = -6   /* a bounded device wait gave up */
} fstat_status;

/* Storage of the SFT bins on the device. */
typedef enum {
    FSTAT_BINS_C64 = 0,   /* complex64: FP32 re, im */
    FSTAT_BINS_F16 = 1,   /* FP16 re, im times a per-SFT FP32 scale */
    FSTAT_BINS_BF16 = 2   /* BF16 re, im times a per-SFT FP32 scale */
} fstat_bins_form;

typedef enum { FSTAT_MEM_HOST = 0, FSTAT_MEM_DEVICE = 1 } fstat_mem;

typedef struct {
    int32_t dterms;       /* D >= 1: the SFT term sums 2D bins around khat */
    int32_t bins_form;    /* fstat_bins_form */
    int32_t topk;         /* toplist length kept by fstat_compute (0..16384) */
    int32_t kahan;        /* 1: compensated (Kahan) summation of Fa, Fb over SFTs */
    int32_t tile_m;       /* templates per thread (0 = chosen by the tuner) */
    int32_t tile_warps;   /* warps per thread block (0 = chosen by the tuner).  The far-field form on
                             a uniform spindown grid with L = 2 runs TMA-ring staging (10 compute
                             warps + 1 copy warp by default; 9 or 11 choose 8 or 10 compute warps);
                             2..8 or 10 select its shared-memory-round staging instead */
    int32_t sft_chunk;    /* SFTs staged per shared-memory round (0 = tuner) */
    int32_t algo;         /* fstat_algo: how the D-term kernel sum is evaluated */
} fstat_opts;

/* Evaluation of the kernel sum over the 2D bins (fstat_opts.algo).
 * DIRECT: every bin's term, two bins per reciprocal (any D, Kahan allowed).
 * FARPOLY (D = 8, no Kahan): the four bins next to kappa's poles exactly, the
 *   other twelve through a degree-5 polynomial in kappa whose coefficients
 *   are precomputed per SFT and window position (interpolation error below
 *   5e-6 of each term); needs two tables of 16 and 48 bytes per stored bin
 *   and SFT.
 * SINCPOLY (D = 8, no Kahan): the whole window term, sin(pi kappa)/2 times
 *   the 2D-bin sum, is entire in kappa; on each half of the bin (kappa < 1/2
 *   and kappa >= 1/2) it is evaluated as a degree-5 polynomial whose
 *   coefficients are precomputed per SFT, window position and half (two
 *   48-byte records per stored bin and SFT; interpolation error below 2.1e-6
 *   of each term; no reciprocal, sine or clamp per template).  It runs in the
 *   TMA-ring staging on a uniform spindown grid: P df T = 2 (5 or 7 templates
 *   per thread) or P df T = 1 with P = 8 (1 or 5); elsewhere it falls back
 *   to FARPOLY.
 * SINCROWS (D = 8, no Kahan, uniform spindown grid of at least 4 spindowns,
 *   no frequency coverage): the same sinc-polynomial records evaluated with
 *   one frequency and up to 10 spindown rows per thread; a row whose window
 *   and half bin equal the previous row's reuses the record held in
 *   registers, so records are read once per run of rows instead of once per
 *   template (plain tables, TMA-ring staging); elsewhere as SINCPOLY.
 * SINCPAIRS (D = 8, no Kahan, P df T = 2, uniform spindown grid of at least
 *   2 spindowns, no frequency coverage): the SINCPOLY ring with each thread
 *   holding its templates in two adjacent spindown rows, one record serving
 *   both rows where their windows and half bins agree; elsewhere as SINCPOLY.
 * SINCROWS and SINCPAIRS give the same results within the stated tolerance
 *   and are slower than SINCPOLY on the workunit-sized bank; they are kept as
 *   options.  Batched workunits use the TMA-ring form where it applies, else
 *   DIRECT.
 * AUTO: the TMA ring where it applies: SINCPOLY, or on banks of one or two
 *   spindowns with L = 2 (where the ring can be bound by its table copies)
 *   whichever of SINCPOLY and FARPOLY's smaller records the planner's model
 *   finds faster; banks of one or two spindowns run blocks of 4 neighbouring
 *   sky points (consecutive ones of the bank, or of a neighbour order of its
 *   sky list) sharing one staged window; else FARPOLY where it applies, else
 *   DIRECT.  Results do not depend on the grouping. */
typedef enum {
    FSTAT_ALGO_AUTO = 0,
    FSTAT_ALGO_DIRECT = 1,
    FSTAT_ALGO_FARPOLY = 2,
    FSTAT_ALGO_SINCPOLY = 3,
    FSTAT_ALGO_SINCROWS = 4,
    FSTAT_ALGO_SINCPAIRS = 5
} fstat_algo;

typedef struct {
    double lat_rad;       /* geodetic latitude of the vertex */
    double lon_rad;       /* longitude of the vertex (east positive) */
    double xarm_az_rad;   /* azimuth of the x-arm from local North, clockwise;
                             the y-arm points at azimuth + pi/2 */
} fstat_detector;

/* One continuous-wave signal for fstat_inject (amplitude set by its SNR). */
typedef struct {
    double alpha, delta;  /* sky position (equatorial, rad) */
    double psi;           /* polarisation angle */
    double cosi;          /* cosine of the inclination */
    double phi0;          /* initial phase at t_ref */
    double f, fdot;       /* frequency (Hz) and spindown (Hz/s) at t_ref */
    double rho;           /* optimal SNR; h0 follows from it and A, B, C */
} fstat_signal;

/* Library version string, static storage. */
const char *fstat_version(void);

/* Create a context on CUDA device `device`.  opts == NULL takes the defaults
 * (D = 8, complex64 storage, topk = 1000, no Kahan, tuned tiles).
 * Errors: EINVAL (D < 1 or > 64, topk outside 0..16384, unknown form or
 * algo, FARPOLY with D != 8 or Kahan), ECUDA (device unavailable), ENOMEM. */
int fstat_create(fstat_ctx **out, int device, const fstat_opts *opts);

/* Release the context and all its device memory.  NULL is ignored. */
void fstat_destroy(fstat_ctx *ctx);

/* Message of the last failed call on ctx ("" if none; ctx may be NULL). */
const char *fstat_last_error(const fstat_ctx *ctx);

/* Load the SFTs of detector `det_index` (0 <= det_index < 8): the "load SFTs"
 * step, one detector's SFTs into the flat data array with its offsets
 * (Section "CUDA", version 2 data structure; the per-detector SFT loop of
 * Listing 1's ComputeFStat reads them).  All detectors
 * of a context share T, k_lo and n_bins.  Loading a detector again replaces
 * its SFTs.
 *   det      geometry of the detector (host)
 *   Tsft     SFT length in seconds (> 0)
 *   k_lo     absolute index of the first stored bin (frequency k_lo / Tsft)
 *   n_bins   stored bins per SFT (>= 2)
 *   n_sft    number of SFTs (>= 1)
 *   t_start  [n_sft] SFT start times, host (finite)
 *   bins     [n_sft][n_bins][2] FP32 (re, im), host or device per `mem`
 * Bins outside [k_lo, k_lo + n_bins) count as zero in every SFT term.
 * Errors: EINVAL (sizes, non-finite times or bins, mismatch with the other
 * detectors' T / k_lo / n_bins), ENOMEM, ECUDA. */
int fstat_set_sfts(fstat_ctx *ctx, int32_t det_index, const fstat_detector *det, double Tsft,
                   int64_t k_lo, int32_t n_bins, int32_t n_sft, const double *t_start,
                   const float *bins, int32_t mem);

/* Set the template bank: n_sky sky positions x n_fdot spindowns x n_f
 * frequencies f_j = f0 + j df, all at reference time t_ref (the frequency
 * band that Listing 1's ComputeFStatFreqBand loops over, for each sky
 * position and spindown).
 *   sky   [n_sky][2] (alpha, delta) radians, host
 *   fdot  [n_fdot] Hz/s, host
 * Errors: EINVAL (counts < 1, df <= 0, non-finite values, more than 2^40
 * templates), ENOMEM. */
int fstat_set_templates(fstat_ctx *ctx, const double *sky, int32_t n_sky, double f0, double df,
                        int32_t n_f, const double *fdot, int32_t n_fdot, double t_ref);

/* Compute 2F of every template and the top-K toplist, asynchronously on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream): the whole
 * of Listing 1 (Section "Einstein@Home") -- ComputeFaFb's sum of
 * some_calculations over each detector's SFTs, ComputeFStat's sum over
 * detectors and the normalized combine, for every frequency of the band.
 * Runs: per-SFT detector state, per-(sky, SFT) timing / antenna / phase and
 * bin bases in FP64, the Dirichlet accumulation and 2F combine in FP32, and
 * the toplist selection.  Results stay on the device until read.
 * Errors: ESTATE (no SFTs or no templates), ECUDA (launch failure). */
int fstat_compute(fstat_ctx *ctx, void *cuda_stream);

/* Copy 2F of templates [offset, offset + count) to `out` (host or device per
 * `mem`), after synchronising the context's stream.  FP32.  (The per-frequency
 * result ComputeFStat returns in Listing 1.)
 * Errors: ESTATE (nothing computed), EINVAL (range); ETIMEOUT (flag bit 2)
 * or ERANGE (flag bit 0) if the computation raised that device flag, with
 * `out` written all the same. */
int fstat_get_2f(fstat_ctx *ctx, float *out, int64_t offset, int64_t count, int32_t mem);

/* Copy the first k (<= topk) toplist entries, ordered by 2F descending then
 * template index ascending, to host arrays idx[k] and twoF[k].  Synchronises.
 * (The candidates the Einstein@Home client keeps from the F-statistic stage
 * for its later stage, Section "Einstein@Home"; the ordering of equal values
 * by index is this library's.)
 * Errors: ESTATE, EINVAL (k out of range); ETIMEOUT / ERANGE as for
 * fstat_get_2f, with the entries written all the same. */
int fstat_get_toplist(fstat_ctx *ctx, int32_t k, int64_t *idx, float *twoF);

/* Per-sky antenna-pattern sums of the last compute: out[n_sky][4] =
 * (A, B, C, D) in FP64 (host).  Synchronises. */
int fstat_get_abcd(fstat_ctx *ctx, double *out);

/* Per-SFT timing and antenna values of sky point `sky` from the last compute,
 * for all SFTs of all detectors in load order (detector 0 first): dtau, tdot
 * (FP64) and a, b (FP64), host arrays of length n_sft_total.  Synchronises. */
int fstat_get_sft_timing(fstat_ctx *ctx, int32_t sky, double *dtau, double *tdot, double *a,
                         double *b);

/* Add n_sig model-exact continuous-wave signals to the loaded SFT bins
 * (all detectors), X_k += (T/2)(a c_a + b c_b) e^{i Phi} (-1)^k sinc(khat - k),
 * the Fourier transform of the signal with its phase linearised about each
 * SFT midpoint, with h0 chosen so that the signal's optimal SNR is rho
 * (rho^2 = (T^2/2)(A|c_a|^2 + B|c_b|^2 + 2C Re(c_a c_b*))).  The sum of the
 * stored bins and all signals is formed in FP64 and rounded to FP32 once.
 *   sig   [n_sig] host;  t_ref reference time of the signals' phase.
 * Errors: ESTATE (no SFTs), EINVAL. */
int fstat_inject(fstat_ctx *ctx, const fstat_signal *sig, int32_t n_sig, double t_ref);

/* Copy the stored complex64 bins of detector det_index (after any
 * injections) to out[n_sft][n_bins][2] FP32, host or device per `mem`.
 * Synchronises.  Errors: EINVAL (detector not loaded), ECUDA. */
int fstat_get_bins(fstat_ctx *ctx, int32_t det_index, float *out, int32_t mem);

/* Device-side error flags raised by the last compute (0 = none); synchronises.
 * Bit 0: a template window left the staged SFT range (clamped).
 * Bit 1: a sky point (or, with coverage, a frequency) had a degenerate
 *        D = AB - C^2 (its 2F set to 0).
 * Bit 2: a wait of the far-field ring pipeline gave up (that block's 2F invalid). */
int fstat_get_error_flags(fstat_ctx *ctx, int32_t *flags);

/* Noise-floor normalisation and noise weights (no counterpart in the paper's
 * white-noise client; the step before the path for coloured, non-stationary
 * noise).  With half_window W in 1..64, from the next fstat_compute on:
 *   S(k) = median of |X_j|^2 (FP32) over the stored bins j with |j - k| <= W
 *          (clipped at the band edges; an even count averages its two middle
 *          values) divided by ln 2;
 *   every bin the path reads is X_k / sqrt(S(k)) (0 where S(k) = 0); the
 *          stored SFTs themselves (fstat_get_bins) are unchanged;
 *   every SFT gets the weight w = (1/Sbar) / mean over all SFTs of (1/Sbar),
 *          Sbar = the SFT's mean S, applied as sqrt(w) a, sqrt(w) b in A, B,
 *          C, Fa and Fb (w = 0 where Sbar = 0, left out of the mean).
 * W = 0 switches it off (the default).  Errors: EINVAL (W outside 0..64). */
int fstat_set_noise_floor(fstat_ctx *ctx, int32_t half_window);

/* Per-SFT frequency coverage: a varying number of SFTs per frequency (the
 * data the paper's version-3 client pads its thread blocks for, Section
 * "CUDA").  SFT i (in load order: all SFTs of detector 0, then detector 1,
 * ...) contributes only to templates whose frequency index j (f = f0 + j df)
 * lies in [j_lo[i], j_hi[i]); each template's A, B, C, D are summed over
 * the SFTs that cover it:
 *   Fa(j) = sum_{i covers j} a_i z_i(j),   A(j) = sum_{i covers j} a_i^2, ...
 * A frequency no SFT covers gets 2F = 0 (no flag); a degenerate D elsewhere
 * raises flag bit 1.  Ranges may reach outside [0, n_f) (clamped).
 * An SFT that covers none of a thread's templates is skipped, so work falls
 * with coverage.  From the next fstat_compute on; both pointers NULL switch
 * coverage off.  Loading SFTs (fstat_set_sfts) switches it off too.
 * Restrictions: n_f <= 8192 while coverage is on; the far-field form runs
 * only in its TMA-ring staging (elsewhere the direct form is used); batched
 * workunits have no coverage.  fstat_get_abcd stays the per-sky sum over
 * all SFTs.
 * Errors: EINVAL (one pointer NULL, n_sft != loaded SFTs, j_lo > j_hi),
 * ESTATE (no SFTs loaded), ECUDA. */
int fstat_set_coverage(fstat_ctx *ctx, const int32_t *j_lo, const int32_t *j_hi, int32_t n_sft);

/* The noise floor S [n_sft][n_bins] (FP32; NULL to skip) and the weights
 * [n_sft] (FP64; NULL to skip) of the last compute, SFTs in detector order,
 * host or device per `mem`; synchronises.  Errors: ESTATE (noise floor off or
 * not computed yet), ECUDA. */
int fstat_get_noise(fstat_ctx *ctx, float *floor, double *weights, int32_t mem);

/* Testing aid for failure detection (no counterpart in the paper): from the
 * next fstat_compute on, the copy warp of the far-field ring form stops after
 * `after_sft` SFTs (after_sft < 0 restores normal operation).  The compute
 * warps' bounded waits then expire after about two seconds per block; each
 * block raises error flag bit 2, waits for its own copies in flight and
 * retires, and the context stays usable.  Has no effect on the other forms.
 * Errors: EINVAL (null context). */
int fstat_test_ring_stall(fstat_ctx *ctx, int32_t after_sft);

/* Tile configuration chosen for the current bank (after fstat_set_templates):
 * out[8] = (P, L, M, warps, sft_chunk, lane-groups per column row,
 *           staged pairs per SFT, kernel variant id; ids 100..111 are the
 *           far-field polynomial form, 112..115 the sinc-polynomial form,
 *           116 the sinc and 117 the far-field form with frequency coverage,
 *           118 and 119 the sinc form for L = 1 banks (P = 8); 107 and up use
 *           the TMA-ring staging). */
int fstat_get_plan(fstat_ctx *ctx, int32_t *out);

/* Number of CUDA kernels this context has launched since it was created. */
int fstat_get_launch_count(fstat_ctx *ctx, int64_t *n_launches);

/* Average device time of the Dirichlet kernel over the last `fstat_compute`
 * calls since the previous query, measured with CUDA events recorded around
 * its launch on the compute stream (milliseconds; 0 if none).  Resets the
 * accumulator.  Synchronises. */
int fstat_take_kernel_time(fstat_ctx *ctx, double *ms_dirichlet, double *ms_total, int32_t *n_calls);

/* ---- Measured tile autotuner ------------------------------------------------
 * Time the Dirichlet kernel for candidate tilings (templates per thread M,
 * SFTs per staging round) on a slice of the current bank (the first sky
 * points, a few waves of blocks) and keep the fastest as the context's tile
 * choice for later computes.  out[4] (host, may be NULL) receives
 * (M, sft_chunk, warps, best kernel time on the slice in microseconds).
 * A batch context (workunits only) tunes on its largest workunit and gives
 * every workunit that M; each keeps the stage count its own plan chooses.
 * Synchronises.  Errors: ESTATE (no SFTs or templates). */
int fstat_autotune(fstat_ctx *ctx, void *cuda_stream, int32_t *out);

/* ---- Batched form: many workunits, one persistent launch ----------------------
 * A workunit is a full problem of its own: SFTs of 1..8 detectors sharing T,
 * k_lo and n_bins, and a template bank.  fstat_batch_compute runs, for all
 * workunits added to the context, the per-(sky, SFT) FP64 kernel of each, one
 * persistent Dirichlet kernel per group of workunits with the same kernel
 * variant (its blocks pull (workunit, sky, column, chunk) items from a device
 * queue until every item of every workunit is done), and the toplist of each
 * workunit; the sequence is captured into a CUDA graph on the first call and
 * replayed on later calls (re-captured when workunits are added).  The
 * context's own single-bank state (fstat_set_sfts / fstat_set_templates) is
 * separate and unaffected. */
typedef struct {
    int32_t n_det;                 /* 1..8 */
    const fstat_detector *det;     /* [n_det] host */
    const int32_t *n_sft;          /* [n_det] host */
    const double *const *t_start;  /* [n_det] host pointers to [n_sft[d]] start times */
    const float *const *bins;      /* [n_det] host pointers to [n_sft[d]][n_bins][2] FP32 */
    double Tsft;
    int64_t k_lo;
    int32_t n_bins;
    const double *sky;             /* [n_sky][2] host */
    int32_t n_sky;
    double f0, df;
    int32_t n_f;
    const double *fdot;            /* [n_fdot] host */
    int32_t n_fdot;
    double t_ref;
} fstat_workunit;

/* Add a workunit (inputs copied, host memory); *wu_id receives its index.
 * Errors: as fstat_set_sfts / fstat_set_templates. */
int fstat_batch_add(fstat_ctx *ctx, const fstat_workunit *wu, int32_t *wu_id);

/* Add model-exact signals to workunit wu's SFTs (see fstat_inject). */
int fstat_batch_inject(fstat_ctx *ctx, int32_t wu, const fstat_signal *sig, int32_t n_sig, double t_ref);

/* Remove all workunits and release their memory. */
int fstat_batch_clear(fstat_ctx *ctx);

/* Number of workunits in the batch. */
int fstat_batch_size(fstat_ctx *ctx, int32_t *n_wu);

/* Run the whole batch asynchronously on cuda_stream (see above).
 * Errors: ESTATE (empty batch), ECUDA. */
int fstat_batch_compute(fstat_ctx *ctx, void *cuda_stream);

/* Compute workunit wu alone with the ordinary (one launch per bank) path,
 * asynchronously on cuda_stream; results are read with the calls below.
 * This is the one-launch-per-workunit reference the batch is compared with. */
int fstat_batch_compute_one(fstat_ctx *ctx, int32_t wu, void *cuda_stream);

/* Toplist / 2F of workunit wu after fstat_batch_compute (synchronise); same
 * contracts as fstat_get_toplist / fstat_get_2f. */
int fstat_batch_get_toplist(fstat_ctx *ctx, int32_t wu, int32_t k, int64_t *idx, float *twoF);
int fstat_batch_get_2f(fstat_ctx *ctx, int32_t wu, float *out, int64_t offset, int64_t count, int32_t mem);

/* Timing of the last batch compute: wu_done_ms[n_wu] (host, may be NULL) =
 * device time from the start of the batch to the completion of each
 * workunit's last Dirichlet item; *total_ms = start to end of the batch
 * (CUDA events on the stream).  Synchronises. */
int fstat_batch_get_times(fstat_ctx *ctx, double *wu_done_ms, double *total_ms);

/* Inspection: the tile plan workunit wu runs with, in fstat_get_plan's
 * layout (out[8], host).  Errors: EINVAL (no such workunit), as
 * fstat_get_plan otherwise. */
int fstat_batch_get_plan(fstat_ctx *ctx, int32_t wu, int32_t *out);

#ifdef __cplusplus
}
#endif
#endif /* FSTAT_H */
