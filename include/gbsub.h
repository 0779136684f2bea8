/*
 * gbsub.h -- C ABI of the GB300 library for the iterative galactic-binary
 * subtraction of arXiv 2602.18560 (Sec. III.A and App. D, "Subtraction
 * algorithm").
 *
 * A catalog of N_b sources (amplitude A, frequency f, frequency derivative
 * fdot) goes in; the foreground S_gal(f_k) on the DFT grid f_k = k / T_obs
 * inside [f_min, f_max], and the set of individually resolved sources, come out.
 *
 * Conventions shared by every call:
 *   - Return codes: SUB_OK (0) or a negative SUB_E* code. SUB_ENOTCONVERGED
 *     means the loop hit max_iter; the results are valid for the last
 *     iteration (S_gal re-estimated from the final resolved set).
 *   - sub_last_error() gives a human-readable reason for the last failure.
 *   - All device work of a context is issued on one CUDA stream: the caller's
 *     (sub_create's stream argument, a cudaStream_t) or one the context owns.
 *     sub_load_catalog and sub_run only enqueue work; sub_run with a non-null
 *     stats pointer, sub_get_stats, sub_get_spectrum and sub_get_resolved_mask
 *     synchronise the stream before they return.
 *   - Input and output buffers belong to the caller; the library copies from
 *     and into them and keeps no pointer after the call returns.  A buffer is
 *     host memory (SUB_HOST, pinned or pageable) or device memory of the
 *     current device (SUB_DEVICE), as the `where` argument says.
 *   - The context owns all of its device memory and frees it in sub_destroy.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef GBSUB_H
#define GBSUB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define SUB_OK 0
#define SUB_EINVAL (-1)          /* invalid argument or parameter                      */
#define SUB_ENOMEM (-2)          /* device or host allocation failed                   */
#define SUB_ECUDA (-3)           /* a CUDA runtime call failed                         */
#define SUB_ENOTCONVERGED (-4)   /* max_iter reached; results valid, not converged     */
#define SUB_ETIMEOUT (-5)        /* a bounded device wait gave up                      */
#define SUB_EBUDGET (-6)         /* the context would exceed its hbm_budget            */
#define SUB_ERANGE (-7)          /* a deposited power exceeded the fixed-point range   */
#define SUB_ESTATE (-8)          /* call out of order (e.g. sub_run before a catalog)  */

/* Running estimators of App. D: Eq. (running mean), Eq. (running median) with
 * the chi^2_2 bias constant C = (1 - 2/(9 nu))^-3 = 729/512, and the median
 * followed by the mean over the same window. */
#define SUB_MEAN 0
#define SUB_MEDIAN 1
#define SUB_MEDIAN_MEAN 2

/* Arithmetic of the per-iteration SNR decision and median selection.
 *   SUB_FP64        : FP64 results.  Each rho^2 > rho_th^2 decision is first
 *                     evaluated in FP32 with a proven error bound; only when
 *                     rho^2 lies within that bound of rho_th^2 is it recomputed
 *                     in FP64, so every decision equals the FP64 one.
 *   SUB_MIXED       : the FP32 value of rho^2 decides alone, and the median
 *                     selects on FP32 keys; deposition and window sums stay exact.
 *   SUB_FP64_STRICT : every rho^2 computed in FP64 (for verification).
 * The spectrum itself is always an exact fixed-point sum. */
#define SUB_FP64 0
#define SUB_MIXED 1
#define SUB_FP64_STRICT 2

/* Location of a caller buffer.  SUB_HOST_MAPPED (catalog only): page-locked host memory
 * that the catalog pass reads in place over the host link, with no copy (see
 * sub_load_catalog). */
#define SUB_HOST 0
#define SUB_DEVICE 1
#define SUB_HOST_MAPPED 2

/* Problem statement (Sec. III.A: T_obs, band, grid 1/T_obs; App. C S_instr;
 * App. D window N, rho_th, kappa). */
typedef struct {
  double T_obs;        /* observation time in seconds (> 0); grid spacing 1/T_obs   */
  double f_min;        /* band lower edge in Hz (> 0); paper: 0.1 mHz               */
  double f_max;        /* band upper edge in Hz (> f_min); paper: 10 mHz            */
  int32_t window;      /* smoothing window N in bins, 1 .. 8192; paper: 2000        */
  int32_t estimator;   /* SUB_MEAN | SUB_MEDIAN | SUB_MEDIAN_MEAN                   */
  double rho_th;       /* SNR threshold (> 0); paper: 7                             */
  double kappa;        /* pre-filter factor: candidates have rho_0 >= kappa rho_th  */
  int32_t max_iter;    /* iteration cap (>= 1)                                      */
  int32_t tdi2;        /* 1: apply the TDI-2.0 factor 4 sin^2(2 f/f*) (App. C)      */
  int32_t precision;   /* SUB_FP64 | SUB_MIXED | SUB_FP64_STRICT                    */
  int32_t reserved0;   /* must be 0                                                 */
  double conv_rtol;    /* also stop when max_k |dS_n|/S_n <= conv_rtol; 0 = off     */
  uint64_t hbm_budget; /* bytes of device memory the context may hold; 0 = no cap   */
} sub_params;

/* Result summary of sub_run. */
typedef struct {
  int32_t iterations;     /* loop iterations executed (the last one found no source) */
  int32_t converged;      /* 1 if the loop stopped because nothing crossed rho_th    */
  int64_t n_sources;      /* N_b of the loaded catalog                               */
  int64_t n_candidates;   /* sources with rho_0 >= kappa rho_th                      */
  int64_t n_resolved;     /* sources removed                                         */
  int64_t n_bins;         /* bins in the band                                        */
  int64_t k_lo;           /* DFT index of the first bin: f = (k_lo + j) / T_obs       */
  int32_t status;         /* return code of the run                                  */
  int32_t reserved;
  int64_t n_live;         /* candidates that can still be resolved: rho_0 > rho_th   */
                          /* (rho <= rho_0 because S_n >= S_instr; the others are    */
                          /* never tested again)                                     */
  int64_t n_exact;        /* SNR decisions recomputed in FP64 (SUB_FP64)             */
  int64_t n_near;         /* SNR decisions taken in FP64 (SUB_FP64, SUB_FP64_STRICT) */
                          /* on a rho with |rho - rho_th| / rho_th < 1e-9, counted   */
                          /* over (candidate, iteration): the decisions that FP64    */
                          /* rounding order alone could flip.  0 in SUB_MIXED.       */
  int64_t n_uncertain;    /* SUB_MIXED: FP32 decisions whose value lies inside the   */
                          /* FP32 screen's error bound around rho_th^2 (FP64 could   */
                          /* decide them differently).  0 in the FP64 modes.         */
} sub_stats;

typedef struct sub_ctx sub_ctx;

/* Fill *p with the paper's defaults: T_obs = 4 yr, band [1e-4, 1e-2] Hz,
 * window 2000, running mean, rho_th = 7, kappa = 1/7, max_iter = 100, TDI-2 on,
 * FP64, no rtol, no budget.  Returns SUB_EINVAL if p is null. */
int sub_params_default(sub_params* p);

/* Create a context: validates *p, builds the grid k_lo .. k_hi
 * (k_lo = ceil(f_min T), k_hi = floor(f_max T)) and the per-bin tables
 * S_instr(f_k) and R(f_k) (App. B, App. C) on the device.
 *   p      : parameters, copied.
 *   stream : cudaStream_t to issue work on, or NULL for a stream the context owns.
 *   out    : receives the context; *out is NULL on failure.
 * Errors: SUB_EINVAL (bad parameters), SUB_ENOMEM, SUB_ECUDA, SUB_EBUDGET. */
int sub_create(const sub_params* p, void* stream, sub_ctx** out);

/* Load a catalog of n sources into the context (SoA, FP64, n >= 0).
 *   A    : strain amplitudes (>= 0), Eq. (GB waveform).
 *   f    : frequencies in Hz at t = 0, Eq. (phase Taylor expansion).
 *   fdot : frequency derivatives in Hz/s (either sign).
 *   where: for all three arrays:
 *          SUB_HOST, SUB_DEVICE: the arrays are copied on the context's stream; page-locked
 *            or device arrays stay unchanged until the stream has passed the copies (a
 *            sub_run that waits, or a stream synchronisation);
 *          SUB_HOST_MAPPED: page-locked host memory (cudaHostAlloc, cudaHostRegister or a
 *            pinned tensor) that every later sub_run reads in place; nothing is copied, and
 *            the caller keeps the arrays alive and unchanged until the next load or
 *            sub_destroy.  Memory that is not page-locked: SUB_EINVAL.
 * Replaces any previous catalog.  Errors: SUB_EINVAL, SUB_ENOMEM, SUB_EBUDGET,
 * SUB_ECUDA. */
int sub_load_catalog(sub_ctx* ctx, const double* A, const double* f, const double* fdot,
                     int64_t n, int where);

/* Generate a catalog on the device instead of loading one (the synthetic population model:
 * f from a power law p(f) ~ f^-gamma on [0.1, 10] mHz, A = 1e-23 X (f / 1 mHz)^(2/3) with
 * X ~ Gamma(shape, 1), fdot the GW-driven chirp of Sec. II.A with Mc ~ U(0.2, 0.8) Msun).
 * Source s is a pure function of (seed, s): a counter-based Philox4x32-10 stream, and
 * single-precision arithmetic of basic operations only, so the same catalog comes out on
 * any machine; it is returned in FP64.
 *   n     : sources (0 .. 2^40);  seed: any 64-bit value
 *   gamma : power-law index, -8 .. 10;  shape: Gamma shape of the amplitude factor, 1 .. 1e6
 *   fused : nonzero: nothing is stored; every sub_run generates each source inside the
 *           catalog pass, so no catalog crosses the host link or sits in device memory;
 *           zero: the catalog is generated once into the context's catalog arrays and runs
 *           read it like a loaded catalog.
 * Replaces any previous catalog.  Errors: SUB_EINVAL, SUB_ENOMEM, SUB_EBUDGET, SUB_ECUDA. */
int sub_load_generated(sub_ctx* ctx, int64_t n, uint64_t seed, double gamma, double shape,
                       int32_t fused);

/* Population parameters of the paper's model (Sec. II.B "Population model", Table I; the
 * number of binaries N_b is the n argument of the calls that take one). */
typedef struct {
  double alpha_pl;  /* power-law index: p(f) ~ f^alpha_pl on [0.1, 10] mHz; prior U(-4, -2)   */
  double alpha_g;   /* Gamma concentration of xi = log10(fdot / Hz s^-1) - mu_g; U(1, 3)       */
  double beta_g;    /* Gamma rate of xi; U(1, 3)                                              */
  double mu_g;      /* offset of log10 fdot; U(-22, -20)                                      */
  double mu;        /* log10((f/Hz)^(-2/3) A) - mu is log-normal; U(-23, -21)                  */
  double sigma;     /* width of that log-normal; U(0.1, 0.3)                                  */
  double rho;       /* Gaussian-copula correlation of f and fdot (App. A), 0 <= rho < 1; U(0, 1) */
} sub_population;

/* Generate a catalog of the paper's population model on the device instead of loading one:
 * f, xi and the rescaled amplitude from their marginals (power law, Gamma, log-normal) with
 * f and xi tied by the Gaussian copula of App. A (sampled by conditioning: xi from its
 * marginal, its CDF value as a normal z2, then z1 = rho z2 + sqrt(1 - rho^2) n and f from the
 * power law at Phi(z1)); fdot = 10^(mu_g + xi), A = f^(2/3) 10^(mu + rescaled amplitude).
 * Source s is a pure function of (seed, s) in single-precision arithmetic of basic
 * operations, as for sub_load_generated.
 *   n, seed, fused : as sub_load_generated;  pop : the parameters above (copied)
 * Errors: SUB_EINVAL (a parameter outside the ranges in sub_last_error), SUB_ENOMEM,
 * SUB_EBUDGET, SUB_ECUDA. */
int sub_load_population(sub_ctx* ctx, int64_t n, uint64_t seed, const sub_population* pop,
                        int32_t fused);

/* Sources start .. start+n-1 of the current catalog into A, f, fdot (n doubles each, at
 * `where`): copied from where the catalog lives, or generated again for a fused generated
 * catalog.  Synchronises.  Errors: SUB_EINVAL, SUB_ESTATE (no catalog), SUB_ECUDA. */
int sub_get_catalog(sub_ctx* ctx, double* A, double* f, double* fdot, int64_t start, int64_t n,
                    int where);

/* Run the subtraction of App. D on the loaded catalog:
 *   rho_0 against S_instr; candidates rho_0 >= kappa rho_th; then repeat
 *   { S_gal = estimator of the residual power; rho against S_instr + S_gal;
 *     resolve every candidate with rho > rho_th } until none is resolved.
 * The loop runs on the device.  If stats is non-null the call waits for the
 * result and fills it; otherwise it returns after enqueueing.
 * Returns SUB_OK, SUB_ENOTCONVERGED (results valid), SUB_ERANGE, SUB_ESTATE,
 * SUB_ECUDA. */
int sub_run(sub_ctx* ctx, sub_stats* stats);

/* Wait for the last sub_run and fill *stats (also returns its status). */
int sub_get_stats(sub_ctx* ctx, sub_stats* stats);

/* Number of sources resolved in each iteration of the last run: hist[i] for
 * iteration i+1, for min(cap, iterations) entries; returns that count (or a
 * negative error code).  Synchronises. */
int sub_get_history(sub_ctx* ctx, int32_t* hist, int32_t cap);

/* Copy S_gal(f_k), k = k_lo .. k_hi, into S_gal (cap doubles at least n_bins).
 * n_bins and k_lo may be null.  where: SUB_HOST or SUB_DEVICE.
 * Errors: SUB_EINVAL (cap too small), SUB_ESTATE (no run yet), SUB_ECUDA. */
int sub_get_spectrum(sub_ctx* ctx, double* S_gal, int64_t cap, int64_t* n_bins, int64_t* k_lo,
                     int where);

/* Copy the resolved mask in catalog order (1 = resolved) into mask[0 .. n).
 * n must equal the catalog size.  where: SUB_HOST or SUB_DEVICE. */
int sub_get_resolved_mask(sub_ctx* ctx, uint8_t* mask, int64_t n, int where);

/* Apply the context's running estimator (window, estimator) to a given spectrum:
 * out = est_W(P) over the n_bins bins of the band, as in Eqs. (running mean) /
 * (running median) of App. D without S_instr; App. E applies the estimators to
 * the residual data in this way.  P and out hold n doubles (n must equal
 * n_bins; P >= 0) in `where` memory; they may not overlap.
 * Errors: SUB_EINVAL, SUB_ECUDA.  Synchronises before returning. */
int sub_estimate(sub_ctx* ctx, const double* P, double* out, int64_t n, int where);

/* Copy the residual power spectrum P_k of the sources not resolved so far
 * (after a run: the residual the final S_gal was estimated from), the one-sided
 * A-channel periodogram level of App. D, into P (n_bins doubles).  P_k is
 * evaluated from the run's exact fixed-point spectrum.  where: SUB_HOST or
 * SUB_DEVICE.  Errors: SUB_EINVAL, SUB_ESTATE (no run yet), SUB_ECUDA. */
int sub_get_power(sub_ctx* ctx, double* P, int64_t n, int where);

/* Copy the per-bin tables S_instr(f_k) (App. C, A channel, times the TDI-2
 * factor when tdi2) and R(f_k) (App. B, same factor) into S and R (n_bins
 * doubles each; either may be null).  where: SUB_HOST or SUB_DEVICE. */
int sub_get_tables(sub_ctx* ctx, double* S, double* R, int64_t n, int where);

/* Device time of the last sub_run split at the end of the catalog pass:
 * prepass_ms (clear + pass over the catalog), loop_ms (all iterations) and
 * total_ms, from CUDA events recorded inside the run's graph.  Synchronises.
 * Any pointer may be null. */
int sub_get_timing(sub_ctx* ctx, float* prepass_ms, float* loop_ms, float* total_ms);

/* Coarse graining (Sec. "Coarse-graining of the data", the bin-averaged spectrum and the
 * bin-averaged frequencies): the band [f_min, f_max] is split into nbins logarithmically
 * spaced bins with edges e_k = 10^(log10 f_min + k (log10 f_max - log10 f_min) / nbins); a
 * grid frequency f_i = (k_lo + i) / T_obs belongs to the highest bin whose lower edge is
 * at most f_i (bin 0 also takes the grid frequencies below e_1).
 *   x         : n_bins values on the grid (host or device per `where`), or null for the
 *               S_gal of the last sub_run (SUB_ESTATE before any run)
 *   add_instr : nonzero to average S_instr + x (the noise PSD S_n) instead of x
 *   nbins     : 1 .. 2^20 (the paper: 100)
 *   S_out[k]  : mean of the series over bin k;  f_out[k]: mean frequency of bin k;
 *   count_out[k]: N_k, the grid frequencies in bin k.  An empty bin gives NaN means.
 *               Any output may be null; all are nbins long, at `where`.
 * Synchronises.  Errors: SUB_EINVAL, SUB_ESTATE, SUB_ENOMEM, SUB_EBUDGET, SUB_ECUDA. */
int sub_coarse_grain(sub_ctx* ctx, const double* x, int32_t add_instr, int32_t nbins,
                     double* S_out, double* f_out, int64_t* count_out, int where);

/* Work items the loop kernels of the last sub_run were handed, summed over its
 * iterations: work[0] chunks (Kc bins each) whose values changed, work[1] chunks within
 * one chunk of such a chunk, work[2] within two, work[3] median tiles (Kc outputs each).
 * Which kernel takes which list depends on the estimator: median-then-mean sorts 0,
 * selects medians on 3, sums prefixes on 1 and window means on 2; median sorts 0 and
 * selects on 3; mean sums prefixes on 0 and window means on 1.  Writes min(n, 4) entries.
 * Synchronises. */
int sub_get_work(sub_ctx* ctx, int64_t* work, int32_t n);

/* Kernels of the path, in the order of SUB_K_* below. */
#define SUB_K_PREPASS 0   /* catalog pass: sweep, deposit, rho_0, candidates  */
#define SUB_K_SORT 1      /* per-chunk sort (median)                           */
#define SUB_K_MEDIAN 2    /* running median (merged ranks, wavelet selection)  */
#define SUB_K_PREFIX 3    /* exact per-chunk prefix sums (mean)                */
#define SUB_K_MEAN 4      /* window means                                      */
#define SUB_K_SNR 5       /* SNR, threshold, removal                           */
#define SUB_K_CONTROL 6   /* loop control                                      */
#define SUB_K_COUNT 7

/* Run the loaded catalog once more with the same kernels launched one by one
 * from the host (no graph), recording a CUDA event pair around every launch;
 * ms[k] receives the summed device time and launches[k] the launch count of
 * kernel k (SUB_K_*).  Results and stats are those of a normal run.  Meant
 * for measurement, not for throughput.  Synchronises. */
int sub_profile(sub_ctx* ctx, float ms[SUB_K_COUNT], int32_t launches[SUB_K_COUNT],
                sub_stats* stats);

/* Both evaluations of rho^2 (Eqs. SNR inner product / inner product; App. D) for every kept
 * candidate (rho_0 > rho_th, see sub_stats.n_live) against the S_gal of the last run, for
 * measuring the FP32 screen that SUB_FP64 decides on first:
 *   src[i]         : the candidate's index in the catalog
 *   rho2_screen[i] : rho^2 in FP32 as the screen evaluates it (through 1 / (1 + S_gal/S_instr)
 *                    of the last estimate, in FP32), summed bin by bin on one thread
 *   rho2_exact[i]  : rho^2 in FP64, summed in the oracle's order (the value SUB_FP64 decides
 *                    on when the screen cannot; for a sweep of more than 4 bins the run sums
 *                    it across a warp, which differs by rounding only)
 *   nbins[i]       : bins of the band the screen summed (the error bound of this one-thread
 *                    sum grows with them)
 * All four are host arrays of cap entries; *n_out (may be null) receives the count.  The
 * call allocates and frees a temporary device buffer of 24 bytes per candidate and
 * synchronises.  Errors: SUB_EINVAL (cap below the count, null output), SUB_ESTATE (no run
 * yet), SUB_ENOMEM, SUB_EBUDGET, SUB_ECUDA. */
int sub_snr_check(sub_ctx* ctx, int64_t* src, float* rho2_screen, double* rho2_exact,
                  int32_t* nbins, int64_t cap, int64_t* n_out);

/* The last sub_profile's device time per loop iteration and kernel: ms[i * SUB_K_COUNT + k]
 * for iteration i + 1 (the catalog pass is not included) and kernel k, for min(cap,
 * iterations) iterations.  Returns the number of iterations profiled (0 before any
 * sub_profile), or SUB_EINVAL. */
int sub_get_profile_iterations(sub_ctx* ctx, float* ms, int32_t cap);

/* Largest inputs of sub_running_mean_noalloc (the size of its static scratch). */
#define SUB_NOALLOC_MAX_BINS 1310720
#define SUB_NOALLOC_MAX_WINDOW 8192

/* Running mean of a caller's spectrum without any device allocation.  The paper
 * has no counterpart to this call; it serves callers that cannot allocate device
 * memory, e.g. a plug-in handed device buffers by a host framework that owns all
 * device memory, or a latency-critical loop that must not enter cudaMalloc (which
 * can synchronise the device and can fail at run time).
 *   x, out : device pointers to n doubles (x >= 0), owned by the caller; they may
 *            not overlap.  out[j] = mean of x over [j - W/2, j - W/2 + W - 1]
 *            cut to [0, n), the same values as sub_estimate with SUB_MEAN.
 *   n      : 1 .. SUB_NOALLOC_MAX_BINS;  window: 1 .. SUB_NOALLOC_MAX_WINDOW.
 *   stream : cudaStream_t to run on (NULL: the legacy default stream).  The call
 *            returns after enqueueing.
 * Scratch lives in one static device array of about 21 MB that every GPU loading
 * the library holds until the process exits.  Every call asks the runtime for the
 * array's address on the current device; the first call on a device loads the module
 * there (which may allocate), so make it before any stream capture and before any
 * phase that must not allocate.  All calls share the array and it keeps the last call's
 * contents: calls that overlap on the GPU race and must be serialised by the caller.  Sizes beyond the limits return SUB_EINVAL with a message in
 * sub_last_error(NULL); CUDA failures return SUB_ECUDA. */
int sub_running_mean_noalloc(const double* x, double* out, int64_t n, int32_t window,
                             void* stream);

/* Bytes of device memory the context holds now. */
int64_t sub_device_bytes(const sub_ctx* ctx);

/* ------------------------------------------------------------------ batches
 * Many catalogs in one launch.  The per-iteration kernels of a single catalog leave most
 * of the GPU idle (only the few chunks that changed are recomputed), so a batch launches
 * every context's whole run (catalog pass and device loop, App. D) as independent
 * branches of one CUDA graph; their kernels overlap on the SMs.  Results are the same
 * bits as each context run alone.
 *   ctxs : n >= 1 distinct contexts on one device, each with its own parameters
 *          (T_obs, window, estimator, precision ...) and, before sub_batch_run, a catalog.
 *          The batch borrows them: destroy the batch before any of its contexts.
 * The graph is built on the first run and rebuilt when a context's catalog size changes.
 * Errors: SUB_EINVAL (bad list; message in sub_last_error(NULL)), SUB_ECUDA. */
typedef struct sub_batch sub_batch;
int sub_batch_create(sub_ctx* const* ctxs, int32_t n, sub_batch** out);

/* Run the batch and wait for it.  stats (may be null) receives n sub_stats, in the order
 * of ctxs; each context's results are then read with sub_get_spectrum etc.  Returns
 * SUB_OK, SUB_ENOTCONVERGED if any context stopped at max_iter, or the first error. */
int sub_batch_run(sub_batch* b, sub_stats* stats);

/* Device time of the last sub_batch_run, in milliseconds (CUDA events around the launch). */
float sub_batch_last_ms(const sub_batch* b);

/* Reason for the last failure of a call on b; never null. */
const char* sub_batch_last_error(const sub_batch* b);

/* Free the batch (its contexts stay). */
void sub_batch_destroy(sub_batch* b);

/* Run the context's chunk kernels, catalog pass and SNR on persistent grids of 1/div of
 * the GPU's resident CTAs (div in 1 .. 64; 1 = the whole GPU, the default).  Smaller grids
 * suit batches, where many catalogs share the GPU; results do not depend on div.
 * Errors: SUB_EINVAL. */
int sub_set_grid_div(sub_ctx* ctx, int32_t div);

/* Launch settings that leave every result unchanged bit for bit (for autotuners):
 *   SUB_TUNE_GRID_DIV       persistent grids at 1/value of the GPU (1 .. 64), as
 *                           sub_set_grid_div
 *   SUB_TUNE_SORT_E         elements per thread of the chunk sort: 2, 4 or 8 with
 *                           kpad / value in 32 .. 1024 (kpad: the power of two >= the chunk
 *                           length), or 0 for the automatic choice
 *   SUB_TUNE_MEDIAN_THREADS threads per median tile: a multiple of 32 up to 512, or 0
 * The context's graph is rebuilt by its next run.  Errors: SUB_EINVAL. */
#define SUB_TUNE_GRID_DIV 0
#define SUB_TUNE_SORT_E 1
#define SUB_TUNE_MEDIAN_THREADS 2
int sub_set_tuning(sub_ctx* ctx, int32_t knob, int32_t value);

/* Test hooks: failures made on purpose, for tests of the error paths.  The catalog pass
 * waits on its staged copies with a bound of about a second; with
 * SUB_TEST_SKIP_CATALOG_COPIES it starts none, every wait runs out, the loop stops and
 * sub_run returns SUB_ETIMEOUT.  The context stays usable: clear the flag (0) and run
 * again.  Errors: SUB_EINVAL for unknown flags. */
#define SUB_TEST_SKIP_CATALOG_COPIES 1
int sub_test_hooks(sub_ctx* ctx, int32_t flags);

/* ------------------------------------------------------------------ serving
 * A request loop for subtraction jobs as a sampler emits them.  Jobs are queued in
 * arrival order and admitted while fewer than max_inflight run and a device-memory budget
 * allows; when the job at the head has to wait, a later job that an idle pooled context can
 * take is admitted past it (it takes nothing the head could use).  Each admitted job runs
 * on a pooled context (one per T_obs and catalog size
 * class, created on demand, the least recently used idle ones destroyed when the budget
 * needs room) on its own stream, so jobs overlap on the GPU (continuous batching).  A
 * job's latency runs from sub_server_submit to its results being in the caller's
 * buffers.  All jobs of a server share the parameters below; T_obs is per job. */
typedef struct {
  uint64_t hbm_budget;   /* bytes of device memory for all contexts; 0 = unlimited     */
  int32_t max_inflight;  /* jobs on the GPU at once, 1 .. 256 (default 16)             */
  int32_t window;        /* as sub_params                                              */
  int32_t estimator;
  int32_t precision;
  int32_t max_iter;
  int32_t tdi2;
  int32_t grid_div;      /* persistent-grid divisor of every context (sub_set_grid_div) */
  int32_t max_contexts;  /* pooled contexts at most (0 = as many as the budget allows); at
                          * the limit a job that a busy context could take waits for it,
                          * and only a job that none could take replaces an idle context
                          * (allocation and freeing synchronise the GPU) */
  double f_min, f_max;
  double rho_th, kappa;
} sub_server_params;

typedef struct {
  int64_t job_id;
  int32_t status;        /* SUB_OK, SUB_ENOTCONVERGED, or the error that ended the job  */
  int32_t reserved;
  sub_stats stats;
  double latency_ms;     /* submit -> results in the caller's buffers                  */
  double queue_ms;       /* submit -> admitted                                          */
  double gpu_ms;         /* device time of the run (catalog pass + loop)                */
} sub_job_result;

typedef struct {
  int64_t queued;
  int64_t contexts_created;
  int64_t device_bytes;       /* held by the pooled contexts now */
  int64_t peak_device_bytes;
  int32_t inflight;
  int32_t contexts;
} sub_server_stats;

int sub_server_params_default(sub_server_params* p);

/* Start a server (a worker thread on the current device).  Errors: SUB_EINVAL, SUB_ECUDA. */
typedef struct sub_server sub_server;
int sub_server_create(const sub_server_params* p, sub_server** out);

/* Queue a job and return at once.  A, f, fdot: host arrays of n sources (pinned memory
 * makes the copies asynchronous); S_gal: host buffer of cap >= n_bins(T_obs) doubles, or
 * null; mask: host buffer of n bytes (1 = resolved), or null.  Results go straight into
 * page-locked buffers; pageable ones receive them from page-locked staging when the job
 * completes (one host copy more).  All must stay valid and
 * untouched until the job's result comes out of sub_server_poll.  A job larger than the
 * whole budget ends with SUB_EBUDGET.  Errors: SUB_EINVAL, SUB_ESTATE (server stopping). */
int sub_server_submit(sub_server* s, int64_t job_id, double T_obs, const double* A,
                      const double* f, const double* fdot, int64_t n, double* S_gal,
                      int64_t cap, uint8_t* mask);

/* Queue a job whose catalog is drawn on the device (sub_load_generated, fused): n sources
 * of the population (gamma, shape) with this seed, so no catalog crosses the host link.
 * S_gal and mask as for sub_server_submit.  Errors: SUB_EINVAL, SUB_ESTATE. */
int sub_server_submit_generated(sub_server* s, int64_t job_id, double T_obs, int64_t n,
                                uint64_t seed, double gamma, double shape, double* S_gal,
                                int64_t cap, uint8_t* mask);

/* Queue a job whose catalog of n sources is drawn on the device from the paper's population
 * model (sub_load_population, fused) with parameters pop (copied) and this seed.  S_gal and
 * mask as for sub_server_submit.  Errors: SUB_EINVAL, SUB_ESTATE. */
int sub_server_submit_population(sub_server* s, int64_t job_id, double T_obs, int64_t n,
                                 uint64_t seed, const sub_population* pop, double* S_gal,
                                 int64_t cap, uint8_t* mask);

/* Move up to cap finished jobs into out, waiting up to timeout_ms for the first one
 * (0: no wait).  Returns how many were written. */
int32_t sub_server_poll(sub_server* s, sub_job_result* out, int32_t cap, int32_t timeout_ms);

/* Create `count` idle contexts for T_obs with room for catalogs of up to n_sources and their
 * graphs built, before traffic arrives (context creation allocates device memory and
 * builds tables and graphs: milliseconds that would otherwise land on the first jobs).
 * Only while no job is queued or running.  Errors: SUB_EINVAL, SUB_ESTATE, SUB_EBUDGET. */
int sub_server_prewarm(sub_server* s, double T_obs, int64_t n_sources, int32_t count);

/* Queue, in-flight and memory counters. */
int sub_server_info(sub_server* s, sub_server_stats* st);

/* Reason for the last rejected submission; never null. */
const char* sub_server_last_error(sub_server* s);

/* Stop: jobs not yet admitted are dropped, running ones finish; then every context is
 * freed. */
void sub_server_destroy(sub_server* s);

/* Free the context and everything it owns; null is allowed. */
void sub_destroy(sub_ctx* ctx);

/* Reason for the last failure of a call on ctx (or of sub_create when ctx is
 * null); never null. */
const char* sub_last_error(const sub_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GBSUB_H */
