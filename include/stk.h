/*
 * stk.h - C ABI of the B300 scorer for all-sky seedless clustering
 * (Thrane & Coughlin, "Seedless clustering in all-sky searches for
 * gravitational-wave transients").
 *
 * The library scores many pseudo-random quadratic Bezier templates, each with a
 * random inter-detector delay tau, against a complex cross-power SNR map and
 * returns the loudest templates.  All arithmetic runs in CUDA kernels on one
 * GPU; the host side only validates arguments, sizes buffers and launches.
 *
 * Conventions
 *   - Every int-returning call returns STK_OK (0) or a negative STK_E* code;
 *     stk_last_error() then holds a one-line message.
 *   - Calls are asynchronous on the context's CUDA stream unless they return
 *     host data (stk_score with STK_OUT_HOST, stk_track_params, stk_load_map,
 *     stk_sync).  The stream is borrowed: the caller keeps ownership.
 *   - Device pointers passed in stay owned by the caller; buffers the library
 *     allocates (packed maps, scratch) are owned by the map or context and are
 *     freed by stk_free_map / stk_destroy.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Template index g runs over counter_offset .. counter_offset + n_tracks-1;
 *     template g is the same on every call, any split of the index range, and
 *     any GPU, so runs over disjoint ranges combine exactly by taking the
 *     largest SNR (Sec. V, "intermediate data files").
 */
#ifndef STK_H
#define STK_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define STK_API __attribute__((visibility("default")))
#else
#define STK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define STK_OK        0
#define STK_EINVAL   -1  /* bad argument: sizes, pointers, flags, non-finite or non-positive inputs */
#define STK_ENOMEM   -2  /* device or host allocation failed */
#define STK_ECUDA    -3  /* a CUDA runtime call failed (message names it) */
#define STK_ETIMEOUT -4  /* a bounded in-kernel wait gave up; results of that call are invalid */
#define STK_ESTATE   -5  /* call out of order, e.g. scoring before stk_set_tracks */
#define STK_EBOUNDS  -7  /* debug build (libstk_debug.so) only: a pixel gather outside its template's
                            bins or the map, or a damaged canary word after a buffer */

/* ---- stk_load_map flags ---------------------------------------------- */
#define STK_HOST_PTR       0x1u /* y and sigma are host pointers (pageable or pinned) */
#define STK_SIGMA_PER_FREQ 0x2u /* sigma holds n_f values, one per frequency bin, constant in time */
#define STK_NORM_PAPER     0x4u /* Eq. 7 as printed: SNR = (1/N) sum Re[e^{2 pi i f tau} y/sigma] */
#define STK_FP16           0x8u /* store each pixel in 4 bytes: |y|/sigma in FP16 (per-frequency or per-pixel
                                   scaling by sigma) and the phase in 1/65536 turns; sums stay FP32 */

/* ---- stk_score flags ------------------------------------------------- */
#define STK_OUT_HOST 0x1u /* out_topk is host memory; the call waits for the result */

/* Largest k accepted by stk_score. */
#define STK_MAX_K 4096

typedef struct stk_ctx stk_ctx; /* opaque; owns scratch and the borrowed stream */
typedef struct stk_map stk_map; /* opaque; the packed map on the device */

/* One selected template.  40 bytes, no padding surprises. */
typedef struct {
    double   snr;      /* detection statistic of the template (see stk_load_map) */
    uint64_t index;    /* template index g */
    uint32_t f[3];     /* control frequency bins f0 (first column), f1 (middle control), f2 (last column) */
    uint32_t reserved; /* zero */
    double   tau;      /* delay in seconds, |tau| < tau_max */
} stk_hit;

/* Library version, 10000*major + 100*minor + patch. */
STK_API int stk_version(void);

/* Build flags of the loaded library: bit 0 set in the debug build (libstk_debug.so,
 * compiled with STK_DEBUG_BOUNDS): every pixel gather checks its column and bin
 * against the template's convex hull of control bins within the map and reports
 * STK_EBOUNDS at the next deferred-error check instead of reading out of range;
 * the packed map and the context's scratch carry trailing canary words, checked
 * (synchronising) after every scoring, refinement and batch call.  0 otherwise. */
STK_API int stk_build_flags(void);

/* Create a context on CUDA device `device`, issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * context.  Errors: STK_EINVAL (out NULL, device out of range), STK_ECUDA. */
STK_API int stk_create(stk_ctx **out, int device, void *cuda_stream);

/* Free the context and its scratch after the stream has finished with them.
 * NULL is a no-op.  Maps created through it must be freed first. */
STK_API void stk_destroy(stk_ctx *ctx);

/* Change the stream later calls are issued on (borrowed, not owned). */
STK_API int stk_set_stream(stk_ctx *ctx, void *cuda_stream);

/* Copy and pack an ft-map (Eq. 6: the complex SNR map p(t; f), here given as
 * a cross-power y with per-pixel standard deviation sigma, Appendix A).
 *   y_c64   complex64 [n_t][n_f], time-major (frequency fastest), interleaved re, im
 *   sigma   float32 [n_t][n_f], or [n_f] with STK_SIGMA_PER_FREQ; every value > 0; +infinity
 *           marks a notched pixel (the black lines of Fig. 1's caption): it adds nothing to
 *           either sum (z = 0, w = 0, whatever y holds there); the paper form keeps n_t; a
 *           template with no un-notched pixel scores 0
 *   n_t     time columns, >= 2 (a template has one pixel per column)
 *   n_f     frequency bins, >= 1; bin k has frequency f_min_hz + k * df_hz
 *   flags   STK_HOST_PTR | STK_SIGMA_PER_FREQ | STK_NORM_PAPER | STK_FP16
 * Statistic selected (Eq. 7 and the footnote to Eq. 5 allowing other weights):
 *   default         SNR = sum_j Re[e^{2 pi i f_j tau} y_j sigma_j^-2] / sqrt(sum_j sigma_j^-2)
 *   STK_NORM_PAPER  SNR = (1/n_t) sum_j Re[e^{2 pi i f_j tau} y_j / sigma_j]
 * Arithmetic: pixel magnitude and angle stored FP32 (FP16 and Q0.16 turns with
 * STK_FP16), sums and normalisation FP32 (square root and
 * division rounded to nearest); the SNR is reported widened to FP64.  The delay phase
 * f tau mod 1 is exact in 64-bit fixed point per template; per pixel it is a
 * 32-bit turn, within 3e-6 rad for n_f <= 8192 (2^-32 turn beyond).
 * The library keeps its own packed copy; the caller may free y and sigma when
 * the call returns (it synchronises the stream).  Errors: STK_EINVAL (sizes,
 * NULL pointers, a non-finite y at a pixel that is not notched, sigma <= 0 or NaN, f_min/df
 * non-finite or df <= 0, |y|/sigma above 65504 with STK_FP16), STK_ENOMEM, STK_ECUDA. */
STK_API int stk_load_map(stk_ctx *ctx, const void *y_c64, const float *sigma, int n_t, int n_f,
                 double f_min_hz, double df_hz, unsigned flags, stk_map **out);

/* Replace a map's data with new y and sigma of the same shape, statistic and
 * precision (flags must equal the map's, STK_HOST_PTR aside), packing into the
 * map's existing device buffers: nothing is allocated except, on the first
 * host-pointer update of a context, its staging buffers.  For streams of
 * same-sized maps (time windows, time shifts).  A map with varying weights or
 * STK_NORM_PAPER keeps its weighting and the call does not wait: host data is
 * copied on the context's stream (pageable buffers before the call returns;
 * pinned ones when the stream gets there, so leave them unchanged until the
 * next stk_sync or STK_OUT_HOST call), and invalid data (non-finite y, sigma
 * <= 0, FP16 overflow) is reported as STK_EINVAL by the next stk_sync or
 * STK_OUT_HOST scoring call.  A constant-weight map is re-examined, as by
 * stk_load_map, and the call synchronises.  Errors: STK_EINVAL (sizes, NULL
 * pointers, flags differing from the map's; invalid data of a constant-weight
 * map), STK_ECUDA; after an error the map's contents are undefined until an
 * update succeeds. */
STK_API int stk_update_map(stk_ctx *ctx, stk_map *map, const void *y_c64, const float *sigma, unsigned flags);

/* Free a packed map (waits for the context's stream).  NULL is a no-op. */
STK_API void stk_free_map(stk_map *map);

/* Report a map's shape and flags (STK_HOST_PTR cleared; any pointer may be NULL). */
STK_API int stk_map_info(const stk_map *map, int *n_t, int *n_f, unsigned *flags);

/* Set the template range scored by later calls (Sec. III: T templates drawn at
 * random, each with a delay uniform on (-tau_max, +tau_max)).
 *   n_tracks        T, >= 1
 *   seed            Philox key word; runs meant to be combined use different seeds (Sec. V)
 *   counter_offset  first template index g
 *   tau_max_s       >= 0, finite (the inter-site light travel time, ~10 ms for the LIGO pair)
 * Errors: STK_EINVAL. */
STK_API int stk_set_tracks(stk_ctx *ctx, uint64_t n_tracks, uint64_t seed, uint64_t counter_offset,
                   double tau_max_s);

/* Score every template of the current range against `map` and return the k
 * loudest (Sec. III: the most significant cluster; k > 1 keeps runners-up),
 * ordered by SNR descending, then index ascending.  `out_topk` holds k
 * entries: device memory, or host memory with STK_OUT_HOST (then the call
 * waits for the result).  k in 1 .. min(STK_MAX_K, n_tracks).
 * Errors: STK_EINVAL, STK_ESTATE (no range set), STK_ENOMEM, STK_ECUDA,
 * STK_ETIMEOUT (reported by a later stk_sync when the output is on the device). */
STK_API int stk_score(stk_ctx *ctx, const stk_map *map, int k, stk_hit *out_topk, unsigned flags);

/* Score every template of the current range and write its SNR (Eq. 7) to
 * out_snr_dev[i] for template counter_offset + i; caller-owned device buffer
 * of n_tracks doubles (the FP32 SNRs widened; 4 bytes per template of
 * context scratch).  Errors: STK_EINVAL, STK_ESTATE, STK_ENOMEM, STK_ECUDA. */
STK_API int stk_score_all(stk_ctx *ctx, const stk_map *map, double *out_snr_dev);

/* Parameters of template g as the scoring kernels draw them (Sec. III):
 * f[3] control bins, *tau delay, and, if bins_host is not NULL, the pixel
 * (frequency bin) of each of the map's n_t columns.  Uses the seed and
 * tau_max of the current range; g need not lie inside it.  Synchronous.
 * Errors: STK_EINVAL, STK_ESTATE, STK_ECUDA. */
STK_API int stk_track_params(stk_ctx *ctx, const stk_map *map, uint64_t g, uint32_t f[3], double *tau,
                     int32_t *bins_host);

/* Score n explicit templates (Eq. 7): f3_dev [n][3] control bins (each < n_f),
 * tau_dev [n] delays in seconds; SNRs to out_snr_dev [n].  All device
 * pointers, caller-owned (4 bytes per template of context scratch).  Bins
 * outside [0, n_f) are clamped to the map edge after the out-of-range
 * template is flagged: the call then returns STK_EINVAL at the next
 * stk_sync.  Errors: STK_EINVAL, STK_ENOMEM, STK_ECUDA. */
STK_API int stk_score_explicit(stk_ctx *ctx, const stk_map *map, const uint32_t *f3_dev, const double *tau_dev,
                       uint64_t n, double *out_snr_dev);

/* ---- general templates and delay priors ---------------------------------
 * Sec. III describes each template by three time-frequency control points
 * P0 (t_start, f_start), P1 (t_mid, f_mid), P2 (t_end, f_end) drawn from six
 * random numbers, the curve persisting at least t_min.  The default templates
 * pin the times to the first, middle and last column; general templates draw
 * integer times t0 <= t1 <= t2 as well: duration t2 - t0 uniform on
 * [t_min, n_t - 1], start uniform on [0, n_t - 1 - duration], t1 uniform on
 * [t0, t2] (Philox block (g, 1, 0, 0); bins and delay as before).  Column j of
 * [t0, t2] takes the bin nearest f(xi_j), t(xi_j) = j (halves up), decided
 * exactly in integer arithmetic; N = t2 - t0 + 1 pixels.  General templates
 * need n_t <= 4096 and n_f <= 8192 and are scored one thread per template
 * (not in batches).
 * Sec. VI suggests drawing the delay from a sky patch's distribution instead of
 * the isotropic uniform one: a delay prior is given as quantiles. */

/* general = 0: pinned times (default); general = 1: random times with
 * t2 - t0 >= t_min columns (t_min >= 1).  Applies to later scoring calls of
 * ctx.  Errors: STK_EINVAL. */
STK_API int stk_set_template_shape(stk_ctx *ctx, int general, int t_min);

/* Delay prior for later scoring calls: quantiles_host[i] is the delay (s) at
 * cumulative probability i / (n - 1), non-decreasing, n in 2 .. 65536; the delay
 * of template g is the linear interpolation at probability (u3 >> 11) 2^-53 of
 * its Philox word u3.  NULL or n = 0 restores the uniform prior on
 * (-tau_max, tau_max).  The table is copied.  Errors: STK_EINVAL, STK_ENOMEM. */
STK_API int stk_set_tau_prior(stk_ctx *ctx, const double *quantiles_host, int n);

/* Control times t[3] of template g under the current shape (0, (n_t-1)/2,
 * n_t - 1 for pinned templates).  Synchronous.  Errors: as stk_track_params. */
STK_API int stk_track_times(stk_ctx *ctx, const stk_map *map, uint64_t g, uint32_t t[3]);

/* Score n explicit general templates: t3_dev [n][3] control times (t0 <= t1 <=
 * t2 < n_t, t0 < t2), f3_dev [n][3] control bins (< n_f), tau_dev [n] delays;
 * SNRs to out_snr_dev [n]; device pointers (4 bytes per template of context
 * scratch).  Invalid templates are flagged (STK_EINVAL at the next stk_sync).
 * Errors: STK_EINVAL, STK_ENOMEM, STK_ECUDA. */
STK_API int stk_score_explicit_general(stk_ctx *ctx, const stk_map *map, const uint32_t *t3_dev,
                                       const uint32_t *f3_dev, const double *tau_dev, uint64_t n,
                                       double *out_snr_dev);

/* ---- continuous templates (refinement of the loudest) -------------------
 * The follow-up of the loudest events (Sec. V) refines a template's control
 * frequencies and delay continuously.  Control frequencies f0, f1, f2 are real
 * numbers in bins; column j of the curve sits at
 *   x_j = ((M-j)^2 f0 + 2 (M-j) j f1 + j^2 f2) / M^2   (clamped to [0, n_f - 1]),
 * the map is interpolated linearly in frequency between bins floor(x_j) and
 * floor(x_j) + 1, and the phase uses the continuous frequency f_min + x_j df:
 *   S = sum_j Re[exp(2 pi i (f_min + x_j df) tau) z(j, x_j)],  W = sum_j w(j, x_j),
 *   SNR = S / sqrt(W), or S / N with STK_NORM_PAPER (Eq. 7 at integer bins).
 * f3_dev: float [n][3]; tau_dev: float [n] seconds; device memory, caller-owned.
 * Arithmetic is FP32 except the curve position and phase (fixed point, Q32.32
 * bins and Q0.64 turns).  A template with a control frequency of magnitude
 * 2^29 bins or more, or a non-finite one or delay, gets NaN. */

/* snr_dev[i] = SNR of continuous template i (float [n]).  Errors: STK_EINVAL, STK_ECUDA. */
STK_API int stk_interp_forward(stk_ctx *ctx, const stk_map *map, const float *f3_dev, const float *tau_dev,
                               uint64_t n, float *snr_dev);

/* Adjoint of stk_interp_forward: for g_dev[i] = dL/dSNR_i writes
 * grad_f3_dev[i][q] = g_i dSNR_i/df_q and grad_tau_dev[i] = g_i dSNR_i/dtau
 * (zero contribution from columns clamped to the band edge; at bin knots the
 * statistic has a kink and the one-sided derivative from above is used).
 * Errors: STK_EINVAL, STK_ECUDA. */
STK_API int stk_interp_adjoint(stk_ctx *ctx, const stk_map *map, const float *f3_dev, const float *tau_dev,
                               const float *g_dev, uint64_t n, float *grad_f3_dev, float *grad_tau_dev);

/* Gradient ascent of n continuous templates' SNR (the follow-up of the loudest
 * events, Sec. V), all steps on the device.  Each step evaluates the SNR and its
 * gradient (stk_interp_adjoint with g = 1) and takes one Adam step (betas 0.9,
 * 0.999, eps 1e-8, bias-corrected) on the loss -SNR over (f0, f1, f2) in bins
 * (learning rate lr_bins) and u = tau / tau_max (learning rate lr_tau_frac),
 * then projects onto f in [0, n_f - 1] and |u| <= 1.  f3_dev float [n][3] and
 * tau_dev float [n] (seconds) are device memory, caller-owned, updated in place.
 * hist_dev (optional, NULL to skip): float [steps + 1][n] device memory, row t
 * the SNRs before step t + 1 (row steps: after the last step).  Context scratch:
 * 12 bytes per step.  One launch runs every step (each template's block loops
 * over the steps: the statistic, its gradient and the Adam step fused, the
 * parameters and moments in registers), after a host-to-device copy of the
 * steps' bias-corrected step sizes (computed in FP64 on the host).
 * Errors: STK_EINVAL (NULL pointer, steps < 0, tau_max <= 0, negative or
 * non-finite rates), STK_ENOMEM, STK_ECUDA. */
STK_API int stk_refine(stk_ctx *ctx, const stk_map *map, float *f3_dev, float *tau_dev, uint64_t n, int steps,
                       float lr_bins, float lr_tau_frac, float tau_max, float *hist_dev);

/* Discrete follow-up of the loudest templates (Sec. V): the refined templates
 * are judged by the discrete statistic of Eq. 7, so this call climbs it directly.
 * For each of n templates: the delay moves to the nearest maximum of SNR(tau)
 * at the template's fixed pixels (the weight sum does not depend on tau and
 * S(tau) is smooth: safeguarded Newton steps, each at most a tenth of the band's
 * shortest period and kept only when the SNR rises), then the control bins take
 * +-1 moves, each round the best of the six moves (its delay maximised again)
 * while it raises the SNR (the first in the order bin 0 -1, bin 0 +1, bin 1 -1,
 * ... among equals), at most `moves` rounds.  With alt_f3_dev / alt_tau_dev
 * (continuous templates, e.g. stk_refine's output; rounded to the nearest bins
 * and clamped, a NaN bin as 0 and a NaN delay as the start's) the alternative is
 * climbed too.  One block of twelve warps a template: six climb from the start
 * and six from the alternative, one move a warp.  The template kept is the start, the polished
 * start or the polished alternative, whichever scores highest by the scorer's
 * own arithmetic (the SNR stk_score_explicit returns; the start wins ties), so
 * no template leaves with a lower SNR than it came with.
 *   f3_dev     uint32 [n][3] control bins, tau_dev double [n] delays (s):
 *              device memory, caller-owned, updated in place
 *   tau_max    delays stay within [-tau_max, tau_max]
 *   snr_dev    double [n] (optional): the kept template's SNR
 *   which_dev  int [n] (optional): 0 start, 1 polished start, 2 polished alternative
 * Asynchronous on the context's stream; no allocation.  Errors: STK_EINVAL (NULL
 * pointer, tau_max <= 0, moves outside [0, 1024], only one of the alternatives),
 * STK_ECUDA. */
STK_API int stk_polish(stk_ctx *ctx, const stk_map *map, uint32_t *f3_dev, double *tau_dev, const float *alt_f3_dev,
                       const float *alt_tau_dev, uint64_t n, double tau_max, int moves, double *snr_dev,
                       int *which_dev);

/* Wait for the context's stream and report the first deferred error raised
 * by a kernel since the last stk_sync (bounded-wait timeout, bad explicit
 * template).  Clears it. */
STK_API int stk_sync(stk_ctx *ctx);

/* Turn per-kernel timing on (1) or off (0).  When on, every scoring and
 * selection kernel is bracketed with CUDA events on the context's stream. */
STK_API int stk_set_profiling(stk_ctx *ctx, int enable);

/* Per-kernel device time of the last stk_score / stk_score_all call, in ms:
 * out[0] scoring kernel, out[1] selection (all top-k kernels), out[2] launch
 * count of that call, out[3] coherent-order pre-pass (0 when not used).
 * Requires profiling on; synchronises the stream. */
STK_API int stk_last_timings(stk_ctx *ctx, double out[4]);

/* ---- many maps in one launch --------------------------------------------
 * A search records the loudest SNR of every map (Sec. V: year-long runs cut
 * into maps, and unphysical time shifts n_ts of each map for the background;
 * Eqs. 9-10 count that work).  A batch scores many maps of uneven size with
 * one persistent kernel: CTAs take (map, template block) tiles from a work
 * counter, largest maps first, stream each tile's map through shared memory,
 * and keep every tile's k loudest; a second kernel merges each map's tiles.
 * The launch sequence is recorded once in a CUDA graph and replayed. */
typedef struct stk_batch stk_batch; /* opaque */

#define STK_ECANCELED -6           /* a batch call was cancelled through stk_batch_cancel */
#define STK_BATCH_MAX_K 32         /* largest k per map in stk_batch_score */

/* Group n_maps maps (loaded on ctx; keep them alive while the batch exists)
 * with per-map template ranges: map i scores templates offsets[i] ..
 * offsets[i] + n_tracks[i] - 1 drawn with seeds[i] (n_tracks[i] in 1 .. 2^32-1),
 * all with delays uniform in (-tau_max_s, tau_max_s).  All maps must share the
 * statistic (weighted or STK_NORM_PAPER), the storage precision and the
 * weighting pattern, and satisfy (n_t - 1)^2 (2 n_f - 1) < 2^32 and n_f <= 8192
 * (the pixel phase is then kept as a 32-bit turn per bin, exact at the centre
 * bin and within 3e-6 rad elsewhere).
 * Errors: STK_EINVAL, STK_ENOMEM, STK_ECUDA. */
STK_API int stk_batch_create(stk_ctx *ctx, const stk_map *const *maps, int n_maps, const uint64_t *n_tracks,
                             const uint64_t *seeds, const uint64_t *offsets, double tau_max_s, stk_batch **out);

/* Free a batch (waits for the context's stream).  NULL is a no-op. */
STK_API void stk_batch_destroy(stk_batch *batch);

/* Score every template of every map and write map i's k loudest (SNR
 * descending, then index ascending) to out[i*k .. i*k + k - 1]; out is device
 * memory, or host memory with STK_OUT_HOST (the call then waits and returns
 * the batch's status).  k in 1 .. STK_BATCH_MAX_K and <= every n_tracks[i].
 * Errors: STK_EINVAL, STK_ENOMEM, STK_ECUDA; STK_ECANCELED or STK_ETIMEOUT
 * (from this call with STK_OUT_HOST, else from the next stk_sync). */
STK_API int stk_batch_score(stk_batch *batch, int k, stk_hit *out, unsigned flags);

/* Set (on != 0) or clear the batch's cancel flag.  It lives in host memory the
 * GPU reads: the persistent kernel checks it before taking each tile, so a
 * running stk_batch_score stops within one tile and reports STK_ECANCELED.
 * The flag stays set until cleared. */
STK_API int stk_batch_cancel(stk_batch *batch, int on);

/* Autotuner: time every candidate launch shape (512/768/1024 threads with 2..5
 * templates per thread, or 512 threads with 6, 8, 10 or 11; 2 or 3 slab
 * buffers: 32 shapes) on a sample of this batch's tiles and keep the fastest
 * for later stk_batch_score calls.  out (may be NULL) receives
 * {threads, templates per thread, slab buffers, sample time in ns}.
 * Errors: STK_EINVAL, STK_ECUDA. */
STK_API int stk_batch_tune(stk_batch *batch, int k, int64_t out[4]);

/* ---- scoring without allocation ------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot call cudaMalloc when they score: code whose device memory belongs to
 * another allocator (a framework's caching allocator, a fixed memory budget)
 * where an extra allocation may fail or fragment, and latency-critical loops
 * that cannot take the device-wide synchronisation of cudaFree.
 *
 * stk_score_noalloc computes exactly what stk_score computes for the range
 * counter_offset .. counter_offset + n_tracks - 1 (seed, tau_max_s as in
 * stk_set_tracks) and writes the k loudest to out_topk_dev (caller-owned
 * device memory, k entries), asynchronously on cuda_stream.  Its scratch (one
 * FP32 SNR per template and the selection state, 5 MiB) is a fixed array
 * in device memory that every GPU loading the library holds until the process
 * exits; the call itself calls no cudaMalloc, cudaFree or other allocating
 * routine.  The map must have been loaded earlier (stk_load_map allocates).
 * cuda_stream first waits for the work already issued on the map context's
 * stream (a pending stk_update_map pack), so the call sees the map's latest
 * data whichever stream the caller uses.  The launch shape and wait limits
 * follow the map context's tuning options (stk_set_option); templates are
 * scored in index order.
 *   n_tracks    1 .. STK_NOALLOC_MAX_TRACKS (2^20); larger ranges: split them
 *               over several calls and keep the k largest SNRs of all of them
 *               (SNR descending, then template index ascending)
 *   k           1 .. min(STK_MAX_K, n_tracks)
 *   status_dev  caller-owned device int or NULL; set to STK_OK, to
 *               STK_ETIMEOUT when a bounded in-kernel wait gave up, or to
 *               STK_EINVAL when the map context holds a deferred error from
 *               packing bad data (non-finite y, sigma <= 0, FP16 range; read and
 *               cleared by the context's next stk_sync)
 * In both failure cases every output hit is marked invalid (snr NaN, index
 * UINT64_MAX), with or without status_dev.
 * The first call on a device resolves the array's device address
 * (cudaGetSymbolAddress, with the map's device current); make that first call
 * before any stream capture.  Every call on a device shares the one array,
 * which keeps the previous call's contents (the call clears what must start
 * at zero): calls that overlap on the GPU (other streams, other host threads)
 * race and corrupt each other's results; serialise them.  The caller's current
 * device is restored on return.  Errors (message from stk_last_error(NULL)):
 * STK_EINVAL (NULL map or output, n_tracks beyond the limit, bad k or
 * tau_max), STK_ECUDA. */
#define STK_NOALLOC_MAX_TRACKS (1u << 20)
STK_API int stk_score_noalloc(const stk_map *map, uint64_t n_tracks, uint64_t seed, uint64_t counter_offset,
                              double tau_max_s, int k, stk_hit *out_topk_dev, int *status_dev,
                              void *cuda_stream);

/* ---- tuning (kernel choice and launch shape; results do not depend on them) */
#define STK_OPT_KERNEL   1 /* 0 automatic, 1 one-thread-per-template kernel, 2 shared-memory slab kernel */
#define STK_OPT_THREADS  2 /* slab kernel block size, 0 = automatic, else 32 .. 1024 */
#define STK_OPT_MAX_R    3 /* slab kernel: most templates held per thread, 1 .. 12 (default 12); 7 .. 12 limit
                              the block to 512 threads and a varying weight to 11, 1 .. 6 allow 1024 threads
                              (up to 5 with a varying weight) */
#define STK_OPT_STAGES   4 /* slab kernel: shared-memory slab buffers, 2 .. 4 (default 2) */
#define STK_OPT_SMEM_KB  5 /* slab kernel: shared-memory budget in KiB, 0 = the device maximum */
#define STK_OPT_WAIT_MS  6 /* slab kernel: limit of each in-kernel wait for a slab copy, ms (0 = 2000) */
#define STK_OPT_WITHHOLD_SLAB 7 /* test of the bounded waits: the first CTA never issues the copy of its
                                   slab number value (-1 = off, the default); the call then ends with
                                   STK_ETIMEOUT after the wait limit and the context stays usable */
#define STK_OPT_ORDER    8 /* slab kernel: 1 (default) scores templates in a coherent order -- a bucket
                              sort of the template indices by a Z-order key of (f0, f1, f2) -- so a warp's
                              pixel gathers fall in a narrow band of bins and shared-memory banks
                              rarely collide; 0 scores in index order.  Results are identical; the
                              order costs 16 bytes per template plus 4 bytes per coarse bucket
                              (at most 8192) per block of 2 x SMs blocks of context scratch */
#define STK_OPT_SELECT_SAMPLE 9 /* top-k selection: templates whose SNRs are sampled to set the
                                   candidate threshold, 0 (default: 16384) or 1 .. 49152.  Results do
                                   not depend on it: a threshold that admits fewer than k templates
                                   (likelier with a small sample) makes the selection fall back to an
                                   exact radix select over every SNR, which is slower */
#define STK_OPT_INTERP_THREADS 10 /* continuous templates (stk_interp_*, stk_refine): threads per
                                     template, 0 (default: 128 up to 1536 templates, else 32), 32,
                                     64 or 128.  Results may differ in the last bits
                                     (the order of the column sums) */

/* Set a tuning option for later scoring calls.  Errors: STK_EINVAL. */
STK_API int stk_set_option(stk_ctx *ctx, int option, int64_t value);

/* Launch shape of the last scoring call: out[0] kernel (1 simple, 2 slab,
 * 3 general templates), [1] templates per thread, [2] threads per block,
 * [3] grid, [4] time columns per slab, [5] slab buffers, [6] template batches,
 * [7] dynamic shared bytes, [8] 1 if templates were scored in coherent order. */
STK_API int stk_last_plan(const stk_ctx *ctx, int64_t out[9]);

/* Message for the last error on ctx (never NULL; "" when none). */
STK_API const char *stk_last_error(const stk_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* STK_H */
