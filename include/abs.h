/*
 * abs.h -- C ABI of the GB300 (sm_103a) visibility-based binned angular
 * bispectrum (ABS) estimator of arXiv 2412.02246, Sec. 2.
 *
 * Problem statement (Sec. 2): measured visibilities V(U_i) at baselines U_i
 * are gridded on a uv grid of spacing dU (Eq. vg); for every ring a_m of the
 * uv plane the ring-restricted grid is Fourier transformed to a real sky-plane
 * field (Eqs. iFT, iFT_I); for every combination of three rings the triple
 * product of the fields is summed over the sky plane and divided by the same
 * sum for unit-mask fields (Eq. estimator_t).  The result is the binned
 * bispectrum B(l1, l2, l3) together with the exact number of closed grid
 * triangles behind each value.
 *
 * Conventions used by every entry point:
 *
 *  - Grid cells g = (gx, gy) with |gx|, |gy| <= n/2 - 1; grids are n x n,
 *    row-major [gy][gx] in FFT order (index gx mod n, gy mod n; the row and
 *    column at index n/2 stay zero).
 *  - dU is used as its IEEE binary32 rounding everywhere.  The nearest grid
 *    point of a baseline coordinate u is floor(fl32(fl32(u / dU) + 0.5)).
 *  - Ring m holds the cells with Q_m <= |g|^2 < Q_{m+1},
 *    Q_m = ceil((l_m / (2 pi dU))^2) evaluated in binary64 on the host
 *    (half-open bins [l_m, l_{m+1}) in l = 2 pi |U_g|).
 *  - Every visibility is also entered at -U_i with V* (the sky is real), so
 *    the gridded data are Hermitian and every field is real.
 *  - A cell is "filled" if at least one visibility's footprint covers it;
 *    the estimator uses the weighted mean X_g = V_g / sum w on filled cells
 *    and unit-mask fields for the denominator, which makes the denominator
 *    N^2 T_ijk with T_ijk the integer number of ordered closed triangles
 *    (g1 in a_i, g2 in a_j, g3 in a_k, all filled, g1 + g2 + g3 = 0).
 *  - Triplets are (i, j, k) with i <= j <= k, listed in lexicographic order.
 *  - The sky grid side N (n_fft) must be at least 3 R + 1, R the largest
 *    |gx| of any ring cell, so that no wrapped triangle enters the sums.
 *
 * Ownership and execution: the caller allocates every d_* buffer on the
 * context's device and keeps it alive until the context's stream has
 * finished the call.  The context owns its workspaces, tables and caches and
 * frees them in abs_destroy.  All device work is enqueued asynchronously on
 * the context's stream.  A call returns ABS_OK once its work is enqueued, an
 * error code for bad arguments (nothing enqueued), or ABS_ERR_CUDA for a
 * launch failure.  Data-dependent device errors (for instance an unsorted
 * triplet list) are latched into the context and reported by abs_sync.
 * Contexts are not thread-safe; use one per host thread.  abs_last_error
 * describes the last non-OK status.
 */
#ifndef ABS_GB300_H
#define ABS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ABS_OK = 0,
    ABS_ERR_INVALID_ARG = 1,  /* argument outside the documented domain; nothing enqueued */
    ABS_ERR_CUDA = 2,         /* a CUDA runtime call or kernel launch failed */
    ABS_ERR_OOM = 3,          /* workspace allocation failed */
    ABS_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    ABS_ERR_UNSUPPORTED = 5,  /* valid request this build does not implement */
    ABS_ERR_DEVICE = 6        /* device-side validation failed (see abs_last_error) */
} abs_status;

enum { ABS_KERNEL_NGP = 0, ABS_KERNEL_GAUSS = 1 };
enum { ABS_FP32 = 0, ABS_SPLIT_BF16 = 1 };
/* Weights W_g of Eqs. iFT and iFT_I (Sec. 2).
 * ABS_W_MEAN_UNITMASK: D fields of the weighted mean X_g = V_g / sum w, unit-mask
 *   I fields (1 on filled cells), so that sum_theta I_i I_j I_k = N^2 T with T the
 *   integer count of closed grid triangles and B is the mean of X1 X2 X3 over them.
 * ABS_W_PAPER_LITERAL: as printed, W_g = 1 / N_g with N_g the number of
 *   visibilities entered at the cell by Eq. vg (each visibility counts once in
 *   every cell of its footprint, and once more at the mirror): D fields of
 *   V_g / N_g, I fields of 1 / N_g.
 * ABS_W_NOISE: noise-optimised weights for equal, uncorrelated visibility noise
 *   (Sec. 2): W_g = N_eff,g = (sum w)^2 / sum w^2, the inverse noise variance of
 *   X_g in units of one visibility's; D fields of N_eff X_g, I fields of N_eff.
 *   With nearest-grid-point gridding N_eff = N_g and D carries the plain sums V_g.
 * The two weighted forms give B = Re S / (A S_W), S_W the sum of W1 W2 W3 over the
 * closed triangles (NaN where it is 0). */
enum { ABS_W_MEAN_UNITMASK = 0, ABS_W_PAPER_LITERAL = 1, ABS_W_NOISE = 2 };

#define ABS_MAX_BINS 254      /* ring ids fit a byte with one code to spare */
#define ABS_MAX_RADIUS 3      /* largest Gaussian footprint half-width (cells) */
#define ABS_MAX_FFT 4096      /* largest sky-grid side N */

typedef struct abs_config {
    int32_t n_grid;           /* uv grid side n: even, 8 <= n <= 8192 */
    double du;                /* grid spacing dU_g in wavelengths (> 0), used as binary32 */
    int32_t kernel;           /* ABS_KERNEL_GAUSS (default) or ABS_KERNEL_NGP (Eq. vg) */
    double sigma_cells;       /* Gaussian kernel width in cells, GAUSS only: > 0.25 and
                                 > (radius_cells + 0.5) / 9, so that every footprint weight
                                 (at most (r + 1/2)^2 / sigma^2 = 81 e-folds down) is a
                                 normal FP32 number and a filled cell has weight sum > 0 */
    int32_t radius_cells;     /* footprint half-width r in cells, 0..ABS_MAX_RADIUS, GAUSS only */
    int32_t n_bins;           /* number of rings, 1..ABS_MAX_BINS */
    const double *ell_edges;  /* host: n_bins + 1 strictly ascending edges in l, edges[0] > 0 */
    int32_t n_fft;            /* sky grid N: 0 = smallest 2^a 3^b 5^c >= 3R+1; else a
                                 2^a 3^b 5^c value with 3R+1 <= N <= ABS_MAX_FFT */
    int32_t precision;        /* triple sums: ABS_FP32 or ABS_SPLIT_BF16 */
    double norm_A;            /* A of Eq. estimator_t (> 0; 1 leaves B in grid units) */
    int32_t weight_mode;      /* ABS_W_MEAN_UNITMASK (default, 0), ABS_W_PAPER_LITERAL or ABS_W_NOISE;
                                 the weighted forms apply to abs_estimate, abs_estimate_many,
                                 abs_estimate_batched and abs_estimate_host (d_count is the integer
                                 count either way); the stage calls give the unit-mask pieces */
} abs_config;

typedef struct abs_ctx abs_ctx;

/* Create a context on CUDA device `device`; all work goes to `cuda_stream`
 * (a cudaStream_t, NULL = the legacy default stream).  *out is set to NULL on error. */
abs_status abs_create(abs_ctx **out, int32_t device, void *cuda_stream);

/* Release the context and everything it owns (synchronises its stream first). */
abs_status abs_destroy(abs_ctx *ctx);

/* Human-readable text for the context's last non-OK status ("" if none). */
const char *abs_last_error(const abs_ctx *ctx);

/* Wait for the context's stream, then report any latched device-side error
 * (ABS_ERR_DEVICE or ABS_ERR_TIMEOUT) and clear it. */
abs_status abs_sync(abs_ctx *ctx);

/* Host-only helpers (no device work).
 * abs_ring_q: the n_bins + 1 integer thresholds Q_m (ring definition above).
 * abs_fft_size: the sky-grid side N the estimator uses for cfg (resolves n_fft = 0).
 * abs_triplets: the closing triplets of cfg in canonical order: i <= j <= k with
 *   sqrt(Q_k) <= sqrt(Q_{i+1} - 1) + sqrt(Q_{j+1} - 1) (integer test), i.e. every
 *   ring combination that can hold a closed triangle ("every possible
 *   combination of three annular rings", Sec. 3).  Writes min(cap, count)
 *   triplets as [t][3] int32 to ijk (may be NULL) and the count to *n_trip. */
abs_status abs_ring_q(const abs_config *cfg, int64_t *q);
abs_status abs_fft_size(const abs_config *cfg, int32_t *n_fft);
abs_status abs_triplets(const abs_config *cfg, int32_t cap, int32_t *n_trip, int32_t *ijk);

/* Stage 1, Eq. vg.  Grid n_vis visibilities: d_uv [n_vis][2] float32 (u, v)
 * in wavelengths, d_vis [n_vis][2] float32 (re, im).  Outputs (n x n, FFT
 * order, fully overwritten): d_grid [n*n][2] float32 = sum_i w V (mirror
 * included), d_wsum [n*n] float32 = sum_i w, d_mask [n*n] uint8 = 1 on
 * filled cells.  Visibilities with a non-finite coordinate are skipped;
 * n_vis may be 0.  Accumulation is compensated FP32 per cell run with FP64
 * cross-run sums. */
abs_status abs_grid(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *d_uv,
                    const float *d_vis, float *d_grid, float *d_wsum, uint8_t *d_mask);

/* Stage 2, Eqs. iFT / iFT_I.  For every ring m: X = d_grid / d_wsum on the
 * filled cells of a_m, zero elsewhere; D_m(p) = sum_g X_g exp(-2 pi i g.p / N)
 * on the N x N sky grid (unnormalised forward DFT, real by Hermitian
 * symmetry).  d_fields [n_bins][N][N] float32, row-major [p_y][p_x]. */
abs_status abs_filter_fft(abs_ctx *ctx, const abs_config *cfg, const float *d_grid,
                          const float *d_wsum, const uint8_t *d_mask, float *d_fields);

/* Stages 3-4, Eq. estimator_t numerator and denominator.
 * d_sum [n_trip] float64 (may be NULL): S_ijk = N^-2 sum_p D_i D_j D_k over the
 *   sky grid (equal to the sum of X1 X2 X3 over the closed triangles), in
 *   cfg->precision.
 * d_count [n_trip] int64 (may be NULL): T_ijk, exact integer triangle counts
 *   from d_mask (= N^-2 sum_p I_i I_j I_k for unit-mask fields).
 * d_ijk [n_trip][3] int32 device, canonical order (i <= j <= k, lexicographic,
 *   k < n_bins); a list that breaks this is reported by abs_sync. */
abs_status abs_triple(abs_ctx *ctx, const abs_config *cfg, const float *d_fields,
                      const uint8_t *d_mask, int32_t n_trip, const int32_t *d_ijk,
                      double *d_sum, int64_t *d_count);

/* Stage 5.  d_B[t] = d_sum[t] / (norm_A * d_count[t]) in FP64, NaN where the
 * count is 0.  d_ellbar [n_bins] (may be NULL): mean l = 2 pi |g| dU over the
 * filled cells of each ring (NaN for an empty ring), from d_mask. */
abs_status abs_normalise(abs_ctx *ctx, const abs_config *cfg, int32_t n_trip,
                         const double *d_sum, const int64_t *d_count, double *d_B,
                         const uint8_t *d_mask, double *d_ellbar);

/* Whole estimate, V -> B: stages 1-5 with workspaces owned by the context.
 * d_ijk NULL = the canonical closing list of abs_triplets (n_trip must then
 * equal its length).  Outputs: d_B [n_trip] f64, d_count [n_trip] i64,
 * d_ellbar [n_bins] f64 (each may be NULL). */
abs_status abs_estimate(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis, const float *d_uv,
                        const float *d_vis, int32_t n_trip, const int32_t *d_ijk, double *d_B,
                        int64_t *d_count, double *d_ellbar);

/* abs_estimate on n_real realisations observed with the same baselines (the
 * ensemble of Sec. 3): d_vis [n_real][n_vis][2] float32, d_B [n_real][n_trip],
 * d_count [n_trip] (counts depend on the baselines only), d_ellbar [n_bins].
 * The baseline plan, the ring tables and the counts are built once. */
abs_status abs_estimate_many(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis,
                             const float *d_uv, int32_t n_real, const float *d_vis,
                             int32_t n_trip, const int32_t *d_ijk, double *d_B,
                             int64_t *d_count, double *d_ellbar);

/* One independent estimate of a batch (abs_estimate_batched): its own
 * configuration, which may differ in grid size, rings and triplets from the
 * other items', and its own device buffers, with the meaning they have in
 * abs_estimate.  cfg and its ell_edges are read during the call only. */
typedef struct abs_item {
    const abs_config *cfg;
    int64_t n_vis;
    const float *d_uv;        /* [n_vis][2] float32 */
    const float *d_vis;       /* [n_vis][2] float32 */
    int32_t n_trip;
    const int32_t *d_ijk;     /* [n_trip][3], NULL = the canonical list */
    double *d_B;              /* [n_trip] or NULL */
    int64_t *d_count;         /* [n_trip] or NULL */
    double *d_ellbar;         /* [n_bins] or NULL */
} abs_item;

/* Many independent estimates of uneven size in one call: the batching form
 * of the ensemble of Sec. 3 (many realisations or channels with their own
 * baselines, grids and rings).  Every item is validated before any work is
 * queued (ABS_ERR_INVALID_ARG names nothing queued).  On a non-default
 * stream the items run concurrently, round-robin over four internal lanes
 * (streams of the context with workspaces of their own, forked from and
 * joined back to the context's stream), and the whole batch is captured as
 * one CUDA graph on its second call with the same items (same
 * configurations and buffer addresses) and replayed from then on; the
 * buffers' contents may change between calls.  A lane's workspaces are sized
 * for the largest item it has run.  Output buffers of different items must
 * not overlap. */
abs_status abs_estimate_batched(abs_ctx *ctx, int32_t n_items, const abs_item *items);

/* abs_estimate_batched from HOST memory: every item's d_uv and d_vis are host
 * inputs and its d_B, d_count and d_ellbar host outputs (each may be NULL), with
 * the layouts of abs_item; d_ijk, if given, is a device list.  Each item's
 * inputs are copied to device buffers of the lane it runs on, its estimate
 * runs there and its outputs are copied back, all on that lane's streams, so
 * one item's copies overlap the other lanes' work.  With page-locked host
 * buffers the copies are part of the batch's CUDA graph (captured on the
 * second call with the same items, as for abs_estimate_batched); pageable
 * buffers work too, without the graph.  Validation as abs_estimate_batched;
 * the call waits until every output is in host memory and reports latched
 * device errors as abs_sync does. */
abs_status abs_estimate_batched_host(abs_ctx *ctx, int32_t n_items, const abs_item *items);

/* abs_estimate_many from HOST memory: copies h_uv, h_vis to the device,
 * runs, copies h_B, h_count, h_ellbar back, and waits for completion.
 * h_ijk NULL = canonical list.  Pinned host buffers make the copies
 * asynchronous; pageable ones work too. */
abs_status abs_estimate_host(abs_ctx *ctx, const abs_config *cfg, int64_t n_vis,
                             const float *h_uv, int32_t n_real, const float *h_vis,
                             int32_t n_trip, const int32_t *h_ijk, double *h_B,
                             int64_t *h_count, double *h_ellbar);

/* Triple sums of the FP32 path that allocate nothing.
 *
 * Some callers cannot allocate device memory at the point where they need the
 * sums: code running inside CUDA stream capture (cudaMalloc is not allowed
 * there), host code of a framework whose device allocator is the only one
 * permitted to call cudaMalloc, or latency-critical loops that must never hit
 * the allocator.  This entry point computes exactly what abs_triple computes
 * for d_sum (cfg->precision is ignored; the FP32 form is used) without a
 * context and without any allocation: its per-split partial sums live in one
 * fixed device array of ABS_STATIC_SCRATCH_BYTES inside the library, which
 * every GPU that loads libabs holds until the process exits.
 *
 * d_fields [n_bins][N][N] float32 and d_ijk [n_trip][3] int32 (canonical
 * order, as for abs_triple) are inputs, d_sum [n_trip] float64 the output; all
 * on the current CUDA device; work is enqueued on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream).  n_trip above
 * ABS_STATIC_SCRATCH_BYTES / 8 is rejected with ABS_ERR_INVALID_ARG (the
 * scratch holds at least one partial per triplet; larger problems use fewer
 * pixel splits).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The address is kept for the life of the
 * process, so resetting a device (cudaDeviceReset) after its first call is
 * not supported: the kept address would no longer be the array's.  A launch
 * failure of this call's own kernels returns ABS_ERR_CUDA; errors left over
 * from earlier work of the caller are neither reported nor cleared.  All
 * calls share the one array and it keeps
 * the last call's contents: calls whose work overlaps on the GPU (different
 * streams, or host threads) race on it and give wrong sums, so serialise them.
 * The paper has no counterpart to this entry point; it is a deployment aid. */
#define ABS_STATIC_SCRATCH_BYTES (8u << 20)
abs_status abs_triple_sums_static(const abs_config *cfg, const float *d_fields, int32_t n_trip,
                                  const int32_t *d_ijk, double *d_sum, void *cuda_stream);

/* Stage profiler (tracing).  When on, every kernel launch of the context is
 * bracketed by CUDA events on the context's stream and its device time is
 * accumulated under a stage name ("grid", "fft_rows", "count_pairs", ...).
 * abs_profile(ctx, 1) turns it on and clears the totals, abs_profile(ctx, 0)
 * turns it off.  abs_profile_read waits for the stream, then writes up to
 * `cap` entries (name, total ms, launches) and the number of stages to *n. */
typedef struct abs_stage_time {
    char name[32];
    double ms;
    int64_t launches;
} abs_stage_time;

abs_status abs_profile(abs_ctx *ctx, int32_t on);
abs_status abs_profile_read(abs_ctx *ctx, int32_t cap, int32_t *n, abs_stage_time *out);

/* Results layer (Sec. 4): B in the (l1, mu, t) shape form, count-weighted, and
 * its ensemble statistics over realisations.  A canonical triplet (i, j, k) is
 * the paper's l1 >= l2 >= l3 as (k, j, i), each side its ring's mean l
 * (d_ellbar, as abs_estimate writes it); mu = (l1^2 + l2^2 - l3^2) / (2 l1 l2),
 * t = l2 / l1, in n_mu x n_t equal bins over [0.5, 1] (values just outside,
 * from ring means, go to the edge bins).  Per realisation r and cell c:
 * B_r(c) = sum T B_r / sum T over the cell's triplets with T > 0 and finite B;
 * then d_mean[c] = <B_r(c)>, d_sigma[c]^2 = <B_r(c)^2> - <B_r(c)>^2 over the
 * n_real realisations, d_weight[c] = sum T.  Cells without triangles: NaN
 * (weight 0).
 *   d_B       [n_real][n_trip] FP64 (abs_estimate_many's output)
 *   d_count   [n_trip] int64 triangle counts
 *   d_ellbar  [n_bins] FP64 mean l per ring
 *   d_ijk     [n_trip][3] canonical triplets, or NULL for cfg's own list
 *   n_mu, n_t bins in mu and t, each in [1, 64]
 *   d_mean, d_sigma, d_weight  [n_bins][n_mu][n_t] FP64 outputs (any may be NULL)
 * Asynchronous on the context's stream; the FP64 sums are atomic, so their
 * last bits may vary from run to run. */
abs_status abs_rebin(abs_ctx *ctx, const abs_config *cfg, int32_t n_real, int32_t n_trip, const double *d_B,
                     const int64_t *d_count, const double *d_ellbar, const int32_t *d_ijk, int32_t n_mu,
                     int32_t n_t, double *d_mean, double *d_sigma, double *d_weight);

/* Discretely sampled analytic prediction [B_Ana]_d (Sec. 4, Fig. 2): Eq. bsana,
 * B_Ana = 2 (f_NG / sigma_T) (C1 C2 + C2 C3 + C3 C1), averaged over the same
 * closed triangles of filled cells that the estimate averages over:
 *   d_out[t] = 2 f_over_sigma sum (C(g1) C(g2) + C(g2) C(g3) + C(g3) C(g1)) / T_t
 * over ordered closed triangles (g1, g2, g3) in the triplet's rings, NaN where
 * T_t = 0.  It runs through the same transforms as the estimate: fields of C
 * on the filled ring cells and of the unit mask, and a mixed triple sum.
 *   d_C      [n_grid][n_grid] FP64, C(l_g) per uv cell in FFT order; C(l_-g)
 *            must equal C(l_g) (a function of |g|, as an angular power spectrum is)
 *   d_mask   [n_grid][n_grid] uint8 filled mask (abs_grid's)
 *   d_count  [n_trip] int64 triangle counts T of the same mask (abs_triple's or
 *            abs_estimate's)
 *   d_ijk    [n_trip][3] canonical triplets or NULL for cfg's list
 *   d_out    [n_trip] FP64
 * Asynchronous on the context's stream. */
abs_status abs_bana_d(abs_ctx *ctx, const abs_config *cfg, const double *d_C, const uint8_t *d_mask,
                      int32_t n_trip, const int32_t *d_ijk, const int64_t *d_count, double f_over_sigma,
                      double *d_out);

/* Visibility simulator (Sec. 3): the sky on an m x m flat grid (pixel (row b,
 * column a) at theta = ((a - m/2) dtheta, (b - m/2) dtheta), radians) times
 * the primary beam, then Eq. vis by direct DFT with Q = 1 (map units):
 *   d_vis[i] = sum over pixels dtheta^2 A(theta) T(theta) exp(+i 2 pi U_i.theta)
 * beam ABS_BEAM_NONE: A = 1; ABS_BEAM_MWA_TILE: Eq. beam, sinc^2(pi (d/lambda)
 * theta_x) sinc^2(pi (d/lambda) theta_y) with beam_param = d / lambda (4 m at
 * 154.25 MHz: 2.058); ABS_BEAM_GAUSS: Eq. A_G, exp(-theta^2 / theta_0^2) with
 * beam_param = theta_0 in radians.
 *   d_sky [m][m] FP32, d_uv [n_vis][2] FP32 wavelengths, d_vis [n_vis][2] FP32 out
 * m in [1, 8192].  Cost: n_vis x m^2 phase terms.  Asynchronous. */
enum { ABS_BEAM_NONE = 0, ABS_BEAM_MWA_TILE = 1, ABS_BEAM_GAUSS = 2 };
abs_status abs_simulate_vis(abs_ctx *ctx, int32_t m, double dtheta, const float *d_sky, int32_t beam,
                            double beam_param, int64_t n_vis, const float *d_uv, float *d_vis);

/* Autotuner of the split-BF16 triple-sum kernel (Sec. 2, Eq. estimator_t on
 * tensor cores).  On the first call of a configuration that runs eagerly (not
 * under stream capture, not while the stage profiler runs) with the canonical
 * triplet list, every launch shape (accumulator columns a work item of 128 or
 * 96, times work items of about 1, 2 or 3 per SM) is timed twice on the
 * call's own fields, kernel and reduction, and the fastest is kept, by
 * configuration, for the context and its batch lanes (an abs_estimate_batched
 * call with an untuned split-BF16 item runs its items one after another for
 * that call).  The ring transforms' pass split (lines per CTA of the column
 * and the row pass) is tuned the same way, per configuration and input form.
 * Tuning synchronises the stream on that first call.  With the autotuner off
 * the shapes come from cost models (128 columns, about 2 items per SM).
 * abs_autotune(ctx, 0 | 1) turns it off / on (on by default); shapes already
 * chosen are kept.  abs_tuned_shape writes the shape chosen for cfg: *set_cols
 * the accumulator columns of a work item (0: none chosen yet), *waves the work
 * items per SM, *measured 1 if the autotuner timed it (0: the cost model).  Any
 * output pointer may be NULL. */
abs_status abs_autotune(abs_ctx *ctx, int32_t enable);

/* Failure detection check: one kernel waits on a device flag of the context
 * that nothing sets, polling at most max_polls times (about 1 us apart), then
 * latches ABS_ERR_TIMEOUT into the context's error word, as every bounded
 * device-side wait of the library does when it gives up.  The next abs_sync
 * returns ABS_ERR_TIMEOUT and clears it; the context stays usable.
 * max_polls in [1, 2^20]. */
abs_status abs_probe_timeout(abs_ctx *ctx, int32_t max_polls);

/* Failure injection on the host: the next `count` workspace allocations of the
 * context fail as if the device were out of memory (no device call is made
 * for them), so the calls that need them return ABS_ERR_OOM; later calls
 * allocate normally.  count >= 0 (0 turns it off). */
abs_status abs_inject_alloc_failures(abs_ctx *ctx, int32_t count);
abs_status abs_tuned_shape(abs_ctx *ctx, const abs_config *cfg, int32_t *set_cols, int32_t *waves,
                           int32_t *measured);

/* ---------------------------------------------------------------------------
 * Multi-frequency (3-D) form.  The paper restricts itself to one frequency and
 * names the three-dimensional bispectrum of multi-frequency data as future work
 * (Sec. 1, Sec. 5), to be reached as the power spectrum was: the angular
 * statistic first, then a transform along frequency.  It gives no formula; this
 * is the reading implemented here:
 *
 *  - every channel c = 0 .. n_chan-1 is gridded on the same uv grid with the
 *    per-channel configuration `base` (Eq. vg), giving its weighted means X_c(g);
 *  - a cell enters only if it is filled in every channel (the common mask);
 *  - its delay modes are the transform along frequency,
 *    Xt(g, t) = sum_c X_c(g) exp(-2 pi i c t / n_chan), integer |t| <= t_max;
 *  - voxel (g, t) lies in bin u = m n_dbins + a when g is in ring a_m and
 *    delay_edges[a] <= |t| < delay_edges[a + 1];
 *  - S_uvw is the sum of Xt Xt Xt over ordered voxel triples, one in each of
 *    the bins u, v, w, with g1 + g2 + g3 = 0 and t1 + t2 + t3 = 0; T_uvw their
 *    number; B_uvw = Re S_uvw / (A T_uvw), NaN where T = 0.
 *
 * On the GPU the sums are taken over an N_z x N x N voxel grid (N_z >= 3 t_max
 * + 1 and N >= 3 R + 1, so no wrapped triangle enters), and the counts are
 * exact integers: T_uvw = T2(rings of u, v, w) x T1(delay bins of u, v, w), the
 * 2-D closed-triangle count on the common mask times the number of closing
 * delay triples of the bins. */
#define ABS_MAX_CHAN 4096     /* largest channel count */
#define ABS_MAX_DELAY 63      /* largest |t| a delay bin may hold */

typedef struct abs_config3d {
    abs_config base;          /* per-channel uv grid, gridding kernel, rings, n_fft, precision
                                 (of the triple sums) and norm_A; weight_mode must be
                                 ABS_W_MEAN_UNITMASK */
    int32_t n_chan;           /* channels, 1..ABS_MAX_CHAN, evenly spaced in frequency */
    int32_t n_dbins;          /* delay bins, >= 1, n_bins x n_dbins <= ABS_MAX_BINS */
    const int32_t *delay_edges; /* host: n_dbins + 1 strictly ascending integers in |t|,
                                 delay_edges[0] >= 0; t_max = delay_edges[n_dbins] - 1 must
                                 satisfy 2 t_max < n_chan and t_max <= ABS_MAX_DELAY */
    int32_t n_z;              /* line-of-sight grid N_z: 0 = 3 t_max + 1, else in
                                 [3 t_max + 1, 4 ABS_MAX_DELAY + 4] */
} abs_config3d;

/* Host only: the canonical bin triplets of cfg, u <= v <= w lexicographic, whose rings
 * (sorted) are in the closing list of abs_triplets(&cfg->base) and whose delay bins hold
 * a closing delay triple.  Writes min(cap, count) triplets as [t][3] int32 to uvw (may be
 * NULL) and the count to *n_trip. */
abs_status abs_triplets_3d(const abs_config3d *cfg, int32_t cap, int32_t *n_trip, int32_t *uvw);

/* Whole multi-frequency estimate: channel cube -> B_uvw.  d_uv, d_vis: [n_chan][n_vis][2]
 * float32 device (channel c's baselines in wavelengths at its own frequency, and its
 * visibilities; the same n_vis in every channel).  d_uvw: [n_trip][3] int32 device in
 * canonical order with bins < n_bins n_dbins, or NULL for the list of abs_triplets_3d
 * (n_trip must then equal its length).  Outputs (each may be NULL): d_B [n_trip] f64,
 * d_count [n_trip] int64 (exact T_uvw), d_ellbar [n_bins] f64 (mean l of each ring over
 * the common mask).  On a non-default stream the channels' gridding runs round-robin over
 * the context's four lanes (the streams abs_estimate_batched uses, forked from and joined back
 * to the context's stream), and the first call with a set of arguments runs eagerly (sizing
 * the workspaces), the second is captured as one CUDA graph and replayed after that; on the
 * legacy default stream every call runs eagerly on that stream.  A caller-given d_uvw in
 * split-BF16 precision is read back and planned on every call (one synchronisation; such a
 * call is not captured).
 * Device memory: about 4 (n_bins n_dbins N_z + 2 n_bins (t_max + 1)) N^2 bytes of fields,
 * plus the split-BF16 operands (8 bytes per bin and voxel) in that precision. */
abs_status abs_estimate_3d(abs_ctx *ctx, const abs_config3d *cfg, int64_t n_vis, const float *d_uv,
                           const float *d_vis, int32_t n_trip, const int32_t *d_uvw, double *d_B,
                           int64_t *d_count, double *d_ellbar);

#ifdef __cplusplus
}
#endif
#endif /* ABS_GB300_H */
