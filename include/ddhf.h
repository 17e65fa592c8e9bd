/*
 * ddhf.h - C ABI of the GB300 DDHF hot path (libddhf.so).
 *
 * DDHF ("Real-Time Drone Detection in Event Cameras via Per-Pixel Frequency
 * Analysis", arXiv 2603.08386) detects drone rotors in an event-camera stream:
 * the events of a window are binned per pixel (Sec. 3.5), each active pixel's
 * non-uniform DFT power spectrum is evaluated directly (Sec. 3.3, Eq. 6),
 * noise-like spectra are rejected by spectral flatness (Sec. 3.4, Eq. 7), a
 * median-normalised harmonic comb picks rotor pixels and their dominant
 * frequency (Eq. 8-11), and the rotor mask becomes drone boxes by 8-connected
 * labelling, an area filter and centroid merging (Sec. 3.5, Eq. 12).
 *
 * Conventions for every entry point:
 *  - Data pointers are CUDA device pointers owned by the caller unless a
 *    parameter says "host". The library never frees or retains them past the
 *    call (except the per-window event lists it copies into its workspace).
 *  - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream). Counts that depend on the data (events kept,
 *    active pixels, boxes) are written to device memory, so a sequence of
 *    calls can be captured into a CUDA graph; ddhf_get_stats() synchronises
 *    and reads them back on the host.
 *  - No call aborts or throws. Each returns a ddhf_status; on failure
 *    ddhf_last_error(ctx) holds a one-line message. Invalid events (outside
 *    the window or the sensor, bad polarity) are dropped and counted, not
 *    errors. Overflow of a caller-sized output is flagged on the device and
 *    reported as DDHF_ERR_CAPACITY by ddhf_get_stats().
 *  - A context is bound to the CUDA device that was current at ddhf_create()
 *    and must be used from one host thread at a time. Its kernels keep work
 *    counters in the context's workspace (one set per window slot, plus
 *    context-wide ones), so calls enqueued on different streams of one
 *    context must not run on the GPU at the same time; the overlap that
 *    ddhf_detect_batch arranges itself (the comb of one window beside the
 *    spectra of the next) uses separate counters.
 */
#ifndef DDHF_H
#define DDHF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ddhf_ctx ddhf_ctx;
typedef void *ddhf_stream; /* cudaStream_t */

typedef enum {
  DDHF_OK = 0,
  DDHF_ERR_INVALID_ARG = 1, /* a pointer, size or parameter is out of range */
  DDHF_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in last_error) */
  DDHF_ERR_CAPACITY = 3,    /* an output or workspace was too small */
  DDHF_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  DDHF_ERR_UNSUPPORTED = 5, /* a configuration the library does not handle */
  DDHF_ERR_STATE = 6        /* calls out of order (e.g. spectrum before binning) */
} ddhf_status;

/* Frequency grid (Sec. 3.3 Eq. 6, Sec. 3.5): bin j = 0..n_bins-1 evaluates
 * a_j = a0 + j*da in units of 1/denom cycles per microsecond, so the phase of
 * an event at tau microseconds is the exact integer residue (a_j*tau) mod
 * denom in units of 1/denom cycles.
 *   Hz grid:   a_j in mHz, denom = 1e9 (f_j = a_j/1000 Hz).
 *   Mode grid: a0 = 0, da = 1, denom = window_us: the paper's integer modes
 *              k = 0..K-1 over timestamps normalised to the window.
 * Requires a0 >= 0, da > 0, 0 < denom < 2^31, n_bins in [1, 16384] and
 * a_{n_bins-1} < 2^32. */
typedef struct {
  int64_t a0;
  int64_t da;
  int64_t denom;
  int32_t n_bins;
  int32_t reserved;
} ddhf_grid;

/* Thresholds of Sec. 3.4-3.5; ddhf_default_params() gives Table 2's final
 * values (0.89, 1.5, 4, 3, 4, 6, 147, 19.05). d is Table 2's Delta k (the
 * harmonic half-width d_k of Eq. 8, in bins). polarity_01 = 1 accepts
 * polarities {0, 1} (0 meaning -1) instead of {-1, +1}.
 * Requires M >= 1, 0 <= d, 1 <= h_min, n_min >= 1, A_min >= 0, alpha >= 0 and
 * M*(2d+1) <= 254. */
typedef struct {
  float tau_sf;
  float tau_comb;
  int32_t M;
  int32_t d;
  int32_t h_min;
  int32_t n_min;
  int32_t A_min;
  int32_t polarity_01;
  double alpha;
} ddhf_params;

/* One detection (Sec. 3.5): inclusive pixel bounds and the number of rotor
 * pixels of the merged components. */
typedef struct {
  int32_t x0, y0, x1, y1, n_px;
} ddhf_box;

/* One window of one event stream for the batched call. Event arrays are
 * device pointers, n events each: x, y int16 pixel coordinates, t_us int64
 * microseconds, p int8 polarity. */
typedef struct {
  const int16_t *x;
  const int16_t *y;
  const int64_t *t_us;
  const int8_t *p;
  int64_t n;
  int64_t t0_us;
  int64_t window_us;
} ddhf_window;

/* Counters of the last binned window (slot 0) and of the last detection. */
typedef struct {
  int64_t n_in;         /* events passed to the last binning call */
  int64_t n_valid;      /* events kept */
  int64_t n_dropped;    /* events outside the window/sensor or bad polarity */
  int64_t n_active;     /* pixels with at least n_min events */
  int64_t n_rotor;      /* rotor-mask pixels of the last detection */
  int64_t n_boxes;      /* boxes of the last detection (may exceed cap) */
  int64_t terms;        /* sum over active pixels of count * n_bins */
  int64_t graph_kernels;/* kernel nodes of the last captured ddhf_detect_batch graph */
  uint32_t device_flags;/* DDHF_FLAG_* bits raised on the device */
  uint32_t reserved;
} ddhf_stats;

#define DDHF_FLAG_CAPACITY 1u /* a caller-sized output overflowed */
#define DDHF_FLAG_TIMEOUT 2u  /* a bounded device-side loop hit its limit */
#define DDHF_FLAG_INTERNAL 4u /* an internal consistency check failed (reported as DDHF_ERR_CUDA) */
#define DDHF_FLAG_INPUT 8u    /* a caller's device array held an out-of-range index (a pixel key
                                 or label at or beyond W*H), skipped; reported as
                                 DDHF_ERR_INVALID_ARG */

/* NDFT evaluation forms for ddhf_power_spectrum (Eq. 6; all give P_j in FP32).
 *  SINCOS   one warp per pixel, lanes own bins; exact integer phase per term,
 *           advanced by an exact modular step, then FP32 sin/cos per term.
 *  RECUR    one warp per pixel; each lane rotates its bins by an exact
 *           per-event step phasor, re-seeded exactly every 32 bins.
 *  BLOCKED  persistent kernel: F[32b + r] = sum_k A[b][k] B[k][r] with exact
 *           seeds A = p e^{-2 pi i a_{32b} tau} and rotations B = u^r, as a
 *           three-multiplication complex product per term; heavy pixels are
 *           split over a thread block. The form used by ddhf_detect.
 *  NAIVE32  precision study only: FP32 phase 2 pi f t from the absolute time.
 *  KAHAN    SINCOS with compensated (Kahan) accumulation.
 *  F64      check path: FP64 phase and accumulation on the GPU.
 *  HYBRID   BLOCKED for most pixels; pixels with at least
 *           max(hybrid_min, 16, ceil(G/2)) events (hybrid_min from the
 *           tuning, 64 when it is 0) take the non-uniform FFT route that the
 *           footnote to Sec. 3.3 mentions: each event, its phase centred on
 *           the middle bin, is spread onto a uniform time grid of spacing
 *           s = floor(denom / (2 da n_bins)) us with an "exponential of
 *           semicircle" kernel of 8 points (Barnett et al. 2019), and the
 *           grid's G = (window_us - 1) / s + 8 values enter one dense complex
 *           product with a table shared by all pixels, deconvolved per bin.
 *           Within a few 1e-6 of the exact Eq. 6 power relative to the
 *           pixel's peak (FP32 sums and hardware exp2 / rsqrt in the
 *           kernel values). A window with G < 16 or G > 1024 (or a grid with
 *           s < 1) runs BLOCKED alone. The first use allocates the path's
 *           workspace (about 64 bytes per max_events plus 12 KiB per bin)
 *           and copies its deconvolution factors with a synchronous copy,
 *           so make it outside stream capture (ddhf_set_tuning with
 *           hybrid_min > 0 does the same allocation up front). */
#define DDHF_FORM_SINCOS 0
#define DDHF_FORM_RECUR 1
#define DDHF_FORM_BLOCKED 2
#define DDHF_FORM_NAIVE32 3
#define DDHF_FORM_KAHAN 4
#define DDHF_FORM_F64 5
#define DDHF_FORM_HYBRID 6

/* Launch tuning of the persistent BLOCKED kernel (chosen by the autotuner).
 *  heavy_min   pixels with at least this many events (>= 32) are processed by
 *              a whole thread block (events split over its warps), the others
 *              by one warp each;
 *  warps_per_block  warps per thread block (2, 4 or 8);
 *  blocks_per_sm    resident blocks per SM used to size the persistent grid
 *                   (0 = as many as fit);
 *  rows_per_lane    32-bin rows held per lane (1, 2, 4, 6 or 8; 0 = chosen
 *                   from n_bins): a pass covers 4 * rows_per_lane rows, and
 *                   every pass re-seeds the phasor rows exactly;
 *  fuse             1: ddhf_detect / ddhf_detect_batch score each spectrum in
 *                   the kernel that computes it (spectra stay on chip); 0:
 *                   per window, a spectrum kernel writes a context-owned
 *                   buffer that a separate comb kernel reads (more warps per
 *                   SM for the latency-bound comb). Same results either way.
 *  overlap          with fuse 0 and several windows: 1 runs the comb kernel of
 *                   window w on a second stream while the spectra of window
 *                   w + 1 are computed (a second spectrum buffer is allocated
 *                   when this is first set); 0 runs them one after the other.
 *  hybrid_min       with fuse 0: pixels with at least max(hybrid_min, 16,
 *                   ceil(G/2)) events take the grid route of DDHF_FORM_HYBRID
 *                   in ddhf_detect / ddhf_detect_batch (its workspace is
 *                   allocated when this is first set); 0 turns it off. The
 *                   fused kernel ignores it.
 * Defaults: heavy_min 1024, 4 warps per block, blocks_per_sm 0, rows_per_lane
 * 0, fuse 0, overlap 0, hybrid_min 0. The unfused path needs the context's
 * spectrum buffer of W*H rows of n_bins floats, allocated by ddhf_create (for
 * more than 4096 bins only when the device has room: without it detection
 * runs fused, and returns DDHF_ERR_UNSUPPORTED when the fused kernel's
 * per-warp shared memory does not fit an SM).
 * Different tunings give spectra that agree within the FP32 rounding of the
 * summation order; each tuning is deterministic. */
typedef struct {
  int32_t heavy_min;
  int32_t warps_per_block;
  int32_t blocks_per_sm;
  int32_t rows_per_lane;
  int32_t fuse;
  int32_t overlap;
  int32_t hybrid_min;
} ddhf_tuning;

const char *ddhf_status_string(ddhf_status s);

/* Host-only (no device, no context): how DDHF_FORM_HYBRID and the
 * hybrid_min tuning treat a window of window_us on `grid` (host pointer).
 * *s_us = floor(denom / (2 da n_bins)), the grid spacing in microseconds;
 * *rows = (window_us - 1) / s + 8, the grid rows G; *threshold =
 * max(hybrid_min, 16, ceil(G / 2)), the event count from which a pixel takes
 * the route; dec[n_bins] (nullable; written when s >= 1) = the per-bin
 * deconvolution factors 1 / psi^((j - floor(n_bins/2)) da s / denom) of the
 * 8-point exponential-of-semicircle kernel. Returns DDHF_ERR_UNSUPPORTED
 * (threshold 0) when the window runs BLOCKED alone (s < 1 or G outside
 * [16, 1024]), DDHF_ERR_INVALID_ARG for a bad grid, window or hybrid_min < 1.
 * The footnote to Sec. 3.3 names the route; its parameters are this
 * library's. Any output pointer may be NULL. */
ddhf_status ddhf_hybrid_geometry(const ddhf_grid *grid, int64_t window_us, int32_t hybrid_min,
                                 int64_t *s_us, int32_t *rows, int32_t *threshold,
                                 float *dec);

/* Test hook, not in the paper: the device allocations that ddhf_create makes
 * (its workspace) succeed n more times, then the next one fails as if the
 * device were out of memory (without calling cudaMalloc), and the hook
 * disarms; n = -1 disarms it. ddhf_create then returns DDHF_ERR_CUDA with
 * every allocation it made released. Process-wide; not for concurrent use
 * with other contexts being created. */
ddhf_status ddhf_debug_fail_alloc_after(int32_t n);

/* Guard bytes: every workspace buffer of ddhf_create has 256 bytes of a fixed
 * pattern before it and at least 256 after it (inside the same allocation),
 * checked on the device by ddhf_get_stats, which reports a changed byte as
 * DDHF_FLAG_INTERNAL (DDHF_ERR_CUDA): a kernel wrote outside its buffer.
 * Test hook, not in the paper: overwrite one byte of the guard after
 * workspace buffer `index` (in allocation order), so that the next
 * ddhf_get_stats must report it. The byte lies inside the allocation. Returns
 * DDHF_ERR_INVALID_ARG for an index beyond the buffers. */
ddhf_status ddhf_debug_corrupt_guard(ddhf_ctx *ctx, int32_t index);

/* Table 2 final values. out: host pointer. */
ddhf_status ddhf_default_params(ddhf_params *out);

/* Create a context for a W x H sensor (1 <= W, H <= 32767, W*H <= 2^26) and
 * one frequency grid. Allocates device workspace on the current device for
 * up to max_windows windows of at most max_events events each (binning
 * scratch, per-window pixel lists, masks, labels, work queues). grid and
 * params are host pointers and are copied. *out receives the context. */
ddhf_status ddhf_create(int32_t W, int32_t H, const ddhf_grid *grid,
                        const ddhf_params *params, int64_t max_events,
                        int32_t max_windows, ddhf_ctx **out);

/* Release the context and its device workspace (synchronises the device). */
ddhf_status ddhf_destroy(ddhf_ctx *ctx);

ddhf_status ddhf_set_tuning(ddhf_ctx *ctx, const ddhf_tuning *tuning);

/* Replace the thresholds of Sec. 3.4-3.5 (same requirements as for
 * ddhf_create; params is a host pointer). Later binning, scoring and box
 * calls use them; a cached ddhf_detect_batch graph is dropped. This is what
 * a hyperparameter search over Table 2's ranges calls between evaluations. */
ddhf_status ddhf_set_params(ddhf_ctx *ctx, const ddhf_params *params);
ddhf_status ddhf_get_tuning(const ddhf_ctx *ctx, ddhf_tuning *out);

/* Iteration limit of the context's bounded device-side loops (the
 * union-find walks of labelling and of the Eq. 12 merge; default 2^24,
 * which no valid input reaches). A loop that reaches the limit stops,
 * raises DDHF_FLAG_TIMEOUT (ddhf_get_stats then returns DDHF_ERR_TIMEOUT and
 * clears it) and leaves in-range but unreliable labels or boxes; the context
 * stays usable. Not in the paper: this is how a test drives the timeout path
 * without stalling the GPU. limit >= 1; a cached ddhf_detect_batch graph is
 * dropped. */
ddhf_status ddhf_set_loop_limit(ddhf_ctx *ctx, int32_t limit);

/* Sec. 3.5 "Event processing": keep events with t0 <= t < t0+window_us,
 * 0 <= x < W, 0 <= y < H and a valid polarity, sort them stably by pixel key
 * y*W + x into the context's per-pixel list (slot 0), and list the active
 * pixels (at least n_min events) in ascending key order. n may be 0.
 * Requires n <= max_events and window_us < 2^31. */
ddhf_status ddhf_bin_events(ddhf_ctx *ctx, const int16_t *x, const int16_t *y,
                            const int64_t *t_us, const int8_t *p, int64_t n,
                            int64_t t0_us, int64_t window_us, ddhf_stream stream);

/* Copy the per-pixel list of slot 0 out of the context:
 *   offsets [W*H+1] uint32: events of pixel k are ev[offsets[k] .. offsets[k+1])
 *   ev      [cap_ev] uint32: bits 0-30 tau = t - t0 (us), bit 31 set for p = -1
 *   active  [W*H]   uint32: active pixel keys, ascending (n_active entries)
 *   counts  [4]     int64:  n_valid, n_dropped, n_active, n_in
 * Any pointer may be NULL to skip it. Overflow of cap_ev raises
 * DDHF_FLAG_CAPACITY and copies cap_ev events. */
ddhf_status ddhf_export_csr(ddhf_ctx *ctx, uint32_t *offsets, uint32_t *ev,
                            int64_t cap_ev, uint32_t *active, int64_t *counts,
                            ddhf_stream stream);

/* Eq. 6 and P_j = |F_j|^2 for every active pixel of slot 0, in active-list
 * order: P[a*n_bins + j] (FP32, row a of the a-th active pixel). `form` is a
 * DDHF_FORM_*. Rows beyond cap_px are not written (DDHF_FLAG_CAPACITY). */
ddhf_status ddhf_power_spectrum(ddhf_ctx *ctx, int32_t form, float *P, int64_t cap_px,
                                ddhf_stream stream);

/* Eq. 7-11 on spectra P laid out as ddhf_power_spectrum writes them (rows in
 * active-list order of slot 0), for any grid of the context: rows are scored
 * in shared memory, or, for the largest grids, where they are in P (then
 * only the comb's scratch needs shared memory: DDHF_ERR_UNSUPPORTED when
 * even that does not fit, which takes both many bins and a median band of
 * more than 32 ranks, M (2d+1) > 30). Per active pixel a: log_sf[a] = ln SF;
 * snr[a] = max_w SNR_M(w) and f0_bin[a] = its first maximising bin w when
 * SF <= tau_sf (else 0 and -1); mask[W*H] (uint8, zeroed by the call) gets 1
 * at rotor pixels (SF <= tau_sf and snr >= tau_comb). log_sf, snr and f0_bin
 * may be NULL. Given the same P, every output is bit-reproducible. */
ddhf_status ddhf_comb_score(ddhf_ctx *ctx, const float *P, int64_t cap_px, float *log_sf,
                            float *snr, int32_t *f0_bin, uint8_t *mask,
                            ddhf_stream stream);

/* Sec. 3.5 "Segmentation mask processing": 8-connected labels of mask[W*H]
 * (nonzero = rotor); labels[k] = smallest linear index of k's component,
 * -1 for background. */
ddhf_status ddhf_label(ddhf_ctx *ctx, const uint8_t *mask, int32_t *labels,
                       ddhf_stream stream);

/* Boxes of the components of labels[W*H] (as ddhf_label writes them), boxes
 * with area (x1-x0+1)(y1-y0+1) < A_min removed, then Eq. 12 centroid merging
 * repeated until no pair is within alpha * max(w1,h1,w2,h2); merged boxes are
 * union boxes. Output sorted by (y0, x0, y1, x1, n_px) into boxes[cap];
 * *n_boxes_dev (device int32) gets the total count, which may exceed cap. */
ddhf_status ddhf_boxes(ddhf_ctx *ctx, const int32_t *labels, ddhf_box *boxes, int32_t cap,
                       int32_t *n_boxes_dev, ddhf_stream stream);

/* The whole per-window pipeline of Sec. 3.5 on one window: binning, the
 * BLOCKED NDFT spectra and the SF + comb scoring (as separate kernels through
 * a context buffer, or fused so that spectra stay on chip, per the tuning's
 * fuse flag), labelling and boxes. mask_out[W*H] (nullable) receives the
 * rotor mask. */
ddhf_status ddhf_detect(ddhf_ctx *ctx, const int16_t *x, const int16_t *y,
                        const int64_t *t_us, const int8_t *p, int64_t n, int64_t t0_us,
                        int64_t window_us, ddhf_box *boxes, int32_t cap,
                        int32_t *n_boxes_dev, uint8_t *mask_out, ddhf_stream stream);

/* ddhf_detect over n_windows windows (windows is a host array) in one
 * sequence of launches: every window is binned into its own slot, one
 * persistent BLOCKED kernel scores the pixels of all windows (heavy pixels
 * first), then labelling and boxes run per window. boxes is [n_windows*cap]
 * (window w at boxes + w*cap), n_boxes_dev[n_windows], masks_out
 * [n_windows*W*H] (nullable). Requires n_windows <= max_windows. When
 * use_graph is nonzero the launch sequence is captured once into a CUDA
 * graph, keyed by the argument values, and replayed on later calls with the
 * same arguments. */
ddhf_status ddhf_detect_batch(ddhf_ctx *ctx, const ddhf_window *windows, int32_t n_windows,
                              ddhf_box *boxes, int32_t cap, int32_t *n_boxes_dev,
                              uint8_t *masks_out, int32_t use_graph, ddhf_stream stream);

/* Per-pixel outputs of slot w of the last ddhf_detect / ddhf_detect_batch:
 * active [W*H] uint32 keys, log_sf, snr [W*H] float, f0_bin [W*H] int32 in
 * active-list order, counts [4] as in ddhf_export_csr. Nullable. */
ddhf_status ddhf_export_scores(ddhf_ctx *ctx, int32_t slot, uint32_t *active, float *log_sf,
                               float *snr, int32_t *f0_bin, int64_t *counts,
                               ddhf_stream stream);

/* Dominant frequency of each detection (Eq. 11 returns one per rotor pixel;
 * a box summarises those of the rotor pixels inside it): for box b <
 * min(*n_boxes_dev, cap) of slot w's last ddhf_detect / ddhf_detect_batch
 * (boxes, n_boxes_dev: device arrays as those calls wrote them), over the
 * rotor pixels of slot w whose (x, y) lies inside the box's inclusive bounds:
 *   f0_bin[b]        the dominant bin of the one with the largest SNR (ties:
 *                    the smallest pixel key), -1 when there is none;
 *   snr[b]           its SNR, 0 when there is none (nullable);
 *   f0_hz_median[b]  the lower median (rank floor((n-1)/2) of the n sorted
 *                    values) of their dominant bins, as a frequency in Hz
 *                    ((a0 + j da) 1e6 / denom), 0 when there is none
 *                    (nullable).
 * Device outputs of cap entries; entries from min(*n_boxes_dev, cap) on are
 * left unchanged. */
ddhf_status ddhf_box_frequencies(ddhf_ctx *ctx, int32_t slot, const ddhf_box *boxes,
                                 const int32_t *n_boxes_dev, int32_t cap, int32_t *f0_bin,
                                 float *snr, float *f0_hz_median, ddhf_stream stream);

/* The 8-connected labels (as ddhf_label writes them) of slot w's rotor mask
 * from the last ddhf_detect / ddhf_detect_batch (Sec. 3.5 "Segmentation mask
 * processing"): labels[W*H] (device int32), a copy of what the detection
 * computed, so that a caller that needs them (row bands) does not label the
 * mask again. */
ddhf_status ddhf_export_labels(ddhf_ctx *ctx, int32_t slot, int32_t *labels, ddhf_stream stream);

/* Tracing: when enable is nonzero, CUDA events bracket the stages of every
 * later ddhf_detect / ddhf_detect_batch call (also inside a captured graph,
 * as external event nodes; enabling or disabling drops a cached graph).
 * ddhf_stage_times() waits for the last recorded call and writes out_ms[5]
 * (host), device milliseconds summed over the call's windows:
 *   [0] binning, [1] classification (NDFT + SF + comb), [2] labels + boxes,
 *   [3] spectrum kernels and [4] comb kernels of the unfused path (0 when
 *   fused, where [1] is the single fused kernel).
 * Returns DDHF_ERR_STATE if nothing was recorded. */
ddhf_status ddhf_enable_stage_timing(ddhf_ctx *ctx, int32_t enable);
ddhf_status ddhf_stage_times(ddhf_ctx *ctx, float *out_ms);

/* ddhf_detect over n_windows windows whose event arrays are in HOST memory
 * (windows[w].x/y/t_us/p host pointers; page-locked memory lets the copies
 * overlap the kernels). The windows go through in groups of G = min(16,
 * max_windows, n_windows): group k + 1's events are copied into one of two
 * context-owned device staging sets on an internal copy stream while group k
 * is processed on `stream` by the batched detection (the kernels and tuning
 * of ddhf_detect_batch, one slot per window of the group, launched without a
 * graph); each window's binning waits only for that window's copy. Results go to host memory: boxes_host[n_windows * cap] (window w
 * at boxes_host + w * cap), n_boxes_host[n_windows], masks_host[n_windows *
 * W * H] (nullable). The call returns once the work is enqueued; host inputs
 * must stay valid and outputs are complete when `stream` has finished. The
 * copies are ordered after the work already queued on `stream`. Any
 * n_windows >= 1; the first call allocates the staging sets (2 x G x
 * max_events events) and the device box buffers. */
ddhf_status ddhf_detect_batch_host(ddhf_ctx *ctx, const ddhf_window *windows, int32_t n_windows,
                                   ddhf_box *boxes_host, int32_t cap, int32_t *n_boxes_host,
                                   uint8_t *masks_host, ddhf_stream stream);

/* Soft comb score and its gradients for the differentiation pattern (not in
 * the paper; built on Eq. 6 and the comb of Eq. 8-10). For each listed pixel
 * a (pixels[n_px]: pixel keys y*W+x of the last binned window) with
 * fundamental f0[a] (Hz):
 *   f_hq = h f0 + q delta_hz,  h = 1..n_h (<= 8), q = -Q..Q (Q <= 8)
 *   G_hq = exp(-(q delta)^2 / (2 sigma_h^2)),  Z_h = sum_q G_hq
 *   S[a] = sum_h w_h (sum_q G_hq P_a(f_hq) / Z_h) / B[a]
 * where P_a(f) = |sum_k p_k exp(-2 pi i f (tau_k - tau_c_us) 1e-6)|^2 is Eq. 6
 * at a real frequency (exact integer-mHz phase plus a sub-mHz remainder; f0
 * and delta_hz are rounded to 1 micro-Hz, tau_c_us to 0.5 us, which changes
 * neither P nor dP/df) and B[a] > 0 a constant background (e.g.
 * ddhf_spectrum_median of the grid spectrum). w, sigma: [n_h] device floats.
 * Requires 1e-6 <= delta_hz < 1e6 and 0 <= tau_c_us < 2^20.
 * Forward (grad_S == NULL): writes S[n_px].
 * Backward (grad_S != NULL, S ignored): with g = grad_S,
 *   grad_f0[a] = g[a] dS_a/df0,  grad_w[h] = sum_a g[a] dS_a/dw_h,
 *   grad_sigma[h] = sum_a g[a] dS_a/dsigma_h,
 *   grad_f[(a n_h + h - 1)(2Q+1) + q + Q] = g[a] dS_a/df_hq
 *     = g[a] w_h G_hq P_a'(f_hq) / (Z_h B[a])   (nullable: the gradient with
 *     respect to each evaluation frequency; dS/df0 = sum_hq h dS/df_hq),
 * using dP/df = 2 Re(conj F dF/df); sums over pixels in a fixed order. */
ddhf_status ddhf_softcomb(ddhf_ctx *ctx, int64_t n_px, const uint32_t *pixels, const float *f0,
                          int32_t n_h, int32_t Q, double delta_hz, double tau_c_us,
                          const float *w, const float *sigma, const float *B, float *S,
                          const float *grad_S, float *grad_f0, float *grad_w, float *grad_sigma,
                          float *grad_f, ddhf_stream stream);

/* Median of each spectrum row P[rows][n_bins] (the mean of the two middle
 * values for an even count, as in Eq. 9-10), exact: median[rows]. */
ddhf_status ddhf_spectrum_median(ddhf_ctx *ctx, const float *P, int64_t rows, float *median,
                                 ddhf_stream stream);

/* Spectra without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * running (for example an embedded real-time detector whose memory is all
 * reserved at start-up, since cudaMalloc may synchronise the device for
 * milliseconds, or a host program whose own allocator owns the device), and
 * so cannot create a context.
 * Computes the same P, bit for bit, as ddhf_power_spectrum(DDHF_FORM_BLOCKED)
 * with the default tuning, from a per-pixel list the caller built and owns
 * (device pointers, the layout ddhf_export_csr writes): offsets[k] ..
 * offsets[k+1] index ev (packed tau | sign << 31) for pixel key k, and must
 * stay within ev[0 .. n_events) for every listed key (rows are unspecified
 * otherwise); active[n_active] lists the pixel keys to evaluate; P[a * n_bins
 * + j] for a < n_active (cap_px >= n_active required). grid is a host pointer.
 * flags_dev (device uint32, nullable) receives, in stream order after the
 * spectra, the DDHF_FLAG_* bits this call raised: DDHF_FLAG_CAPACITY when its
 * list of heavy pixels overflowed (only possible with offsets beyond
 * n_events; those pixels' rows are NaN).
 * Limits: n_events <= 2^25 events in ev, n_active <= 2^26. Larger sizes
 * return DDHF_ERR_INVALID_ARG. Its scratch is one fixed 256 KiB __device__
 * array (kept by every device that loads the library until exit). The first
 * call in a CUDA context looks up that array's address and loads all of this
 * entry point's kernels (so that later calls, on any grid, load nothing under
 * lazy module loading): make it before any stream capture and outside any
 * time budget. All calls share the array, so calls that overlap on the GPU
 * race: serialise them. */
ddhf_status ddhf_power_spectrum_noalloc(const ddhf_grid *grid, const uint32_t *offsets,
                                        const uint32_t *ev, int64_t n_events,
                                        const uint32_t *active, int64_t n_active, float *P,
                                        int64_t cap_px, uint32_t *flags_dev, ddhf_stream stream);

/* ---------------------------------------------------------------- row bands
 * The per-pixel steps (binning, Eq. 6-11) are independent per pixel, so a
 * sensor can be split into row bands processed by separate contexts (one per
 * GPU). Only the segmentation of Sec. 3.5 couples the bands: components that
 * cross a band boundary are joined through the labels of the two boundary
 * rows, then the area filter and the Eq. 12 merge run once on the joined
 * components. The paper describes a single device; this is the same
 * computation split by rows. */

/* One connected component of a band's rotor mask in sensor coordinates:
 * label = smallest sensor linear index y*W_sensor + x of its pixels,
 * inclusive bounding box, pixel count. */
typedef struct {
  int32_t label, x0, y0, x1, y1, n_px;
} ddhf_component;

/* Make the context a row band: its rows 0..H-1 are sensor rows row0..row0+H-1.
 * Binning then keeps events with row0 <= y < row0 + H (others are dropped and
 * counted), and pixel keys and outputs stay band-local. row0 >= 0. */
ddhf_status ddhf_set_row_offset(ddhf_ctx *ctx, int32_t row0);

/* Components of labels[W*H] (as ddhf_label writes them, band-local) with no
 * area filter and no merging, in sensor coordinates for a band whose row 0 is
 * sensor row row0 (labels and y shifted by row0 * W and row0). Order is
 * unspecified. comps[cap] device array; *n_dev (device int32) gets the total,
 * which may exceed cap. */
ddhf_status ddhf_components(ddhf_ctx *ctx, const int32_t *labels, int32_t row0,
                            ddhf_component *comps, int32_t cap, int32_t *n_dev,
                            ddhf_stream stream);

/* Host-only: the boxes of a W x H sensor split into n_bands row bands, equal
 * to what ddhf_boxes gives on the whole sensor's labels. Band b covers rows
 * [band_row0[b], band_row0[b+1]) (band_row0 has n_bands + 1 entries,
 * increasing, from 0 to H). edge_labels[b*2*W + k*W + x] is band b's own
 * label (band-local, as ddhf_label writes it; -1 for background) of its first
 * (k = 0) and last (k = 1) row at column x. comps holds every band's
 * components (as ddhf_components writes them, in sensor coordinates),
 * band b's at comps[comp_off[b] .. comp_off[b+1]). Components touching
 * across a boundary (8-connected) are joined; boxes with area < A_min are
 * removed; Eq. 12 merging is repeated to a fixed point with params->alpha;
 * output sorted by (y0, x0, y1, x1, n_px) into boxes[cap], the total in
 * *n_boxes (may exceed cap). All pointers are host memory. */
ddhf_status ddhf_merge_bands(int32_t W, int32_t H, int32_t n_bands, const int32_t *band_row0,
                             const int32_t *edge_labels, const ddhf_component *comps,
                             const int64_t *comp_off, const ddhf_params *params,
                             ddhf_box *boxes, int32_t cap, int32_t *n_boxes);

/* ------------------------------------------------------ sliding window
 * Sec. 3.3 notes that the direct NDFT can add the contribution of each event
 * on its own as it arrives. These calls keep Eq. 6 current while a window of
 * window_us slides over one event stream: the context holds, per pixel, the
 * complex sum F_j = sum_k p_k e^{-2 pi i a_j (t_k - t_begin) / denom} over
 * the events in the window (phases from exact integer residues, as in
 * ddhf_power_spectrum) and the window's event count, and each push adds the
 * terms of the events that enter and subtracts those of the events that
 * leave. |F_j|^2 equals Eq. 6's P_j over the window [t_end - window_us,
 * t_end) (the time origin only multiplies F_j by a unit phase factor).
 * Memory: W*H*ceil32(n_bins)*8 bytes of state plus 12 bytes per ring entry.
 * A context has at most one sliding window. It shares the context's
 * workspace and slot 0 with ddhf_detect and friends, so calls on one context
 * must be ordered (one stream, or events between streams). Pushes depend on
 * host-side ring bookkeeping, so they are not for stream capture. */

/* Counters of the sliding window (ddhf_slide_get_stats). */
typedef struct {
  int64_t t_end_us;    /* end of the window after the last push */
  int64_t pushes;      /* pushes since ddhf_slide_begin */
  int64_t rebuilds;    /* pushes that recomputed the state from the window's events */
  int64_t n_added;     /* events added, all pushes */
  int64_t n_dropped;   /* pushed events not added (time, sensor or polarity) */
  int64_t n_expired;   /* events that have left the window */
  int64_t n_window;    /* events in the window now */
  int64_t last_delta;  /* events whose terms the last push evaluated */
  int64_t last_pixels; /* pixels whose state the last push changed */
  int64_t ring_used;   /* ring entries held */
} ddhf_slide_stats;

/* Start (or restart) a sliding window of window_us microseconds over a stream
 * that begins at t_begin_us: the state is zero and t_end = t_begin_us.
 * capacity: ring entries (events) held, at least the events of one window
 * plus those of one push; requires capacity <= max_events and < 2^31.
 * rebuild_every = R > 0: every R-th push recomputes the state from the events
 * still in the window instead of updating it, so the FP32 rounding of at most
 * R - 1 updates accumulates in F (R = 1: every push recomputes); R = 0: never.
 * Allocates the state (synchronises the device). */
ddhf_status ddhf_slide_begin(ddhf_ctx *ctx, int64_t window_us, int64_t t_begin_us,
                             int64_t capacity, int32_t rebuild_every);

/* Release the sliding window's state (synchronises the device). */
ddhf_status ddhf_slide_end(ddhf_ctx *ctx);

/* Advance the window to end at t_end_us (>= the previous end). Events x, y, t_us,
 * p (device arrays of n, n may be 0; any order) are added when
 * max(t_prev, t_end_us - window_us) <= t < t_end_us (t_prev = the previous end),
 * the pixel is on the sensor (row offset applied) and the polarity is valid;
 * the others are dropped and counted. Events with t < t_end_us - window_us
 * leave the window. Returns DDHF_ERR_CAPACITY, with nothing done, when the
 * ring cannot hold the push. */
ddhf_status ddhf_slide_push(ddhf_ctx *ctx, const int16_t *x, const int16_t *y,
                            const int64_t *t_us, const int8_t *p, int64_t n, int64_t t_end_us,
                            ddhf_stream stream);

/* Spectra of the window: the pixels with at least n_min events in the window
 * become slot 0's active list (ascending keys; ddhf_export_scores(ctx, 0, ...)
 * reads it and the counts) and P[a*n_bins + j] = |F_j|^2 of the a-th of them
 * (FP32; rows beyond cap_px are not written and raise DDHF_FLAG_CAPACITY;
 * cap_px = 0 lists the pixels only). */
ddhf_status ddhf_slide_spectra(ddhf_ctx *ctx, float *P, int64_t cap_px, ddhf_stream stream);

/* Detection on the current window: the active list as in ddhf_slide_spectra,
 * then the SF + comb scoring, labelling and boxes of ddhf_detect on |F|^2
 * (outputs and their layout as in ddhf_detect; slot 0's scores). The comb
 * kernel squares the state as it reads it: no spectrum buffer is written. */
ddhf_status ddhf_slide_detect(ddhf_ctx *ctx, ddhf_box *boxes, int32_t cap, int32_t *n_boxes_dev,
                              uint8_t *mask_out, ddhf_stream stream);

/* Synchronise and read the sliding window's counters (host struct). */
ddhf_status ddhf_slide_get_stats(ddhf_ctx *ctx, ddhf_slide_stats *out);

/* ------------------------------------------------------ pipe peaks
 * Not in the paper: the roofline denominators of the NDFT and comb kernels,
 * measured on the current device instead of derived from unit counts. Four
 * kernels each run 8 independent dependency chains per thread for `iters`
 * steps (1 <= iters <= 2^24; 2^16 takes a few milliseconds per kernel on a
 * GB300) on 8 blocks of 256 threads per SM, timed with CUDA events on
 * `stream` after one warm-up launch:
 *   ffma_per_s        FP32 fused multiply-adds per second (one per instruction),
 *   ffma2_lane_per_s  FP32 fused multiply-adds per second issued as paired
 *                     f32x2 instructions (two per instruction),
 *   sin_approx_per_s  sin.approx.f32 results per second (special-function unit),
 *   lg2_approx_per_s  lg2.approx.f32 results per second,
 * whole device, at whatever clock the device runs during the measurement.
 * sm_count and sm_clock_max_mhz come from the device attributes. Synchronous;
 * allocates (and frees) one 1 KiB device buffer. out: host pointer. */
typedef struct {
  int32_t sm_count;
  int32_t sm_clock_max_mhz;
  double ffma_per_s;
  double ffma2_lane_per_s;
  double sin_approx_per_s;
  double lg2_approx_per_s;
  float elapsed_ms[4];
} ddhf_pipe_peaks;

ddhf_status ddhf_measure_pipes(ddhf_pipe_peaks *out, int32_t iters, ddhf_stream stream);

/* Synchronise the context's last stream and read its counters and device
 * flags. Returns DDHF_ERR_CAPACITY / DDHF_ERR_TIMEOUT when the matching
 * flag is set (the stats are filled either way); the flags are then cleared. */
ddhf_status ddhf_get_stats(ddhf_ctx *ctx, ddhf_stats *out);

/* One-line description of the last failure of this context ("" if none). */
const char *ddhf_last_error(const ddhf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* DDHF_H */
