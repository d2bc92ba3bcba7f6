/*
 * hdr_lpa.h - C ABI of the GB300 (sm_103a) multi-sensor HDR reconstruction library.
 *
 * Method: Kronander, Gustavson, Bonnet, Ynnerman, Unger, "A Unified Framework
 * for Multi-Sensor HDR Video Reconstruction". For every output pixel the
 * library gathers the raw Bayer samples of all sensors around the pixel's
 * point in the reference frame (Section 4.2), converts them to radiant power
 * with their plug-in variance (Section 6, Eqs. 18 and 20; saturated samples
 * excluded, Section 6.1), fits a weighted local polynomial of order M <= 2 per
 * colour channel with a truncated Gaussian window times the inverse variance
 * (Sections 5.1-5.3, Eq. 6, Eq. 8) and returns the fit's constant term C_0.
 * With several window scales it keeps, per channel, the last scale whose
 * running intersection of confidence intervals C_0 +- gamma*sqrt(Var C_0)
 * (ascending scales) is non-empty; with no usable scale it lowers the order at
 * the largest scale; with no sample at all the output is NaN.
 *
 * Conventions for every entry point:
 *  - Status codes only; no exception crosses the ABI. hdr_last_error() returns
 *    a message for the calling thread's last failed call.
 *  - Argument errors are reported synchronously. Device-side errors (a
 *    bounded wait that ran out, a staging-window overrun) are recorded in a
 *    per-context status word and reported by hdr_check().
 *  - Pointers named *_dev are device pointers owned by the caller; they must
 *    stay valid until the work queued on the given stream has finished.
 *    Pointers named *_host are host pointers, read or written before the call
 *    returns.
 *  - One hdr_ctx may be used by one thread at a time.
 *  - Colour planes are ordered R, G, B. RGGB Bayer layout: sensor pixel
 *    (x even, y even) is R, (x odd, y odd) is B, the others are G.
 */
#ifndef HDR_LPA_H
#define HDR_LPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HDR_MAX_SENSORS 8
#define HDR_MAX_SCALES 8

typedef enum {
  HDR_OK = 0,
  HDR_E_INVALID = 1,     /* bad argument (reported before any GPU work)          */
  HDR_E_NOMEM = 2,       /* device or host allocation failed                     */
  HDR_E_CUDA = 3,        /* a CUDA runtime/driver call failed                    */
  HDR_E_BUSY = 4,        /* resource in use                                      */
  HDR_E_TIMEOUT = 5,     /* a bounded device-side wait ran out                   */
  HDR_E_UNSUPPORTED = 6, /* valid but outside what this build implements         */
  HDR_E_INTERNAL = 7     /* a device-side consistency check failed               */
} hdr_status;

typedef struct hdr_ctx hdr_ctx;

/* One sensor s of a rig (Sections 3, 4 and 6). */
typedef struct {
  int32_t width, height;      /* raw frame size in pixels                                  */
  int32_t pitch_elems;        /* row pitch in uint16 elements; pitch_elems*2 % 16 == 0     */
  int32_t cfa;                /* Bayer layout; only 0 = RGGB is implemented                */
  double gain;                /* g_s, digital values per electron (Section 6, Eq. 17)      */
  double exposure;            /* t_s (Section 6, Eq. 16)                                   */
  double nd;                  /* exposure scaling n_s (Section 3)                          */
  double read_var;            /* Var r_s in DN^2, > 0 (Section 6.1, Eq. 20)                */
  double black;               /* bias b_s in DN (Section 6, Eq. 18)                        */
  double sat;                 /* saturation level in DN: y >= sat is excluded (Sec. 6.1)   */
  double affine[6];           /* T_s: sensor px -> reference px, row-major 2x3 (Sec. 4.2)  */
  /* Optional per-pixel calibration, HOST pointers to [height][width] arrays, NULL = use
   * the scalar above. Copied to the device by hdr_set_rig. */
  const float *bias_frame;    /* b_{s,i}                                                   */
  const float *prnu_frame;    /* a_{s,i}, > 0 (Section 6, Eq. 16)                          */
  const float *read_var_frame;/* Var r_{s,i}, > 0                                          */
  const uint16_t *sat_frame;  /* saturation frame (Section 6.1)                            */
} hdr_sensor_desc;

/* Reconstruction parameters (Sections 5.3 and 5.3.1). */
typedef struct {
  int32_t order;              /* polynomial order M in {0, 1, 2}                           */
  int32_t n_scales;           /* J in [1, HDR_MAX_SCALES]; 1 = a single window scale       */
  double sigma[HDR_MAX_SCALES]; /* R/B Gaussian scales in reference px, strictly ascending   */
  double green_ratio;         /* sigma_G / sigma_RB (Section 5.3.1: 1/sqrt(2))             */
  double trunc_k;             /* window radius k*sigma; the window is lowered by exp(-k^2/2) */
  double ici_gamma;           /* confidence-interval half-width in standard deviations     */
  double min_pivot;           /* a fit is usable only if every pivot of its equilibrated
                                 normal matrix exceeds this and it has >= (M+1)(M+2)/2 samples */
  double cond_fallback;       /* redo a solve in FP64 when the FP32 condition estimate exceeds
                                 this; <= 0 disables the fallback                           */
  int32_t out_w, out_h;       /* output size in pixels                                     */
  double out_affine[6];       /* output px -> reference px, row-major 2x3 (Section 4.2)    */
  int32_t out_dtype;          /* 0 = float32, 1 = float16; planar [3][out_h][out_w]        */
  int32_t accum;              /* 0 = plain FP32 moment sums, 1 = compensated (two-sum)     */
  int32_t tab_weights;        /* 1 = tabulated window weights where the rig allows (default),
                                 0 = never. Section 8: when every sensor is a pure translation of
                                 the reference frame and the output mapping is a translation at
                                 1x, all output pixels of one parity class see the same window
                                 offsets in each colour phase, so the window cells, offsets and
                                 weights are tabulated once per frame and the kernel reads them
                                 instead of searching and evaluating each window. The fit is the
                                 same; only rounding differs. */
  int32_t weight_mode;        /* noise weight of Eq. 6: 0 = K / s2, the inverse variance of the
                                 Gaussian likelihood the paper derives it from (default); 1 = K / s
                                 as printed in Section 5.2, for comparisons (Var C_0 then uses
                                 w^2 s2 = K^2). weight_mode 1 is supported by hdr_reconstruct,
                                 hdr_reconstruct_host and hdr_reconstruct_noalloc; the level maps,
                                 batches, the serving loop and the adaptive passes reject it with
                                 HDR_E_UNSUPPORTED. The paper's window exp(-|d|^2 / h) with
                                 h_G = h_RB / sqrt 2 is sigma = sqrt(h / 2) with
                                 green_ratio = 2^(-1/4). */
} hdr_params;

/* Fill *p with the defaults: order 2, scales {0.5, 0.8, 1.2, 1.8}, green_ratio 1/sqrt(2),
 * trunc_k 3, ici_gamma 2, min_pivot 1e-3, cond_fallback 1e6, identity output mapping,
 * float32 output, plain accumulation, tabulated weights allowed, inverse-variance weight.
 * out_w/out_h are set to 0 and must be filled. */
void hdr_params_default(hdr_params *p);

/* Create a context on CUDA device `device` (allocates its status word). */
hdr_status hdr_create(int device, hdr_ctx **out);

/* Destroy a context and every rig it holds. NULL is a no-op. */
void hdr_destroy(hdr_ctx *ctx);

/* Define (or replace) rig `rig_id` (0 <= rig_id < 64) of `n_sensors` (1..HDR_MAX_SENSORS)
 * sensors. Calibration and any per-pixel frames are copied to the device; the host
 * descriptors may be freed after the call. Replacing a rig waits for the device. */
hdr_status hdr_set_rig(hdr_ctx *ctx, int32_t rig_id, int32_t n_sensors, const hdr_sensor_desc *sensors);

/* Reconstruct one frame on `cuda_stream` (a cudaStream_t, NULL = the legacy default stream).
 *   raw_dev[s]  device pointer to sensor s's raw frame, [height][pitch_elems] uint16,
 *               16-byte aligned;
 *   out_dev     device pointer to the planar output [3][out_h][out_w] of out_dtype;
 *   choice_dev  optional device pointer [3][out_h][out_w] uint8: per channel the level
 *               used - 0..J-1 = order M at scale j, J+i = order M-1-i at the largest scale,
 *               255 = no sample (NaN output). NULL = not written.
 * Outputs of at least 152 x 256 pixels (one wave of 16 x 16 tiles) are reconstructed in two
 * launches: every raw sample is first converted once (Eq. 18, inverse of Eq. 20) into a buffer the
 * context owns (grown on demand, which waits for the device; calls on any stream are ordered
 * through it by an event), then the reconstruction copies converted footprints; smaller outputs
 * convert each footprint inside one launch. The results are the same either way.
 * Asynchronous: returns after queueing the launches. */
hdr_status hdr_reconstruct(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                           const uint16_t *const *raw_dev, void *out_dev, uint8_t *choice_dev,
                           void *cuda_stream);

/* Diagnostic variant of hdr_reconstruct: computes every level (no early exit) and also
 * writes levels_dev [3][J+M][out_h][out_w][2] float32 = (C_0, Var C_0) per level, NaN for
 * an unusable level. Slower; for parity and precision studies. */
hdr_status hdr_reconstruct_levels(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                  const uint16_t *const *raw_dev, void *out_dev, uint8_t *choice_dev,
                                  float *levels_dev, void *cuda_stream);

/* End-to-end variant with HOST buffers: copies raw_host[s] ([height][pitch_elems]) to
 * device staging owned by the context, reconstructs, copies the output back to out_host
 * (and choice to choice_host when non-NULL) and waits. Staging grows on demand. The output
 * runs in row bands of at least 8 tile rows, at most 16: the raw rows a band's windows reach are
 * copied in while the previous band is reconstructed, and each finished band is copied out
 * while the next one runs (copy streams owned by the context; pinned host buffers make the
 * copies asynchronous). Consecutive bands alternate between cuda_stream and a second stream of
 * the context, so that one band's CTAs fill the SMs the previous band's last wave leaves idle;
 * the work starts after earlier work on cuda_stream and cuda_stream is ordered after all of it. */
hdr_status hdr_reconstruct_host(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                const uint16_t *const *raw_host, void *out_host, uint8_t *choice_host,
                                void *cuda_stream);

/* Parameters of the adaptive reconstruction (Sections 5.4-5.5; the three passes are described
 * with hdr_reconstruct_adaptive below). */
typedef struct {
  double grad_sigma;   /* R/B scale of the pass-1 gradient fit (G uses green_ratio times it) */
  double window_sigma; /* Gaussian scale of pass 2, in output pixels; 3 window_sigma <= 10   */
  double alpha;        /* structure sensitivity in [0, 4] (0: gamma = 1)                      */
  double lambda1;      /* elongation regulariser in [1e-6, 1e6]                               */
  double lambda2;      /* scaling regulariser in [1e-12, 1e12]                                */
  double min_eig;      /* clamp of C's eigenvalues, 1e-6 <= min_eig <= max_eig <= 1e6; the   */
  double max_eig;      /*   staged window footprint grows by 1 / sqrt(min_eig)                */
  double grad_scale;   /* pass 2 uses grad_scale times the gradients, in (0, 1e6]: the paper
                          fixes lambda1 and lambda2 without stating the unit of the radiant
                          power, so this sets that unit (1 = the unit of the rig's calibration) */
} hdr_calpa_params;

/* One frame of a batch: rig, parameters and caller-owned device buffers, as for
 * hdr_reconstruct (raw_dev[s] for s < the rig's sensor count). With `calpa` set the frame is
 * reconstructed with the adaptive windows of Sections 5.4-5.5 exactly as hdr_reconstruct_adaptive
 * does (gradient and steering-matrix passes, then the steered fit); the two first passes run on
 * the batch's stream before its graph launch, in scratch the context owns (the serving loop keeps
 * a frame's scratch in its pool block). */
typedef struct {
  int32_t rig_id;
  const hdr_params *params;
  const uint16_t *raw_dev[HDR_MAX_SENSORS];
  void *out_dev;
  uint8_t *choice_dev;          /* optional level map, NULL = not written */
  const hdr_calpa_params *calpa; /* NULL = the window of Eq. 8; else the adaptive window */
} hdr_frame;

/* Launch configuration of a batched reconstruction. Both forms run as one CUDA-graph launch:
 *  form 0: one grid per frame (the single-frame kernel over that frame's tiles), all frames as
 *          independent branches of one graph, so that small frames fill the tails of large ones;
 *  form 1: one persistent kernel per polynomial order whose CTAs take tiles of every frame of that
 *          order from a device-wide queue (tile list and counters in device memory). */
typedef struct {
  int32_t tile_h;               /* output rows per tile: 8 (128-thread CTAs) or 16 (256 threads) */
  int32_t ctas_per_sm;          /* form 1: persistent CTAs per SM; 0 = as many as fit            */
  int32_t cost_order;           /* 1 = the most expensive frames first, 0 = the given order      */
  int32_t form;                 /* 0 or 1, see above                                              */
  int32_t px_per_thread;        /* form 0: output pixels per thread, 0 or 1 = one; 2 = two, each
                                   thread its pixels one after the other (tile_h 16 only: 16-row
                                   tiles of 128 threads); adaptive frames always take one        */
  int32_t stages;               /* form 0: staging buffers per CTA, 0 or 1 = one tile per CTA; 2 =
                                   each CTA takes four tiles and bulk-copies the next tile's raw
                                   footprints into a second buffer while it reconstructs the
                                   current one (one pixel per thread; frames with compensated sums
                                   or adaptive windows take one). Results are identical.          */
} hdr_batch_config;

/* Reconstruct n_frames (1..4096) frames of any sizes, rigs, orders and scales in one graph launch
 * on `cuda_stream`. A graph is recorded once per launch shape and replayed: form 0 updates the
 * kernel parameters of its nodes; form 1 copies the frame and tile tables from pinned staging
 * owned by the context (double-buffered: the call waits only if the launch before the previous
 * one is still reading) and clears the tile counters. `cfg` NULL = the configuration
 * hdr_tune_batch found for batches of this kind, else the default {16, 0, 1, 0}. All frames must
 * use the same `accum` and weight_mode 0 (HDR_E_UNSUPPORTED otherwise). Asynchronous like
 * hdr_reconstruct. Form 0 results are identical to reconstructing each frame with hdr_reconstruct
 * (hdr_reconstruct_adaptive for frames with `calpa`); form 1 walks every window once per scale
 * and searches it (no tabulated weights), so its sums round differently: the same fit within the
 * parity tolerance. A batch with adaptive frames always runs form 0. */
hdr_status hdr_reconstruct_batch(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames,
                                 const hdr_batch_config *cfg, void *cuda_stream);

/* Autotuner: times every candidate configuration (form, tile height 8/16, pixels per thread,
 * staging buffers, CTAs per SM, frame order) on this batch, keeps the fastest for batches of the same kind (orders present, largest
 * sensor count, scale count, output-size bucket) and writes it to *best. Synchronous. */
hdr_status hdr_tune_batch(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames, hdr_batch_config *best,
                          void *cuda_stream);

/* ---------------------------------------------------------------- serving
 * A request loop over one context. The paper overlaps the transfer of one frame with the
 * reconstruction of the previous one on two streams (Section 8); this loop generalises that to
 * many concurrent video streams. Frames of any size, rig and order are submitted from any
 * thread. A scheduler thread admits them in arrival order while a slot and room in the server's
 * device-memory pool are free, copies their raw frames into the pool on a copy stream, and
 * repeatedly launches one batched step over the pending tiles of the admitted frames, oldest
 * frame first, at most step_tiles per step, with up to three steps queued on the device: frames that
 * arrive while a step runs join a later one (continuous batching at tile granularity; with
 * hdr_server_config.order 1 the frames with the least remaining work go first). When a step
 * completes, the output rows of its frames whose tiles are all done are copied back to the host
 * buffers on a second copy stream; a frame whose last rows have landed completes and its memory
 * returns to the pool. Each pixel is computed as hdr_reconstruct (an adaptive request: as
 * hdr_reconstruct_adaptive) computes it, whatever else shares the step; an adaptive request runs
 * its gradient and steering-matrix passes in the step that takes its first tiles, into scratch in
 * its pool block (20 bytes per output pixel), and needs the default tile height (16). The server uses its context exclusively until hdr_server_destroy (no
 * other call on that context meanwhile); rigs must be set before serving starts. A device-side
 * error fails every request whose tiles were on the device when it was seen. */
typedef struct hdr_server hdr_server;

typedef struct {
  int32_t max_frames;           /* frames admitted at once (slots), >= 1                         */
  uint64_t pool_bytes;          /* device pool for raw frames, outputs and level maps            */
  int32_t step_tiles;           /* tile budget of one step; 0 = every pending tile               */
  hdr_batch_config batch;       /* launch configuration of the steps (tile_h 0 = default)        */
  int32_t order;                /* tiles of a step: 0 = frames in admission order (first come,
                                   first served: the lowest worst-case latency at equal relative
                                   deadlines); 1 = the least remaining work first (tiles x sensors:
                                   a lower median, a longer tail for the largest frames)          */
} hdr_server_config;

typedef struct {
  int32_t rig_id;
  hdr_params params;            /* copied at submission                                           */
  const uint16_t *raw_host[HDR_MAX_SENSORS]; /* host raw frames [height][pitch_elems]; read until
                                   the request completes (pinned memory copies fastest)           */
  void *out_host;               /* host output [3][out_h][out_w] of out_dtype, written at completion */
  uint8_t *choice_host;         /* optional host level map, NULL = not produced                  */
  int32_t stream_id;            /* caller's video stream, for its own bookkeeping               */
  int32_t adaptive;             /* 1 = the adaptive reconstruction (Sections 5.4-5.5) with calpa */
  hdr_calpa_params calpa;       /* copied at submission; read when adaptive = 1                  */
} hdr_request;

typedef struct {
  hdr_status status;            /* HDR_OK once the output is in out_host                         */
  double queue_ms;              /* submission -> admission                                       */
  double total_ms;              /* submission -> output in host memory                           */
  int32_t steps;                /* batched steps the frame's tiles ran in                        */
} hdr_result;

typedef struct {
  uint64_t completed, submitted;
  double p50_ms, p99_ms, max_ms;    /* of total_ms over completed requests                    */
  double mean_queue_ms;
  uint64_t steps, output_pixels;
  double busy_s;                    /* wall time between the first admission and the last completion */
  double gpu_step_ms;               /* device time of the batched steps, summed (each from the start of
                                       its first kernel to the end of its last)                   */
  double gpu_gap_ms;                /* device time between the end of one step and the start of the
                                       next, summed: the compute stream idles there               */
  double host_step_ms_mean;         /* host time to build and launch one step (planning, graph
                                       update, launch), mean and maximum                          */
  double host_step_ms_max;
} hdr_server_stats;

/* Start a server on `ctx` (allocates the pool, streams and the scheduler thread). */
hdr_status hdr_server_create(hdr_ctx *ctx, const hdr_server_config *cfg, hdr_server **out);
/* Queue one frame and return its ticket; the request is validated here (HDR_E_INVALID) and
 * HDR_E_UNSUPPORTED is returned if the frame can never fit the pool. */
hdr_status hdr_submit(hdr_server *srv, const hdr_request *req, uint64_t *ticket);
/* Wait up to timeout_ms (< 0 = forever) for a ticket. HDR_E_BUSY if it is not done by then; the
 * result of a finished ticket is returned once and then forgotten. */
hdr_status hdr_poll(hdr_server *srv, uint64_t ticket, int32_t timeout_ms, hdr_result *result);
/* Latency and throughput of every request completed so far. */
hdr_status hdr_server_stats_get(hdr_server *srv, hdr_server_stats *stats);
/* Finish every submitted request, stop the scheduler and free the server (not the context);
 * results not yet polled are discarded. */
void hdr_server_destroy(hdr_server *srv);

/* Wait for `cuda_stream`, then read and clear the context's device status word.
 * Returns HDR_E_TIMEOUT or HDR_E_INTERNAL if a kernel recorded one, HDR_E_CUDA on a
 * CUDA error, else HDR_OK. */
hdr_status hdr_check(hdr_ctx *ctx, void *cuda_stream);

/* Self-test of failure detection (no counterpart in the paper): launches one block whose bounded
 * wait can never complete (an mbarrier expecting bytes that no copy delivers); the wait gives up
 * within about 0.1 s and sets the same device status a reconstruction whose staging copies never
 * land would set. Nothing faults or hangs: the next hdr_check on that stream returns HDR_E_TIMEOUT
 * and clears the status, reconstructions launched before that check retire without writing, and
 * the context stays usable. Asynchronous on `cuda_stream`. */
hdr_status hdr_selftest_timeout(hdr_ctx *ctx, void *cuda_stream);

/* Message of the calling thread's last failed call ("" if none). */
const char *hdr_last_error(void);

/* ---------------------------------------------------------------- calibration (Section 6.2)
 * Estimates of the camera parameters the reconstruction needs, from stacks of raw frames of one
 * sensor: black frames (lens covered) and flat fields. All pointers are DEVICE pointers; frames
 * are uint16 [height][pitch_elems], output and statistics frames float32 [height][width]. */

/* Per-pixel mean and unbiased variance over n_frames (2..4096) frames, frame f at
 * frames_dev + f * frame_stride_elems. From black frames these are the bias frame b_{s,i} and
 * the read-noise variance Var r_{s,i}; from flat fields, E[y_{s,i}] and Var y_{s,i}. The sums
 * are exact integers, so each value is one FP64 rounding of the exact statistic, then FP32.
 * frames_dev must be 16-byte aligned; pitch_elems and frame_stride_elems multiples of 8, the
 * pitch at least the width rounded up to 8. Asynchronous on `cuda_stream`. */
hdr_status hdr_calib_stack_stats(hdr_ctx *ctx, const uint16_t *frames_dev, int32_t n_frames, int32_t width,
                                 int32_t height, int32_t pitch_elems, int64_t frame_stride_elems, float *mean_dev,
                                 float *var_dev, void *cuda_stream);

/* Sensor gain by Eq. 21, (Var y - Var b) / (E[y] - E[b]) = g_s, pooled as the ratio of the sums
 * over usable pixels: flat mean at least min_signal DN above the black mean and below max_level
 * DN (away from saturation). *gain = NaN if no pixel is usable; *n_used (optional) = the count.
 * Synchronous; the summation order is fixed, so repeated calls give identical results. */
hdr_status hdr_calib_gain(hdr_ctx *ctx, const float *flat_mean, const float *flat_var, const float *black_mean,
                          const float *black_var, int32_t width, int32_t height, double min_signal, double max_level,
                          double *gain, int64_t *n_used, void *cuda_stream);

/* Exposure scaling n_s (Section 6.2): the spatial mean over pixels usable in both sensors of
 * rho_i = ((E y - b) / (g t))_s / ((E y - b) / (g t))_ref, the pixel-wise ratio of the radiant-power
 * estimates of Eq. 18 (with n = a = 1) of sensor s to those of a reference sensor seeing the same
 * flat field. When prnu_dev is non-NULL it receives the non-uniformity a_{s,i} = rho_i / n_s at
 * usable pixels and 1 elsewhere (the reference sensor's own non-uniformity is taken as 1). Use
 * exposure times that expose both sensors well. Synchronous; *nd = NaN if no pixel is usable. */
hdr_status hdr_calib_exposure(hdr_ctx *ctx, const float *flat_mean, const float *black_mean, double gain,
                              double exposure, const float *ref_flat_mean, const float *ref_black_mean,
                              double ref_gain, double ref_exposure, int32_t width, int32_t height, double min_signal,
                              double max_level, double *nd, float *prnu_dev, int64_t *n_used, void *cuda_stream);

/* ---------------------------------------------------------------- adaptive windows (Sections 5.4-5.5)
 * CALPA: the window of every fit is steered by the local image structure. Three passes, each a
 * kernel on the caller's stream:
 *   1. gradients: the isotropic order-1 fit of the green channel at scale grad_sigma; its two
 *      linear coefficients are the radiance gradient at the output pixel (Section 5.5 takes the
 *      structure from G, which has twice the R/B sample density);
 *   2. steering matrix: per output pixel, from the Gaussian-weighted gradients of the output
 *      pixels within 3 window_sigma (M = the number of those inside the image), the singular
 *      values s1 >= s2 and the dominant direction u1 of the gradient matrix give the elongation
 *      sigma = (s1 + lambda1) / (s2 + lambda1), the scaling gamma = ((s1 s2 + lambda2) / M)^alpha
 *      and C = gamma (sigma u1 u1^T + u2 u2^T / sigma), whose eigenvalues are then clamped to
 *      [min_eig, max_eig];
 *   3. the reconstruction of Sections 5.1-5.3 with the window exp(-d^T C d / (2 sigma_j^2)) on
 *      d^T C d < (k sigma_j)^2 in place of Eq. 8's, lowered by exp(-k^2/2) as there: narrow across
 *      an edge, long along it.
 * Readings taken where the paper leaves the form open: C enters the exponent directly (no
 * determinant normalisation: the fit's solution does not depend on a constant factor of the
 * weights), the weights of pass 2 are Gaussian in the output-pixel distance, and the clamp of
 * C's eigenvalues bounds every window between k sigma_J / sqrt(max_eig) and k sigma_J / sqrt(min_eig). */
/* hdr_calpa_params: defined with the frame description above. */

/* Defaults: grad_sigma 1.2, window_sigma 1, alpha 0.3, lambda1 1, lambda2 1e-3 (as the paper
 * fixes them), eigenvalues clamped to [0.25, 16], grad_scale 0.1 (chosen on synthetic HDR scenes
 * whose radiance spans 1e-2 to 1e4 in the calibration's unit). */
void hdr_calpa_params_default(hdr_calpa_params *c);

/* Pass 1. grad_dev: device [out_h][out_w][2] float32, the (x, y) gradient in radiance per output
 * reference pixel at each output pixel; 0 where the fit is not usable (fewer than 3 samples, or
 * a pivot at or below min_pivot). params supplies the rig geometry, output mapping, green_ratio,
 * trunc_k, min_pivot, cond_fallback and accum; its order, scales and tab_weights are not used.
 * Asynchronous on `cuda_stream`. */
hdr_status hdr_calpa_gradients(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const hdr_calpa_params *calpa,
                               const uint16_t *const *raw_dev, float *grad_dev, void *cuda_stream);

/* Pass 2. grad_dev as pass 1 writes it; metric_dev: device [out_h][out_w][3] float32 = C11, C12,
 * C22. The structure tensor is summed and its eigenvalues formed in FP64 (the small one of a
 * straight edge is a difference of large sums); the rest runs in FP32, so gradients up to about
 * 1e18 in magnitude are supported. Asynchronous on `cuda_stream`. */
hdr_status hdr_calpa_metric(hdr_ctx *ctx, int32_t out_w, int32_t out_h, const hdr_calpa_params *calpa,
                            const float *grad_dev, float *metric_dev, void *cuda_stream);

/* Pass 3: hdr_reconstruct with the steered window of metric_dev ([out_h][out_w][3], as pass 2
 * writes it; any symmetric C whose eigenvalues are at least calpa->min_eig may be given: a window
 * reaching beyond the footprint staged for that bound is reported by hdr_check as HDR_E_INTERNAL).
 * Asynchronous on `cuda_stream`. */
hdr_status hdr_reconstruct_steered(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                   const hdr_calpa_params *calpa, const uint16_t *const *raw_dev,
                                   const float *metric_dev, void *out_dev, uint8_t *choice_dev, void *cuda_stream);

/* The three passes in one call, with the gradient and metric planes in scratch owned by the
 * context (grown on demand, which waits for the device; calls that share a context must be
 * serialised on one stream). Asynchronous on `cuda_stream`. */
hdr_status hdr_reconstruct_adaptive(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                    const hdr_calpa_params *calpa, const uint16_t *const *raw_dev, void *out_dev,
                                    uint8_t *choice_dev, void *cuda_stream);

/* hdr_reconstruct_adaptive from HOST buffers: copies raw_host[s] ([height][pitch_elems]) into the
 * context's staging, runs the three passes, copies the output (and choice when non-NULL) back to
 * out_host and waits. Copies and passes run in order on `cuda_stream` (pinned host buffers make the
 * copies asynchronous to the host). */
hdr_status hdr_reconstruct_adaptive_host(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                         const hdr_calpa_params *calpa, const uint16_t *const *raw_host,
                                         void *out_host, uint8_t *choice_host, void *cuda_stream);

/* Size of the fixed device array that hdr_reconstruct_noalloc uses as scratch. */
#define HDR_NOALLOC_SCRATCH_BYTES (4u << 20)

/* Reconstruct one frame without allocating anything, for callers that cannot allocate device
 * memory: a real-time capture thread that must not enter the allocator, or a host program whose
 * GPU memory is wholly reserved by another runtime's pool. The paper has no counterpart; this is
 * a convenience of this library. No context is needed and nothing is allocated (no cudaMalloc,
 * no cudaFree, no allocating library routine); the call is synchronous.
 *   device      CUDA device to run on (made current by the call);
 *   sensors     the rig, as for hdr_set_rig (per-pixel frames are HOST pointers, copied on each call);
 *   params, raw_dev, out_dev, choice_dev, cuda_stream   as for hdr_reconstruct.
 * Scratch: the kernel's status word and the rig's per-pixel calibration frames are placed in one
 * fixed device array of HDR_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits. A call whose frames do not fit (256 bytes plus each frame rounded up to 256
 * bytes) is rejected with HDR_E_UNSUPPORTED before any GPU work. The array keeps the last call's
 * contents; each call clears the status word and rewrites the frames it uses. All calls share the
 * one array per device, so calls that overlap on the GPU (other threads or other streams) race:
 * serialise them. The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and the tensor-map encoder; make that first call before any stream
 * capture. Returns HDR_E_TIMEOUT / HDR_E_INTERNAL for device-side errors, like hdr_check. */
hdr_status hdr_reconstruct_noalloc(int device, int32_t n_sensors, const hdr_sensor_desc *sensors,
                                   const hdr_params *params, const uint16_t *const *raw_dev, void *out_dev,
                                   uint8_t *choice_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* HDR_LPA_H */
