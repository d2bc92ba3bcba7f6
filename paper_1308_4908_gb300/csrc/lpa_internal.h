// Library-internal entry points shared between the host translation units (not the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "hdr_lpa.h"

// One batched launch over tiles [ranges[f].x, ranges[f].y) of each frame (all tiles when ranges
// is NULL); the implementation behind hdr_reconstruct_batch. Adaptive frames (calpa set) keep
// their gradients and steering matrices in scratch[f] (5 floats per output pixel), or, when
// scratch is NULL, in scratch the context owns; their first two passes run in the launch that
// takes their first tile. Frames converted ahead of the reconstruction (lpa_conv_eligible) read
// their converted planes from conv[f] (lpa_conv_elems float2), which lpa_convert_frame has filled
// when conv_done, else which the launch that takes their first tile fills; with conv NULL, the
// context's conversion buffer. With two staging buffers, or in form 1, every frame converts its
// footprints in the kernel.
hdr_status lpa_batch_run(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames, const int2 *ranges,
                         const hdr_batch_config *cfg, cudaStream_t stream, float *const *scratch = nullptr,
                         float2 *const *conv = nullptr, bool conv_done = false);
// Convert one frame into conv (lpa_conv_elems float2) on `st`.
hdr_status lpa_convert_frame(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                             float2 *conv, cudaStream_t st);
// Whether a frame with these parameters is converted in a pass of its own before its
// reconstruction, and the float2 elements of its converted planes for a rig.
bool lpa_conv_eligible(const hdr_params *p, bool adaptive);
size_t lpa_conv_elems(const hdr_ctx *ctx, int rig_id);
// Validate adaptive-reconstruction parameters.
hdr_status lpa_check_calpa(const hdr_calpa_params *c);
// Passes 1 and 2 of the adaptive reconstruction of one frame into scratch (gradients [2 npx],
// then steering matrices [3 npx]) on `st`.
hdr_status lpa_calpa_prepare(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const hdr_calpa_params *calpa,
                             const uint16_t *const *raw_dev, float *scratch, cudaStream_t st);
int lpa_ctx_device(const hdr_ctx *ctx);
// Sensors of a rig (0 if the rig is not defined) and each sensor's raw pitch and height.
int lpa_ctx_rig_sensors(const hdr_ctx *ctx, int rig_id);
void lpa_ctx_rig_sizes(const hdr_ctx *ctx, int rig_id, int *pitch, int *height);
// Record a message for hdr_last_error and return st; validate parameters.
hdr_status lpa_fail(hdr_status st, const char *msg);
hdr_status lpa_check_params(const hdr_params *p);
// Read and clear the context's device status word without waiting for any stream (launches
// still running may set it later); HDR_E_TIMEOUT / HDR_E_INTERNAL as hdr_check reports them.
hdr_status lpa_take_status(hdr_ctx *ctx);
// Plan and launch one frame with the kernel of `mode` (LPA_STEERED: aux = the steering matrices,
// the window's reach grown by `reach`; LPA_GRADIENTS: aux receives the gradients and no output
// is written). The window is always searched. ahead: the frame is converted into the context's
// conversion buffer first where lpa_conv_eligible (not while a batch holds plans into it).
hdr_status lpa_launch_mode(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                           int mode, float *aux, double reach, void *out_dev, uint8_t *choice_dev, cudaStream_t st,
                           bool ahead);
// Staging reach of the steered window for these adaptive parameters (1 / sqrt(min_eig)).
double lpa_calpa_reach(const hdr_calpa_params *calpa);
// Device scratch of at least `bytes` owned by the context for the adaptive reconstruction
// (growing it waits for the device).
hdr_status lpa_ctx_calpa_scratch(hdr_ctx *ctx, size_t bytes, void **ptr);
