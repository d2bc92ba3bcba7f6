// Library-internal entry points shared between the host translation units (not the C ABI).
#pragma once
#include <cuda_runtime.h>

#include "hdr_lpa.h"

// One persistent launch over tiles [ranges[f].x, ranges[f].y) of each frame (all tiles when
// ranges is NULL); the implementation behind hdr_reconstruct_batch.
hdr_status lpa_batch_run(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames, const int2 *ranges,
                         const hdr_batch_config *cfg, cudaStream_t stream);
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
