// Per-order kernel launchers (one translation unit each, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include "lpa_launch.h"

cudaError_t lpa_launch_order0(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order1(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order2(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);

// Persistent launch over the tiles of several frames (tile height 8 or 16).
cudaError_t lpa_launch_batch(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st);
// Resident CTAs per SM of the batch kernel for that configuration (0 on error).
int lpa_batch_ctas_per_sm(bool comp, int tile_h, uint32_t smem_bytes);
