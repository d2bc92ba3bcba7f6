// Per-order kernel launchers (one translation unit each, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include "lpa_launch.h"

cudaError_t lpa_launch_order0(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order1(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order2(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
