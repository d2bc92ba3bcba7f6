// Instantiations of the persistent many-frame kernel (orders 0-2 dispatched per tile).
#include "lpa_dispatch.h"
#include "lpa_kernel.cuh"

template <bool COMP, int TH>
static cudaError_t launch_batch_t(const LpaBatch &B, int grid, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct_batch<COMP, TH>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem_bytes);
  if (e != cudaSuccess) return e;
  k<<<grid, LPA_TILE * TH, B.smem_bytes, st>>>(B);
  return cudaGetLastError();
}

cudaError_t lpa_launch_batch(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st) {
  if (tile_h == 8) return comp ? launch_batch_t<true, 8>(B, grid, st) : launch_batch_t<false, 8>(B, grid, st);
  return comp ? launch_batch_t<true, 16>(B, grid, st) : launch_batch_t<false, 16>(B, grid, st);
}

int lpa_batch_ctas_per_sm(bool comp, int tile_h, uint32_t smem_bytes) {
  int n = 0;
  cudaError_t e;
  if (tile_h == 8) {
    auto k = comp ? lpa::lpa_reconstruct_batch<true, 8> : lpa::lpa_reconstruct_batch<false, 8>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, LPA_TILE * 8, smem_bytes);
  } else {
    auto k = comp ? lpa::lpa_reconstruct_batch<true, 16> : lpa::lpa_reconstruct_batch<false, 16>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, LPA_TILE * 16, smem_bytes);
  }
  return e == cudaSuccess ? n : 0;
}
