// Per-order kernel launchers (one translation unit each, compiled in parallel).
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <set>
#include <utility>

#include "lpa_launch.h"

// Largest dynamic shared memory a block of the current device may opt in to.
inline int lpa_smem_optin() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64 && cache[dev]) return cache[dev];
  int v = 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  if (dev >= 0 && dev < 64) cache[dev] = v;
  return v;
}

// Opt a kernel in to the largest dynamic shared memory its static shared memory leaves, never to
// one launch's size: a graph recorded with a larger launch stays valid whatever smaller launches
// of the same kernel run in between.
// Done once per kernel and device (the attribute persists).
inline cudaError_t lpa_opt_in(const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({fn, dev})) return cudaSuccess;
  }
  cudaFuncAttributes a;
  e = cudaFuncGetAttributes(&a, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lpa_smem_optin() - (int)a.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  done.insert({fn, dev});
  return cudaSuccess;
}

// One CTA per tile of L with the kernel of L.mode (cudaErrorInvalidConfiguration where that mode
// is not instantiated for the order or tile height).
cudaError_t lpa_launch_order0(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order1(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);
cudaError_t lpa_launch_order2(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st);

// The single-frame kernel of order M for that configuration (for graph kernel nodes): mode is one
// of LPA_SEARCHED .. LPA_TABULATED_F32, tile_h the rows of a tile, px the pixels per thread (the CTA
// has 16 x tile_h / px threads), stages the staging buffers per CTA (the grid is then
// lpa_grid_ctas(tiles, stages)); nullptr where that combination is not instantiated.
const void *lpa_kernel_order0(bool comp, bool diag, int mode, int tile_h, int px, int stages);
const void *lpa_kernel_order1(bool comp, bool diag, int mode, int tile_h, int px, int stages);
const void *lpa_kernel_order2(bool comp, bool diag, int mode, int tile_h, int px, int stages);
inline const void *lpa_kernel(int order, bool comp, bool diag, int mode, int tile_h, int px = 1, int stages = 1) {
  return order == 0   ? lpa_kernel_order0(comp, diag, mode, tile_h, px, stages)
         : order == 1 ? lpa_kernel_order1(comp, diag, mode, tile_h, px, stages)
                      : lpa_kernel_order2(comp, diag, mode, tile_h, px, stages);
}

// Conversion of rows R of every sensor of L into its planes (LpaSensorK::conv), for a plan with
// conv = 1; lit: the printed noise weight (square root of the inverse variance).
cudaError_t lpa_launch_convert(const LpaLaunch &L, const LpaRows &R, bool lit, cudaStream_t st);
// The conversion kernel (parameters: LpaLaunch, LpaRows; 256 threads) and its grid, for graph nodes.
const void *lpa_convert_kernel(bool lit);
dim3 lpa_convert_grid(const LpaLaunch &L, const LpaRows &R);

// Persistent launch of order M over its segment of a many-frame tile list (tile height 8 or 16).
cudaError_t lpa_launch_batch_order0(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st);
cudaError_t lpa_launch_batch_order1(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st);
cudaError_t lpa_launch_batch_order2(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st);
// Resident CTAs per SM of that kernel with that much dynamic shared memory (0 on error).
int lpa_batch_ctas_per_sm_order0(bool comp, int tile_h, uint32_t smem_bytes);
int lpa_batch_ctas_per_sm_order1(bool comp, int tile_h, uint32_t smem_bytes);
int lpa_batch_ctas_per_sm_order2(bool comp, int tile_h, uint32_t smem_bytes);

inline cudaError_t lpa_launch_batch(int order, const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st) {
  return order == 0   ? lpa_launch_batch_order0(B, comp, tile_h, grid, st)
         : order == 1 ? lpa_launch_batch_order1(B, comp, tile_h, grid, st)
                      : lpa_launch_batch_order2(B, comp, tile_h, grid, st);
}
inline int lpa_batch_ctas_per_sm(int order, bool comp, int tile_h, uint32_t smem_bytes) {
  return order == 0   ? lpa_batch_ctas_per_sm_order0(comp, tile_h, smem_bytes)
         : order == 1 ? lpa_batch_ctas_per_sm_order1(comp, tile_h, smem_bytes)
                      : lpa_batch_ctas_per_sm_order2(comp, tile_h, smem_bytes);
}

// One-thread self-test of the bounded wait (sets LPA_ERR_TIMEOUT in *status).
cudaError_t lpa_launch_selftest_wait(unsigned int *status, cudaStream_t st);
