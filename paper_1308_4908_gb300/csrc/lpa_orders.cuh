// Launchers of the reconstruction kernels of one polynomial order (included once per order by
// lpa_m0.cu, lpa_m1.cu and lpa_m2.cu, which compile in parallel).
//
// Instantiated per order: the searched window (Eq. 8) with and without the level maps, the
// tabulated window (Section 8), tile heights 8 and 16, and 16-row tiles with two pixels per
// thread; the steered window (Section 5.4) and the printed noise weight K / s at tile height 16;
// the gradient pass (Section 5.4) for order 1 only.
#pragma once
#include "lpa_dispatch.h"
#include "lpa_kernel.cuh"

namespace lpa_orders {

template <int ORDER, int MODE, int TH, int PX>
constexpr bool instantiated() {
  if (PX == 2)  // two pixels per thread: 16-row tiles of 8-row CTAs, the windows batches use
    return TH == 8 && (MODE == LPA_SEARCHED || MODE == LPA_SEARCHED_F32 || lpa_mode_tab(MODE));
  if (MODE == LPA_GRADIENTS) return ORDER == 1 && TH == 16;
  if (lpa_mode_steered(MODE) || MODE == LPA_LITERAL) return TH == 16;
  return true;
}

template <int ORDER, bool COMP, bool DIAG, int TH, int MODE, int PX, int STAGES>
const void *kernel_fn() {
  if constexpr (!instantiated<ORDER, MODE, TH, PX>() ||
                (DIAG && (PX != 1 || (MODE != LPA_SEARCHED && MODE != LPA_SEARCHED_F32))) ||
                (STAGES == 2 && (DIAG || PX != 1 || !lpa_stages2_built(MODE, COMP))))
    return nullptr;
  else return (const void *)lpa::lpa_reconstruct<ORDER, COMP, DIAG, TH, MODE, PX, STAGES>;
}

template <int ORDER, bool COMP, bool DIAG, int TH, int PX = 1, int STAGES = 1>
const void *kernel_mode(int mode) {
  switch (mode) {
    case LPA_SEARCHED: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_SEARCHED, PX, STAGES>();
    case LPA_TABULATED: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_TABULATED, PX, STAGES>();
    case LPA_STEERED: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_STEERED, PX, STAGES>();
    case LPA_GRADIENTS: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_GRADIENTS, PX, STAGES>();
    case LPA_LITERAL: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_LITERAL, PX, STAGES>();
    case LPA_SEARCHED_F32: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_SEARCHED_F32, PX, STAGES>();
    case LPA_STEERED_F32: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_STEERED_F32, PX, STAGES>();
    case LPA_TABULATED_F32: return kernel_fn<ORDER, COMP, DIAG, TH, LPA_TABULATED_F32, PX, STAGES>();
    default: return nullptr;
  }
}

// The single-frame kernel of this order for a configuration (tile_h rows per tile, px pixels per
// thread: CTAs of 16 x tile_h / px threads; stages staging buffers per CTA); nullptr if not
// instantiated.
template <int ORDER>
const void *kernel(bool comp, bool diag, int mode, int tile_h, int px, int stages) {
  if (stages == 2) {
    if (px != 1 || diag || comp) return nullptr;
    return tile_h == 8 ? kernel_mode<ORDER, false, false, 8, 1, 2>(mode) : kernel_mode<ORDER, false, false, 16, 1, 2>(mode);
  }
  if (stages != 1) return nullptr;
  if (px == 2) {
    if (tile_h != 16 || diag) return nullptr;
    return comp ? kernel_mode<ORDER, true, false, 8, 2>(mode) : kernel_mode<ORDER, false, false, 8, 2>(mode);
  }
  if (px != 1) return nullptr;
  if (tile_h == 8) {
    if (comp) return diag ? kernel_mode<ORDER, true, true, 8>(mode) : kernel_mode<ORDER, true, false, 8>(mode);
    return diag ? kernel_mode<ORDER, false, true, 8>(mode) : kernel_mode<ORDER, false, false, 8>(mode);
  }
  if (comp) return diag ? kernel_mode<ORDER, true, true, 16>(mode) : kernel_mode<ORDER, true, false, 16>(mode);
  return diag ? kernel_mode<ORDER, false, true, 16>(mode) : kernel_mode<ORDER, false, false, 16>(mode);
}

// One CTA per tile of L (tiles L.tile0 .. L.tile0 + grid - 1) with the kernel L.mode selects.
template <int ORDER>
cudaError_t launch(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  // the diagnostic (level maps) kernel is instantiated for the searched window only
  const int px = L.px > 1 ? L.px : 1;
  const int stages = L.stages > 1 ? L.stages : 1;
  const void *fn = kernel<ORDER>(comp, diag, L.mode, L.tile_h, px, stages);
  if (!fn) return cudaErrorInvalidConfiguration;
  cudaError_t e = lpa_opt_in(fn);
  if (e != cudaSuccess) return e;
  const int grid = lpa_grid_ctas(L.tile_count > 0 ? L.tile_count : L.tiles_x * L.tiles_y - L.tile0, stages);
  void *args[] = {const_cast<LpaLaunch *>(&L)};
  return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3((unsigned)(LPA_TILE * L.tile_h / px)), args, L.smem_bytes, st);
}

template <int ORDER, bool COMP, int TH>
cudaError_t launch_batch_t(const LpaBatch &B, int grid, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct_batch<ORDER, COMP, TH>;
  cudaError_t e = lpa_opt_in((const void *)k);
  if (e != cudaSuccess) return e;
  k<<<grid, LPA_TILE * TH, B.smem_bytes, st>>>(B);
  return cudaGetLastError();
}

template <int ORDER>
cudaError_t launch_batch(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st) {
  if (tile_h == 8)
    return comp ? launch_batch_t<ORDER, true, 8>(B, grid, st) : launch_batch_t<ORDER, false, 8>(B, grid, st);
  return comp ? launch_batch_t<ORDER, true, 16>(B, grid, st) : launch_batch_t<ORDER, false, 16>(B, grid, st);
}

template <int ORDER, bool COMP, int TH>
int fit_t(uint32_t smem_bytes) {
  auto k = lpa::lpa_reconstruct_batch<ORDER, COMP, TH>;
  int n = 0;
  if (lpa_opt_in((const void *)k) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, LPA_TILE * TH, smem_bytes) != cudaSuccess) return 0;
  return n;
}

template <int ORDER>
int batch_ctas_per_sm(bool comp, int tile_h, uint32_t smem_bytes) {
  if (tile_h == 8) return comp ? fit_t<ORDER, true, 8>(smem_bytes) : fit_t<ORDER, false, 8>(smem_bytes);
  return comp ? fit_t<ORDER, true, 16>(smem_bytes) : fit_t<ORDER, false, 16>(smem_bytes);
}

}  // namespace lpa_orders

// The extern entry points of order N (declared in lpa_dispatch.h).
#define LPA_ORDER_ENTRY_POINTS(N)                                                                           \
  cudaError_t lpa_launch_order##N(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {             \
    return lpa_orders::launch<N>(L, comp, diag, st);                                                       \
  }                                                                                                        \
  const void *lpa_kernel_order##N(bool comp, bool diag, int mode, int tile_h, int px, int stages) {        \
    return lpa_orders::kernel<N>(comp, diag, mode, tile_h, px, stages);                                    \
  }                                                                                                        \
  cudaError_t lpa_launch_batch_order##N(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st) { \
    return lpa_orders::launch_batch<N>(B, comp, tile_h, grid, st);                                         \
  }                                                                                                        \
  int lpa_batch_ctas_per_sm_order##N(bool comp, int tile_h, uint32_t smem_bytes) {                         \
    return lpa_orders::batch_ctas_per_sm<N>(comp, tile_h, smem_bytes);                                     \
  }
