// Instantiations of the single-frame and the persistent many-frame reconstruction kernels for
// polynomial order M = 1.
#include "lpa_dispatch.h"
#include "lpa_kernel.cuh"

template <bool COMP, bool DIAG, int TH, bool TAB>
static cudaError_t launch_one(const LpaLaunch &L, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct<1, COMP, DIAG, TH, TAB>;
  cudaError_t e = lpa_opt_in((const void *)k);
  if (e != cudaSuccess) return e;
  const int grid = L.tile_count > 0 ? L.tile_count : L.tiles_x * L.tiles_y - L.tile0;
  k<<<grid, LPA_TILE * TH, L.smem_bytes, st>>>(L);
  return cudaGetLastError();
}

template <int TH>
static cudaError_t launch_th(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  const bool tab = L.tab_cells != nullptr;  // the diagnostic (levels) path always searches
  if (comp) {
    if (diag) return launch_one<true, true, TH, false>(L, st);
    return tab ? launch_one<true, false, TH, true>(L, st) : launch_one<true, false, TH, false>(L, st);
  }
  if (diag) return launch_one<false, true, TH, false>(L, st);
  return tab ? launch_one<false, false, TH, true>(L, st) : launch_one<false, false, TH, false>(L, st);
}

cudaError_t lpa_launch_order1(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  return L.tile_h == 8 ? launch_th<8>(L, comp, diag, st) : launch_th<16>(L, comp, diag, st);
}

template <bool COMP, int TH>
static cudaError_t launch_batch_t(const LpaBatch &B, int grid, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct_batch<1, COMP, TH>;
  cudaError_t e = lpa_opt_in((const void *)k);
  if (e != cudaSuccess) return e;
  k<<<grid, LPA_TILE * TH, B.smem_bytes, st>>>(B);
  return cudaGetLastError();
}

cudaError_t lpa_launch_batch_order1(const LpaBatch &B, bool comp, int tile_h, int grid, cudaStream_t st) {
  if (tile_h == 8) return comp ? launch_batch_t<true, 8>(B, grid, st) : launch_batch_t<false, 8>(B, grid, st);
  return comp ? launch_batch_t<true, 16>(B, grid, st) : launch_batch_t<false, 16>(B, grid, st);
}

template <bool COMP, int TH>
static int fit_t(uint32_t smem_bytes) {
  auto k = lpa::lpa_reconstruct_batch<1, COMP, TH>;
  int n = 0;
  if (lpa_opt_in((const void *)k) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, LPA_TILE * TH, smem_bytes) != cudaSuccess) return 0;
  return n;
}

int lpa_batch_ctas_per_sm_order1(bool comp, int tile_h, uint32_t smem_bytes) {
  if (tile_h == 8) return comp ? fit_t<true, 8>(smem_bytes) : fit_t<false, 8>(smem_bytes);
  return comp ? fit_t<true, 16>(smem_bytes) : fit_t<false, 16>(smem_bytes);
}

template <int TH>
static const void *kernel_th(bool comp, bool diag, bool tab) {
  if (comp) {
    if (diag) return (const void *)lpa::lpa_reconstruct<1, true, true, TH, false>;
    return tab ? (const void *)lpa::lpa_reconstruct<1, true, false, TH, true>
               : (const void *)lpa::lpa_reconstruct<1, true, false, TH, false>;
  }
  if (diag) return (const void *)lpa::lpa_reconstruct<1, false, true, TH, false>;
  return tab ? (const void *)lpa::lpa_reconstruct<1, false, false, TH, true>
             : (const void *)lpa::lpa_reconstruct<1, false, false, TH, false>;
}

const void *lpa_kernel_order1(bool comp, bool diag, bool tab, int tile_h) {
  return tile_h == 8 ? kernel_th<8>(comp, diag, tab) : kernel_th<16>(comp, diag, tab);
}
