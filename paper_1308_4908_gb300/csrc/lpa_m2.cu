// Instantiations of the single-frame reconstruction kernel for polynomial order M = 2.
#include "lpa_dispatch.h"
#include "lpa_kernel.cuh"

template <bool COMP, bool DIAG, int TH>
static cudaError_t launch_one(const LpaLaunch &L, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct<2, COMP, DIAG, TH>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  k<<<L.tiles_x * L.tiles_y, LPA_TILE * TH, L.smem_bytes, st>>>(L);
  return cudaGetLastError();
}

template <int TH>
static cudaError_t launch_th(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  if (comp) return diag ? launch_one<true, true, TH>(L, st) : launch_one<true, false, TH>(L, st);
  return diag ? launch_one<false, true, TH>(L, st) : launch_one<false, false, TH>(L, st);
}

cudaError_t lpa_launch_order2(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  return L.tile_h == 8 ? launch_th<8>(L, comp, diag, st) : launch_th<16>(L, comp, diag, st);
}
