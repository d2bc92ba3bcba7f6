// Instantiations of the reconstruction kernel for polynomial order M = 2.
#include "lpa_kernel.cuh"
#include "lpa_dispatch.h"

template <bool COMP, bool DIAG>
static cudaError_t launch_one(const LpaLaunch &L, cudaStream_t st) {
  auto k = lpa::lpa_reconstruct<2, COMP, DIAG>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  k<<<L.tiles_x * L.tiles_y, LPA_THREADS, L.smem_bytes, st>>>(L);
  return cudaGetLastError();
}

cudaError_t lpa_launch_order2(const LpaLaunch &L, bool comp, bool diag, cudaStream_t st) {
  if (comp) return diag ? launch_one<true, true>(L, st) : launch_one<true, false>(L, st);
  return diag ? launch_one<false, true>(L, st) : launch_one<false, false>(L, st);
}
