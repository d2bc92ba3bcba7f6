// Instantiations of the single-frame and the persistent many-frame reconstruction kernels for
// polynomial order M = 0, and the self-test of the bounded wait.
#include "lpa_orders.cuh"

LPA_ORDER_ENTRY_POINTS(0)

cudaError_t lpa_launch_selftest_wait(unsigned int *status, cudaStream_t st) {
  lpa::lpa_selftest_wait<<<1, 32, 0, st>>>(status, 4096u, 200000000ll);  // ~0.1 s at 2 GHz at most
  return cudaGetLastError();
}
