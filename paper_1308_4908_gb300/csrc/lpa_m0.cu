// Instantiations of the single-frame and the persistent many-frame reconstruction kernels for
// polynomial order M = 0, the conversion of frames ahead of a reconstruction, and the self-test of
// the bounded wait.
#include <algorithm>

#include "lpa_orders.cuh"

LPA_ORDER_ENTRY_POINTS(0)

cudaError_t lpa_launch_selftest_wait(unsigned int *status, cudaStream_t st) {
  lpa::lpa_selftest_wait<<<1, 32, 0, st>>>(status, 4096u, 200000000ll);  // ~0.1 s at 2 GHz at most
  return cudaGetLastError();
}

const void *lpa_convert_kernel(bool lit) {
  return lit ? (const void *)lpa::lpa_convert<true> : (const void *)lpa::lpa_convert<false>;
}

dim3 lpa_convert_grid(const LpaLaunch &L, const LpaRows &R) {
  long most = 0;
  for (int s = 0; s < L.n_sensors; s++) most = std::max<long>(most, (long)(R.r1[s] - R.r0[s]) * ((L.s[s].conv_pitch + 3) / 4));
  return dim3((unsigned)std::max<long>(1, std::min<long>((most + 255) / 256, 152 * 16)), (unsigned)L.n_sensors);
}

cudaError_t lpa_launch_convert(const LpaLaunch &L, const LpaRows &R, bool lit, cudaStream_t st) {
  const dim3 grid = lpa_convert_grid(L, R);
  if (lit) lpa::lpa_convert<true><<<grid, 256, 0, st>>>(L, R);
  else lpa::lpa_convert<false><<<grid, 256, 0, st>>>(L, R);
  return cudaGetLastError();
}
