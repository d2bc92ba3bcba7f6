// Radiometric calibration estimates of Section 6.2 (hdr_calib_*): per-pixel statistics of raw
// frame stacks, the gain of Eq. 21 and the exposure scaling / non-uniformity against a reference
// sensor. The stack statistics stream every frame once (HBM-bound); the two estimates are
// deterministic two-level reductions in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <vector>

#include "hdr_lpa.h"
#include "lpa_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxFrames = 4096;      // exact integer sums: n * sum y^2 < 2^63
constexpr int kReduceBlocks = 304;    // fixed grid: the summation order does not depend on timing

// One thread: 8 consecutive pixels of one row (one 16-byte load per frame, eight frames in flight).
// The loads of a CTA cover one contiguous row segment per frame; the kernel is bound by the exact
// 64-bit integer sums rather than by the reads (the same loads with trivial arithmetic stream at
// 5.7 TB/s). Exact sums S1 = sum y (< 2^32) and S2 = sum y^2 (< 2^45); mean = S1 / n and the
// unbiased variance (n S2 - S1^2) / (n (n - 1)), each one FP64 division of FP64-rounded integers,
// stored as FP32.
__global__ void __launch_bounds__(kThreads) calib_stats(const uint16_t *__restrict__ frames, int n, int width,
                                                        int height, int pitch, long long stride,
                                                        float *__restrict__ mean, float *__restrict__ var) {
  const int groups = (width + 7) >> 3;
  const long long t = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (t >= (long long)groups * height) return;
  const int row = (int)(t / groups), x = (int)(t % groups) * 8;
  const uint16_t *p = frames + (long long)row * pitch + x;
  uint32_t s1[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  unsigned long long s2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 8
  for (int f = 0; f < n; f++) {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(p + (long long)f * stride));
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t lo = w[k] & 0xffffu, hi = w[k] >> 16;
      s1[2 * k] += lo;
      s1[2 * k + 1] += hi;
      s2[2 * k] += (unsigned long long)lo * lo;
      s2[2 * k + 1] += (unsigned long long)hi * hi;
    }
  }
  const double dn = (double)n, dnn = (double)n * (double)(n - 1);
  float *m = mean + (long long)row * width + x, *vr = var + (long long)row * width + x;
#pragma unroll
  for (int k = 0; k < 8; k++) {
    if (x + k >= width) break;
    m[k] = (float)((double)s1[k] / dn);
    const long long num = (long long)n * (long long)s2[k] - (long long)s1[k] * (long long)s1[k];
    vr[k] = (float)((double)num / dnn);
  }
}

// Block sum of up to three doubles in a fixed order (strided per thread, then a tree).
__device__ void block_sum3(double a, double b, double c, double *out) {
  __shared__ double sh[3][kThreads];
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = c;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; q++) out[q] = sh[q][0];
}

__device__ __forceinline__ bool usable(float fm, float bm, double min_signal, double max_level) {
  return (double)fm - (double)bm >= min_signal && (double)fm < max_level;
}

// Eq. 21 pooled: partial sums of Var y - Var b and E[y] - E[b] over usable pixels, and their count.
__global__ void __launch_bounds__(kThreads) calib_gain_partial(const float *fm, const float *fv, const float *bm,
                                                               const float *bv, long long npx, double min_signal,
                                                               double max_level, double *partial) {
  double num = 0.0, den = 0.0, cnt = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < npx; i += (long long)gridDim.x * kThreads) {
    if (!usable(fm[i], bm[i], min_signal, max_level)) continue;
    num += (double)fv[i] - (double)bv[i];
    den += (double)fm[i] - (double)bm[i];
    cnt += 1.0;
  }
  block_sum3(num, den, cnt, partial + 3 * blockIdx.x);
}

// rho_i = ((E y - b) / (g t))_s / ((E y - b) / (g t))_ref at pixels usable in both sensors.
__device__ __forceinline__ bool exposure_rho(const float *fm, const float *bm, const float *rfm, const float *rbm,
                                             long long i, double gt, double rgt, double min_signal,
                                             double max_level, double *rho) {
  if (!usable(fm[i], bm[i], min_signal, max_level) || !usable(rfm[i], rbm[i], min_signal, max_level)) return false;
  const double fs = ((double)fm[i] - (double)bm[i]) / gt;
  const double fr = ((double)rfm[i] - (double)rbm[i]) / rgt;
  *rho = fs / fr;
  return true;
}

__global__ void __launch_bounds__(kThreads) calib_exposure_partial(const float *fm, const float *bm, const float *rfm,
                                                                   const float *rbm, long long npx, double gt,
                                                                   double rgt, double min_signal, double max_level,
                                                                   double *partial) {
  double sum = 0.0, cnt = 0.0;
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < npx; i += (long long)gridDim.x * kThreads) {
    double rho;
    if (!exposure_rho(fm, bm, rfm, rbm, i, gt, rgt, min_signal, max_level, &rho)) continue;
    sum += rho;
    cnt += 1.0;
  }
  block_sum3(sum, cnt, 0.0, partial + 3 * blockIdx.x);
}

// a_{s,i} = rho_i / n_s where usable in both sensors, 1 elsewhere.
__global__ void __launch_bounds__(kThreads) calib_prnu(const float *fm, const float *bm, const float *rfm,
                                                       const float *rbm, long long npx, double gt, double rgt,
                                                       double min_signal, double max_level, const double *n_s,
                                                       float *a) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= npx) return;
  double rho;
  a[i] = exposure_rho(fm, bm, rfm, rbm, i, gt, rgt, min_signal, max_level, &rho) ? (float)(rho / *n_s) : 1.f;
}

// Sum the per-block partials in block order on one thread; n_s = sum / count for the exposure.
__global__ void calib_finish(const double *partial, int blocks, int kind, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, b = 0.0, c = 0.0;
  for (int k = 0; k < blocks; k++) {
    a += partial[3 * k];
    b += partial[3 * k + 1];
    c += partial[3 * k + 2];
  }
  out[0] = a;
  out[1] = b;
  out[2] = c;
  if (kind == 1) out[3] = b > 0.0 ? a / b : NAN;  // exposure: mean of rho over usable pixels
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

hdr_status check_frame_args(int32_t width, int32_t height, const void *a, const void *b) {
  if (width < 1 || height < 1) return lpa_fail(HDR_E_INVALID, "width and height must be >= 1");
  if (!a || !b) return lpa_fail(HDR_E_INVALID, "a frame pointer is NULL");
  return HDR_OK;
}

// Device scratch for the reductions: partial sums then the finished values.
hdr_status reduce_scratch(double **d) {
  cudaError_t e = cudaMalloc(d, (3 * kReduceBlocks + 4) * sizeof(double));
  if (e != cudaSuccess) return lpa_fail(HDR_E_NOMEM, cudaGetErrorString(e));
  return HDR_OK;
}

}  // namespace

extern "C" {

hdr_status hdr_calib_stack_stats(hdr_ctx *ctx, const uint16_t *frames_dev, int32_t n_frames, int32_t width,
                                 int32_t height, int32_t pitch_elems, int64_t frame_stride_elems, float *mean_dev,
                                 float *var_dev, void *cuda_stream) {
  if (!ctx) return lpa_fail(HDR_E_INVALID, "ctx is NULL");
  if (!frames_dev || !mean_dev || !var_dev) return lpa_fail(HDR_E_INVALID, "a pointer is NULL");
  if (n_frames < 2 || n_frames > kMaxFrames) return lpa_fail(HDR_E_INVALID, "n_frames must be in [2, 4096]");
  if (width < 1 || height < 1) return lpa_fail(HDR_E_INVALID, "width and height must be >= 1");
  if (pitch_elems < ((width + 7) / 8) * 8 || pitch_elems % 8)
    return lpa_fail(HDR_E_INVALID, "pitch_elems must be a multiple of 8 and cover the width rounded up to 8");
  if (frame_stride_elems < (int64_t)pitch_elems * height || frame_stride_elems % 8)
    return lpa_fail(HDR_E_INVALID, "frame_stride_elems must be a multiple of 8 and cover a frame");
  if (!aligned16(frames_dev)) return lpa_fail(HDR_E_INVALID, "frames_dev must be 16-byte aligned");
  cudaError_t e = cudaSetDevice(lpa_ctx_device(ctx));
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  const long long threads = (long long)((width + 7) / 8) * height;
  const long long blocks = (threads + kThreads - 1) / kThreads;
  if (blocks > 0x7fffffffLL) return lpa_fail(HDR_E_UNSUPPORTED, "frame too large");
  calib_stats<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)cuda_stream>>>(
      frames_dev, n_frames, width, height, pitch_elems, (long long)frame_stride_elems, mean_dev, var_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  return HDR_OK;
}

hdr_status hdr_calib_gain(hdr_ctx *ctx, const float *flat_mean, const float *flat_var, const float *black_mean,
                          const float *black_var, int32_t width, int32_t height, double min_signal, double max_level,
                          double *gain, int64_t *n_used, void *cuda_stream) {
  if (!ctx || !gain) return lpa_fail(HDR_E_INVALID, "ctx and gain must be non-NULL");
  hdr_status st = check_frame_args(width, height, flat_mean, flat_var);
  if (st) return st;
  st = check_frame_args(width, height, black_mean, black_var);
  if (st) return st;
  cudaError_t e = cudaSetDevice(lpa_ctx_device(ctx));
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  double *d = nullptr;
  st = reduce_scratch(&d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long npx = (long long)width * height;
  calib_gain_partial<<<kReduceBlocks, kThreads, 0, s>>>(flat_mean, flat_var, black_mean, black_var, npx, min_signal,
                                                         max_level, d);
  calib_finish<<<1, 32, 0, s>>>(d, kReduceBlocks, 0, d + 3 * kReduceBlocks);
  double out[4] = {0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 3 * kReduceBlocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  *gain = out[1] > 0.0 ? out[0] / out[1] : NAN;
  if (n_used) *n_used = (int64_t)out[2];
  return HDR_OK;
}

hdr_status hdr_calib_exposure(hdr_ctx *ctx, const float *flat_mean, const float *black_mean, double gain,
                              double exposure, const float *ref_flat_mean, const float *ref_black_mean,
                              double ref_gain, double ref_exposure, int32_t width, int32_t height, double min_signal,
                              double max_level, double *nd, float *prnu_dev, int64_t *n_used, void *cuda_stream) {
  if (!ctx || !nd) return lpa_fail(HDR_E_INVALID, "ctx and nd must be non-NULL");
  hdr_status st = check_frame_args(width, height, flat_mean, black_mean);
  if (st) return st;
  st = check_frame_args(width, height, ref_flat_mean, ref_black_mean);
  if (st) return st;
  if (!(gain > 0.0) || !(exposure > 0.0) || !(ref_gain > 0.0) || !(ref_exposure > 0.0))
    return lpa_fail(HDR_E_INVALID, "gains and exposure times must be > 0");
  cudaError_t e = cudaSetDevice(lpa_ctx_device(ctx));
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  double *d = nullptr;
  st = reduce_scratch(&d);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const long long npx = (long long)width * height;
  const double gt = gain * exposure, rgt = ref_gain * ref_exposure;
  calib_exposure_partial<<<kReduceBlocks, kThreads, 0, s>>>(flat_mean, black_mean, ref_flat_mean, ref_black_mean, npx,
                                                             gt, rgt, min_signal, max_level, d);
  calib_finish<<<1, 32, 0, s>>>(d, kReduceBlocks, 1, d + 3 * kReduceBlocks);
  if (prnu_dev)
    calib_prnu<<<(unsigned)((npx + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        flat_mean, black_mean, ref_flat_mean, ref_black_mean, npx, gt, rgt, min_signal, max_level,
        d + 3 * kReduceBlocks + 3, prnu_dev);
  double out[4] = {0, 0, 0, 0};
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 3 * kReduceBlocks, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d);
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  *nd = out[3];
  if (n_used) *n_used = (int64_t)out[1];
  return HDR_OK;
}

}  // extern "C"
