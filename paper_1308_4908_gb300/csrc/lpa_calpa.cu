// Adaptive windows (CALPA, Sections 5.4-5.5): the steering-matrix pass and the entry points of the
// three passes. The gradient pass (isotropic order-1 green fit) and the steered reconstruction are
// modes of the reconstruction kernel (lpa_kernel.cuh).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "hdr_lpa.h"
#include "lpa_internal.h"
#include "lpa_launch.h"

namespace {

constexpr int kRmax = 10;  // largest radius (output pixels) of the pass-2 disc
constexpr int kBX = 32, kBY = 8;

struct MetricArgs {
  const float2 *grad;
  float *metric;
  int W, H, r;
  int rw[2 * kRmax + 1];           // half width of the disc in row offset dj (|di| <= rw)
  double w[2 * kRmax * kRmax + 1];  // Gaussian weight by di^2 + dj^2
  double scale2;                    // grad_scale^2: T of the scaled gradients
  float alpha, lambda1, lambda2, min_eig, max_eig;
};

// One thread per output pixel. The gradients of the block and its halo are staged in shared
// memory as the FP64 products gx^2, gx gy, gy^2 (exact: products of two FP32 values), so each
// neighbour costs three FP64 FMAs. T = sum_i w_i g_i g_i^T over the disc is summed in FP64: T of
// a straight edge is nearly rank one, and its small eigenvalue is the difference of large sums.
// The eigenvalues l1,2 = h +- sqrt(((a - c) / 2)^2 + b^2) and the components of the eigenvector
// of l1 ((b, l1 - a) or (l1 - c, b), the longer) are formed in FP64 too; what follows them (square
// roots, the direction's normalisation, elongation, the power and the matrix) has no cancellation
// and runs in FP32.
__global__ void __launch_bounds__(kBX *kBY) calpa_metric(const __grid_constant__ MetricArgs A) {
  constexpr int kTile = (kBY + 2 * kRmax) * (kBX + 2 * kRmax);
  __shared__ double sxx[kTile], sxy[kTile], syy[kTile];
  const int r = A.r, TW = kBX + 2 * r, TH = kBY + 2 * r;
  // one-dimensional grid over the 32 x 8 blocks (any output height)
  const int nbx = (A.W + kBX - 1) / kBX;
  const int bx0 = (int)(blockIdx.x % nbx) * kBX, by0 = (int)(blockIdx.x / nbx) * kBY;
  const int tid = threadIdx.y * kBX + threadIdx.x;
  for (int e = tid; e < TW * TH; e += kBX * kBY) {
    const int X = bx0 - r + e % TW, Y = by0 - r + e / TW;
    const float2 g = (X >= 0 && X < A.W && Y >= 0 && Y < A.H) ? A.grad[(size_t)Y * A.W + X] : make_float2(0.f, 0.f);
    const double gx = g.x, gy = g.y;
    sxx[e] = gx * gx;
    sxy[e] = gx * gy;
    syy[e] = gy * gy;
  }
  __syncthreads();
  const int u = bx0 + threadIdx.x, v = by0 + threadIdx.y;
  if (u >= A.W || v >= A.H) return;
  double a = 0.0, b = 0.0, c = 0.0;
  int M = 0;
  for (int dj = -r; dj <= r; dj++) {
    const int vv = v + dj;
    if (vv < 0 || vv >= A.H) continue;
    const int rw = A.rw[dj + r];
    M += min(u + rw, A.W - 1) - max(u - rw, 0) + 1;  // disc cells of this row inside the image
    const int row = (threadIdx.y + r + dj) * TW + threadIdx.x + r;
    for (int di = -rw; di <= rw; di++) {
      const double wt = A.w[di * di + dj * dj];
      a = fma(wt, sxx[row + di], a);
      b = fma(wt, sxy[row + di], b);
      c = fma(wt, syy[row + di], c);
    }
  }
  a *= A.scale2;
  b *= A.scale2;
  c *= A.scale2;
  const double h = 0.5 * (a + c), d = sqrt(0.25 * (a - c) * (a - c) + b * b);
  const double l1 = h + d, l2 = fmax(h - d, 0.0);
  double vx = b, vy = l1 - a;
  const double fx = l1 - c, fy = b;
  if (fx * fx + fy * fy > vx * vx + vy * vy) {
    vx = fx;
    vy = fy;
  }
  // the direction to FP32 with its exponent removed exactly (no underflow for tiny T)
  int ex = 0;
  frexp(fmax(fabs(vx), fabs(vy)), &ex);
  float ux = (float)ldexp(vx, -ex), uy = (float)ldexp(vy, -ex);
  const float n2 = ux * ux + uy * uy;
  if (n2 == 0.f) {  // T = 0
    ux = 1.f;
    uy = 0.f;
  } else {
    const float nrm = sqrtf(n2);
    ux /= nrm;
    uy /= nrm;
  }
  const float s1 = sqrtf((float)l1), s2 = sqrtf((float)l2);
  const float elong = (s1 + A.lambda1) / (s2 + A.lambda1);
  const float gamma = powf((s1 * s2 + A.lambda2) / (float)M, A.alpha);
  const float ea = fminf(fmaxf(gamma * elong, A.min_eig), A.max_eig);  // along u1: across the edge
  const float eb = fminf(fmaxf(gamma / elong, A.min_eig), A.max_eig);  // along u2: along the edge
  float *o = A.metric + ((size_t)v * A.W + u) * 3;
  o[0] = ea * ux * ux + eb * uy * uy;
  o[1] = (ea - eb) * ux * uy;
  o[2] = ea * uy * uy + eb * ux * ux;
}

hdr_status check_calpa(const hdr_calpa_params *c) {
  if (!c) return lpa_fail(HDR_E_INVALID, "calpa is NULL");
  auto fin = [](double x) { return std::isfinite(x); };
  if (!(c->grad_sigma > 0.0) || !fin(c->grad_sigma))
    return lpa_fail(HDR_E_INVALID, "grad_sigma must be finite and > 0");
  if (!(c->window_sigma > 0.0) || !(3.0 * c->window_sigma < kRmax + 1.0))
    return lpa_fail(HDR_E_INVALID, "window_sigma must be > 0 with 3 window_sigma < 11");
  // bounds keep every FP32 quantity of the matrix pass inside the normal range
  if (!(c->alpha >= 0.0) || !(c->alpha <= 4.0)) return lpa_fail(HDR_E_INVALID, "alpha must be in [0, 4]");
  if (!(c->lambda1 >= 1e-6 && c->lambda1 <= 1e6) || !(c->lambda2 >= 1e-12 && c->lambda2 <= 1e12))
    return lpa_fail(HDR_E_INVALID, "lambda1 in [1e-6, 1e6] and lambda2 in [1e-12, 1e12] required");
  if (!(c->min_eig >= 1e-6) || !(c->max_eig >= c->min_eig) || !(c->max_eig <= 1e6))
    return lpa_fail(HDR_E_INVALID, "1e-6 <= min_eig <= max_eig <= 1e6 required");
  if (!(c->grad_scale > 0.0) || !(c->grad_scale <= 1e6)) return lpa_fail(HDR_E_INVALID, "grad_scale must be in (0, 1e6]");
  return HDR_OK;
}

}  // namespace

hdr_status lpa_check_calpa(const hdr_calpa_params *c) { return check_calpa(c); }

double lpa_calpa_reach(const hdr_calpa_params *calpa) { return 1.0 / std::sqrt(calpa->min_eig); }

namespace {
// Pass 1: one isotropic order-1 fit at grad_sigma (ahead: see lpa_launch_mode).
hdr_status gradients(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const hdr_calpa_params *calpa,
                     const uint16_t *const *raw_dev, float *grad_dev, cudaStream_t st, bool ahead) {
  hdr_status s = check_calpa(calpa);
  if (s) return s;
  if (!params) return lpa_fail(HDR_E_INVALID, "params is NULL");
  hdr_params p = *params;
  p.order = 1;
  p.n_scales = 1;
  p.sigma[0] = calpa->grad_sigma;
  return lpa_launch_mode(ctx, rig_id, &p, raw_dev, LPA_GRADIENTS, grad_dev, 1.0, nullptr, nullptr, st, ahead);
}
}  // namespace

hdr_status lpa_calpa_prepare(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const hdr_calpa_params *calpa,
                             const uint16_t *const *raw_dev, float *scratch, cudaStream_t st) {
  const size_t npx = (size_t)params->out_w * params->out_h;
  if (npx == 0) return HDR_OK;
  float *grad = scratch, *metric = scratch + npx * 2;
  // inside a batch, whose plans may point into the context's conversion buffer: the pass converts
  // its footprints itself
  hdr_status s = gradients(ctx, rig_id, params, calpa, raw_dev, grad, st, false);
  if (s) return s;
  return hdr_calpa_metric(ctx, params->out_w, params->out_h, calpa, grad, metric, st);
}

extern "C" {

void hdr_calpa_params_default(hdr_calpa_params *c) {
  if (!c) return;
  c->grad_sigma = 1.2;
  c->window_sigma = 1.0;
  c->alpha = 0.3;
  c->lambda1 = 1.0;
  c->lambda2 = 1e-3;
  c->min_eig = 0.25;
  c->max_eig = 16.0;
  c->grad_scale = 0.1;
}

hdr_status hdr_calpa_gradients(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const hdr_calpa_params *calpa,
                               const uint16_t *const *raw_dev, float *grad_dev, void *cuda_stream) {
  return gradients(ctx, rig_id, params, calpa, raw_dev, grad_dev, (cudaStream_t)cuda_stream, true);
}

hdr_status hdr_calpa_metric(hdr_ctx *ctx, int32_t out_w, int32_t out_h, const hdr_calpa_params *calpa,
                            const float *grad_dev, float *metric_dev, void *cuda_stream) {
  if (!ctx) return lpa_fail(HDR_E_INVALID, "ctx is NULL");
  hdr_status st = check_calpa(calpa);
  if (st) return st;
  if (out_w < 0 || out_h < 0) return lpa_fail(HDR_E_INVALID, "negative output size");
  if ((long long)out_w * out_h > (1LL << 31) / 4) return lpa_fail(HDR_E_UNSUPPORTED, "output too large");
  if ((long long)out_w * out_h == 0) return HDR_OK;
  if (!grad_dev || !metric_dev) return lpa_fail(HDR_E_INVALID, "grad_dev and metric_dev are required");
  if (reinterpret_cast<uintptr_t>(grad_dev) % 8) return lpa_fail(HDR_E_INVALID, "grad_dev not 8-byte aligned");
  if (cudaSetDevice(lpa_ctx_device(ctx)) != cudaSuccess) return lpa_fail(HDR_E_CUDA, "cudaSetDevice failed");
  MetricArgs A{};
  A.grad = reinterpret_cast<const float2 *>(grad_dev);
  A.metric = metric_dev;
  A.W = out_w;
  A.H = out_h;
  const double ws = calpa->window_sigma, R = 3.0 * ws;
  A.r = (int)std::floor(R);
  for (int dj = -A.r; dj <= A.r; dj++) {
    int rw = 0;
    while (rw + 1 <= A.r && (double)((rw + 1) * (rw + 1) + dj * dj) <= R * R) rw++;
    A.rw[dj + A.r] = rw;
  }
  for (int k = 0; k <= 2 * A.r * A.r; k++) A.w[k] = std::exp(-(double)k / (2.0 * ws * ws));
  A.scale2 = calpa->grad_scale * calpa->grad_scale;
  A.alpha = (float)calpa->alpha;
  A.lambda1 = (float)calpa->lambda1;
  A.lambda2 = (float)calpa->lambda2;
  A.min_eig = (float)calpa->min_eig;
  A.max_eig = (float)calpa->max_eig;
  const unsigned blocks = (unsigned)(((long long)out_w + kBX - 1) / kBX * (((long long)out_h + kBY - 1) / kBY));
  calpa_metric<<<blocks, dim3(kBX, kBY), 0,
                 (cudaStream_t)cuda_stream>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
  return HDR_OK;
}

hdr_status hdr_reconstruct_steered(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                   const hdr_calpa_params *calpa, const uint16_t *const *raw_dev,
                                   const float *metric_dev, void *out_dev, uint8_t *choice_dev, void *cuda_stream) {
  hdr_status st = check_calpa(calpa);
  if (st) return st;
  if (!params) return lpa_fail(HDR_E_INVALID, "params is NULL");
  if (!metric_dev && (long long)params->out_w * params->out_h > 0) return lpa_fail(HDR_E_INVALID, "metric_dev is NULL");
  return lpa_launch_mode(ctx, rig_id, params, raw_dev, LPA_STEERED, const_cast<float *>(metric_dev),
                         lpa_calpa_reach(calpa), out_dev, choice_dev, (cudaStream_t)cuda_stream, true);
}

hdr_status hdr_reconstruct_adaptive(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                    const hdr_calpa_params *calpa, const uint16_t *const *raw_dev, void *out_dev,
                                    uint8_t *choice_dev, void *cuda_stream) {
  if (!ctx) return lpa_fail(HDR_E_INVALID, "ctx is NULL");
  hdr_status st = check_calpa(calpa);
  if (st) return st;
  st = lpa_check_params(params);
  if (st) return st;
  const size_t npx = (size_t)params->out_w * params->out_h;
  if (npx == 0) return HDR_OK;
  void *scratch = nullptr;
  st = lpa_ctx_calpa_scratch(ctx, npx * 5 * sizeof(float), &scratch);
  if (st) return st;
  float *grad = static_cast<float *>(scratch), *metric = grad + npx * 2;
  st = hdr_calpa_gradients(ctx, rig_id, params, calpa, raw_dev, grad, cuda_stream);
  if (st) return st;
  st = hdr_calpa_metric(ctx, params->out_w, params->out_h, calpa, grad, metric, cuda_stream);
  if (st) return st;
  return hdr_reconstruct_steered(ctx, rig_id, params, calpa, raw_dev, metric, out_dev, choice_dev, cuda_stream);
}

}  // extern "C"
