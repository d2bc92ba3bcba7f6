// Host side of the C ABI declared in include/hdr_lpa.h: contexts, device-resident
// rigs, launch planning (staging footprints, tensor maps) and the kernel launch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <array>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "hdr_lpa.h"
#include "lpa_dispatch.h"
#include "lpa_internal.h"
#include "lpa_launch.h"

static_assert(HDR_MAX_SENSORS == LPA_MAX_SENSORS, "sensor limits differ");
static_assert(HDR_MAX_SCALES == LPA_MAX_SCALES, "scale limits differ");

namespace {

thread_local std::string g_err;

hdr_status fail(hdr_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(e_ == cudaErrorMemoryAllocation ? HDR_E_NOMEM : HDR_E_CUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(e_), __FILE__, __LINE__);                           \
  } while (0)

constexpr int kMaxRigs = 64;

struct RigSensor {
  hdr_sensor_desc d;   // host copy; frame pointers below replace the caller's
  float *bias = nullptr, *prnu = nullptr, *rvar = nullptr;
  uint16_t *satf = nullptr;
};

struct Rig {
  int n = 0;
  RigSensor s[HDR_MAX_SENSORS];
};

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace

// Device tables and recorded graphs of the batched launch. The host staging is double-buffered:
// a launch may be prepared while the previous one still runs (each buffer has its own graphs).
struct BatchState {
  size_t cap_frames = 0, cap_tiles = 0;
  LpaLaunch *frames_dev = nullptr;
  int2 *tiles_dev = nullptr;
  int *bounds_dev = nullptr;                                  // [4] segment bounds per order
  unsigned int *counters_dev = nullptr;                       // [3]
  struct Staging {
    LpaLaunch *frames = nullptr;                              // pinned
    int2 *tiles = nullptr;
    int *bounds = nullptr;
    cudaEvent_t done = nullptr;                               // the launch that read this buffer ended
    bool pending = false;
  } stage[2];
  int cur = 0;
  struct Key {
    int comp, tile_h, buf;
    int grid[3];                                              // per order; 0 = no tiles of that order
    uint32_t smem[3];
    size_t cap_frames, cap_tiles;
    bool operator<(const Key &o) const {
      return std::tie(comp, tile_h, buf, grid[0], grid[1], grid[2], smem[0], smem[1], smem[2], cap_frames, cap_tiles) <
             std::tie(o.comp, o.tile_h, o.buf, o.grid[0], o.grid[1], o.grid[2], o.smem[0], o.smem[1], o.smem[2],
                      o.cap_frames, o.cap_tiles);
    }
  };
  std::map<Key, cudaGraphExec_t> graphs;
  std::map<uint64_t, hdr_batch_config> tuned;
  // form 0: one kernel node per frame, keyed by each node's (order, accum, tile height, grid,
  // shared memory); replays update the nodes' parameters
  struct FrameGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;
  };
  std::map<std::vector<std::array<int64_t, 5>>, FrameGraph> frame_graphs;
};

// Host-side caches of a context's launch planning.
struct PlanCache {
  // encoded tensor maps by (raw pointer, width, height, pitch, box): encoding is a driver call
  std::map<std::array<uint64_t, 4>, CUtensorMap> tmaps;
  // Tabulated-weight tables on the device, by a hash of their contents. Tables are small (tens of
  // KB) and kept until the context is destroyed, at most max_tables of them: the next one evicts
  // them all (after the device has finished the work that may use them).
  std::map<uint64_t, void *> dev;
  // the inputs a table is built from (sensor count, scales, window constants, scales per pass, each sensor's
  // translation) -> the device table, so that a repeated configuration skips the host build
  std::map<std::vector<double>, void *> by_inputs;
  uint64_t epoch = 0;  // bumped at each eviction (plans holding evicted tables are stale)
  size_t max_tables = 4096;
  // Plans made but not yet launched (a batch plans every frame before its one launch) may hold
  // tables an eviction removes: inside a hold scope evicted tables are retired, not freed; a later
  // eviction frees those retired in earlier scopes (whose launches it has waited for).
  int hold = 0;
  uint64_t scope = 0;
  std::vector<std::pair<void *, uint64_t>> retired;  // (table, scope that retired it)
};

// Keeps the tables that plans made in its scope point at allocated until it ends.
struct TableHold {
  PlanCache &c;
  explicit TableHold(PlanCache &cache) : c(cache) {
    c.hold++;
    c.scope++;
  }
  ~TableHold() { c.hold--; }
};

#ifndef LPA_FRAME_STAGES
#define LPA_FRAME_STAGES 1   // staging buffers per CTA of single-frame launches
#endif
#ifndef LPA_FRAME_CONV
#define LPA_FRAME_CONV 1     // single-frame calls convert the frame in one pass before the reconstruction
#endif
#ifndef LPA_HOST_BANDS
#define LPA_HOST_BANDS 16    // most row bands of hdr_reconstruct_host (each of at least 8 tile rows)
#endif
#ifndef LPA_HOST_BAND_STREAMS
#define LPA_HOST_BAND_STREAMS 2  // compute streams the row bands alternate on
#endif
constexpr int kMaxBands = 16;
static_assert(LPA_HOST_BANDS >= 1 && LPA_HOST_BANDS <= kMaxBands, "row bands of the host-buffer path");

struct hdr_ctx {
  int device = 0;
  PlanCache tabs;
  unsigned int *status = nullptr;
  BatchState batch;
  Rig rigs[kMaxRigs];
  EncodeTiledFn encode = nullptr;
  // staging for the host-buffer entry point
  uint16_t *raw_stage[HDR_MAX_SENSORS] = {};
  size_t raw_cap[HDR_MAX_SENSORS] = {};
  void *out_stage = nullptr;
  size_t out_cap = 0;
  uint8_t *choice_stage = nullptr;
  size_t choice_cap = 0;
  // copy streams and band events of the host-buffer entry point (created on first use)
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[kMaxBands] = {}, ev_done[kMaxBands] = {};
  cudaStream_t band2 = nullptr;  // host-buffer path: the second stream the row bands alternate on
  // frames converted ahead of single-frame reconstructions: one buffer, and the event after its
  // last use (a call on any stream waits for it before converting into the buffer again)
  float2 *conv_buf = nullptr;
  size_t conv_cap = 0;  // float2 elements
  cudaEvent_t conv_ev = nullptr;
  // gradient and steering-matrix planes of the adaptive reconstruction
  void *calpa = nullptr;
  size_t calpa_cap = 0;
  // launch plans of single-frame calls by (rig, rig generation, parameters, raw pointers): a
  // repeated call skips the planning; hdr_set_rig bumps the rig's generation
  uint64_t rig_gen[kMaxRigs] = {};
  std::map<std::vector<uint8_t>, LpaLaunch> plans;
};

namespace {

void free_rig(Rig &r) {
  for (int i = 0; i < r.n; i++) {
    cudaFree(r.s[i].bias);
    cudaFree(r.s[i].prnu);
    cudaFree(r.s[i].rvar);
    cudaFree(r.s[i].satf);
    r.s[i] = RigSensor();
  }
  r.n = 0;
}

bool finite6(const double *a) {
  for (int i = 0; i < 6; i++)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// 2x3 affine inverse (FP64).
void invert_affine(const double m[6], double inv[6]) {
  double det = m[0] * m[4] - m[1] * m[3];
  inv[0] = m[4] / det;
  inv[1] = -m[1] / det;
  inv[3] = -m[3] / det;
  inv[4] = m[0] / det;
  inv[2] = -(inv[0] * m[2] + inv[1] * m[5]);
  inv[5] = -(inv[3] * m[2] + inv[4] * m[5]);
}

// c = a o b (apply b first).
void compose_affine(const double a[6], const double b[6], double c[6]) {
  c[0] = a[0] * b[0] + a[1] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[4];
  c[2] = a[0] * b[2] + a[1] * b[5] + a[2];
  c[3] = a[3] * b[0] + a[4] * b[3];
  c[4] = a[3] * b[1] + a[4] * b[4];
  c[5] = a[3] * b[2] + a[4] * b[5] + a[5];
}

// Validate the descriptors of a rig of n_sensors sensors.
hdr_status check_sensors(int32_t n_sensors, const hdr_sensor_desc *sensors) {
  if (n_sensors < 1 || n_sensors > HDR_MAX_SENSORS)
    return fail(HDR_E_INVALID, "n_sensors %d not in [1,%d]", n_sensors, HDR_MAX_SENSORS);
  if (!sensors) return fail(HDR_E_INVALID, "sensors is NULL");
  for (int s = 0; s < n_sensors; s++) {
    const hdr_sensor_desc &d = sensors[s];
    if (d.width < 1 || d.height < 1 || d.pitch_elems < d.width || (d.pitch_elems * 2) % 16)
      return fail(HDR_E_INVALID, "sensor %d: bad size %dx%d / pitch %d (pitch*2 must be a multiple of 16)", s,
                  d.width, d.height, d.pitch_elems);
    if (d.width > (1 << 20) || d.height > (1 << 20)) return fail(HDR_E_UNSUPPORTED, "sensor %d too large", s);
    if (d.cfa != 0) return fail(HDR_E_UNSUPPORTED, "sensor %d: only the RGGB layout (cfa 0) is implemented", s);
    if (!(d.gain > 0) || !(d.exposure > 0) || !(d.nd > 0) || !std::isfinite(d.gain * d.exposure * d.nd))
      return fail(HDR_E_INVALID, "sensor %d: gain, exposure and nd must be finite and > 0", s);
    if (!d.read_var_frame && !(d.read_var > 0)) return fail(HDR_E_INVALID, "sensor %d: read_var must be > 0", s);
    if (!std::isfinite(d.black) || !std::isfinite(d.sat)) return fail(HDR_E_INVALID, "sensor %d: black/sat not finite", s);
    if (!finite6(d.affine)) return fail(HDR_E_INVALID, "sensor %d: affine not finite", s);
    const double det = d.affine[0] * d.affine[4] - d.affine[1] * d.affine[3];
    if (!(std::fabs(det) > 1e-12)) return fail(HDR_E_INVALID, "sensor %d: affine is singular", s);
    const size_t npx = (size_t)d.width * d.height;
    for (size_t i = 0; d.prnu_frame && i < npx; i++)
      if (!(d.prnu_frame[i] > 0.f) || !std::isfinite(d.prnu_frame[i]))
        return fail(HDR_E_INVALID, "sensor %d: prnu_frame must be finite and > 0", s);
    for (size_t i = 0; d.read_var_frame && i < npx; i++)
      if (!(d.read_var_frame[i] > 0.f) || !std::isfinite(d.read_var_frame[i]))
        return fail(HDR_E_INVALID, "sensor %d: read_var_frame must be finite and > 0", s);
  }
  return HDR_OK;
}

hdr_status check_params(const hdr_params *p) {
  if (!p) return fail(HDR_E_INVALID, "params is NULL");
  if (p->order < 0 || p->order > 2) return fail(HDR_E_INVALID, "order %d not in {0,1,2}", p->order);
  if (p->n_scales < 1 || p->n_scales > HDR_MAX_SCALES)
    return fail(HDR_E_INVALID, "n_scales %d not in [1,%d]", p->n_scales, HDR_MAX_SCALES);
  for (int j = 0; j < p->n_scales; j++) {
    if (!(p->sigma[j] > 0.0) || !std::isfinite(p->sigma[j])) return fail(HDR_E_INVALID, "sigma[%d] must be > 0", j);
    if (j > 0 && !(p->sigma[j] > p->sigma[j - 1])) return fail(HDR_E_INVALID, "sigma must be strictly ascending");
  }
  if (!(p->green_ratio > 0.0) || !(p->trunc_k > 0.0) || !(p->ici_gamma >= 0.0) || !(p->min_pivot >= 0.0) ||
      !std::isfinite(p->green_ratio) || !std::isfinite(p->trunc_k) || !std::isfinite(p->ici_gamma))
    return fail(HDR_E_INVALID, "green_ratio, trunc_k > 0 and ici_gamma, min_pivot >= 0 required");
  if (p->out_w < 0 || p->out_h < 0) return fail(HDR_E_INVALID, "negative output size");
  if ((long long)p->out_w * p->out_h > (1LL << 31) / 4)
    return fail(HDR_E_UNSUPPORTED, "output of %dx%d exceeds this build's size limit", p->out_w, p->out_h);
  if (!finite6(p->out_affine)) return fail(HDR_E_INVALID, "out_affine not finite");
  if (p->out_dtype != 0 && p->out_dtype != 1) return fail(HDR_E_INVALID, "out_dtype must be 0 or 1");
  if (p->accum != 0 && p->accum != 1) return fail(HDR_E_INVALID, "accum must be 0 or 1");
  if (p->tab_weights != 0 && p->tab_weights != 1) return fail(HDR_E_INVALID, "tab_weights must be 0 or 1");
  if (p->weight_mode != 0 && p->weight_mode != 1) return fail(HDR_E_INVALID, "weight_mode must be 0 or 1");
  return HDR_OK;
}

// What launch planning needs besides the rig: the tensor-map encoder, the device status word
// the kernel reports to, and the device.
struct PlanEnv {
  EncodeTiledFn encode;
  unsigned int *status;
  int device;
  PlanCache *tabs;  // NULL: no caches (the entry point may not allocate): nothing tabulated
  bool tabulate;    // tabulated weights allowed (the persistent batch kernels search every window)
};

bool is_identity_linear(const double *a) {
  return std::fabs(a[0] - 1.0) <= 1e-12 && std::fabs(a[1]) <= 1e-12 && std::fabs(a[3]) <= 1e-12 &&
         std::fabs(a[4] - 1.0) <= 1e-12;
}

int floor_div2_parity(long long v) { return (int)(((v % 2) + 2) % 2); }

// Section 8: with every sensor a pure translation of the reference frame and a 1x output mapping,
// the window of output pixel (u, v) in colour phase (ox, oy) of sensor s holds the samples
// (bxe + ox + 2 qx, bye + oy + 2 qy), bxe = even part of u + floor(G2) - ox, at offsets
// d = (2 qx - rx, 2 qy - ry) with rx = parity(u + floor(G2) - ox) + frac(G2): the same for every
// pixel of one parity class. The window cells (|d| < k sigma), offsets and weights are listed once.
}  // namespace

// Frames converted in a pass of their own before the reconstruction: at least one wave of 16x16
// tiles on the GPU's 152 SMs (smaller frames cost their launches, not the repeated conversion of
// overlapping footprints), outside the adaptive passes (their kernels convert footprints).
bool lpa_conv_eligible(const hdr_params *p, bool adaptive) {
  return LPA_FRAME_CONV && !adaptive && (long long)p->out_w * p->out_h >= 152LL * 256;
}

namespace {

// Layout of a frame converted ahead of the reconstruction: per sensor float2 [4][(h + 1) / 2][pitch],
// the pitch (x >> 1 columns) even so that rows are 16-byte multiples, sensors 256-byte aligned.
int conv_pitch_of(int w) { return ((w + 1) / 2 + 1) & ~1; }
size_t conv_elems_of(int w, int h) { return ((size_t)4 * ((h + 1) / 2) * conv_pitch_of(w) + 31) / 32 * 32; }
size_t conv_elems(const Rig &rig) {
  size_t n = 0;
  for (int s = 0; s < rig.n; s++) n += conv_elems_of(rig.s[s].d.width, rig.s[s].d.height);
  return n;
}

hdr_status build_tables(const PlanEnv &env, const Rig &rig, const hdr_params *p, bool f64_possible, LpaLaunch &L) {
  L.tab_hdr = nullptr;
  L.tab_cells = nullptr;
  L.tab_nsp = 0;
  if (!env.tabs || !env.tabulate || p->tab_weights != 1 || !is_identity_linear(p->out_affine)) return HDR_OK;
  // order 2 with the FP64 re-solve compiled in walks once per scale (the sums of two scales do not
  // fit beside it), the searched window with it compiled out feeds two scales from one walk; the
  // latter is the faster (4.04 against 4.14 ms on the translational paper rig)
  if (p->order == 2 && f64_possible) return HDR_OK;
  for (int s = 0; s < rig.n; s++)
    if (!is_identity_linear(rig.s[s].d.affine)) return HDR_OK;
  const int J = p->n_scales;
  const int nsp = lpa_scales_per_walk(p->order, p->accum != 0, f64_possible ? LPA_TABULATED : LPA_TABULATED_F32);
  const int npass = lpa_n_passes(J, nsp);
  std::vector<double> inputs = {(double)rig.n, (double)J, p->trunc_k, p->green_ratio, (double)nsp};
  for (int j = 0; j < J; j++) inputs.push_back(p->sigma[j]);
  for (int s = 0; s < rig.n; s++) {
    inputs.push_back(L.s[s].G[2]);
    inputs.push_back(L.s[s].G[5]);
    L.s[s].ix_shift = (int)std::floor(L.s[s].G[2]);
    L.s[s].iy_shift = (int)std::floor(L.s[s].G[5]);
  }
  const size_t n_hdr = (size_t)rig.n * 16 * npass * 2;
  auto known = env.tabs->by_inputs.find(inputs);
  if (known != env.tabs->by_inputs.end()) {
    L.tab_hdr = static_cast<const int4 *>(known->second);
    L.tab_cells = reinterpret_cast<const float4 *>(static_cast<const int4 *>(known->second) + n_hdr);
    L.tab_nsp = nsp;
    L.mode = LPA_TABULATED;
    return HDR_OK;
  }
  const double taper = std::exp(-0.5 * p->trunc_k * p->trunc_k);
  std::vector<int4> hdr(n_hdr);
  std::vector<float4> cells;
  auto pack = [](int lo, int hi) { return (lo & 0xffff) | (hi << 16); };
  for (int s = 0; s < rig.n; s++) {
    const double gx = L.s[s].G[2], gy = L.s[s].G[5];
    const double flx = std::floor(gx), fly = std::floor(gy);
    for (int pu = 0; pu < 2; pu++)
      for (int pv = 0; pv < 2; pv++)
        for (int ph = 0; ph < 4; ph++) {
          const int ox = ph & 1, oy = ph >> 1;
          const double gscale = (ox != oy) ? p->green_ratio : 1.0;  // phases (1,0), (0,1): G
          const double rx = floor_div2_parity((long long)pu + (long long)flx - ox) + (gx - flx);
          const double ry = floor_div2_parity((long long)pv + (long long)fly - oy) + (gy - fly);
          for (int pass = 0, j0 = 0, nj = lpa_first_pass_scales(J, nsp); pass < npass; pass++, j0 += nj, nj = nsp) {
            // the cells inside the window of the pass's largest scale, nearest first (ties by lattice
            // position, so that the table is a function of its inputs); slot q holds scale
            // j0 + q - lead, and its cells are the first n_q
            const int lead = nsp - nj;
            double sg[4], R2[4];
            for (int q = 0; q < nsp; q++) {
              sg[q] = p->sigma[q >= lead ? j0 + q - lead : j0] * gscale;
              const double R = p->trunc_k * sg[q];
              R2[q] = q >= lead ? R * R : -1.0;
            }
            const double R = p->trunc_k * sg[nsp - 1];
            struct Cell {
              double r2, dx, dy;
              int qx, qy;
            };
            std::vector<Cell> in;
            const int x0 = (int)std::floor((rx - R) / 2) - 1, x1 = (int)std::ceil((rx + R) / 2) + 1;
            const int y0 = (int)std::floor((ry - R) / 2) - 1, y1 = (int)std::ceil((ry + R) / 2) + 1;
            for (int qy = y0; qy <= y1; qy++)
              for (int qx = x0; qx <= x1; qx++) {
                const double dx = 2.0 * qx - rx, dy = 2.0 * qy - ry, r2 = dx * dx + dy * dy;
                if (r2 < R2[nsp - 1]) in.push_back({r2, dx, dy, qx, qy});
              }
            std::sort(in.begin(), in.end(), [](const Cell &a, const Cell &b) {
              return a.r2 != b.r2 ? a.r2 < b.r2 : a.qy != b.qy ? a.qy < b.qy : a.qx < b.qx;
            });
            int4 *h = &hdr[(((((size_t)s * 2 + pu) * 2 + pv) * 4 + ph) * npass + pass) * 2];
            h[0].x = (int)(cells.size() / 2);
            h[0].y = (int)in.size();
            int nq[4] = {0, 0, 0, 0};
            int qxmin = 1 << 14, qxmax = -(1 << 14), qymin = 1 << 14, qymax = -(1 << 14);
            for (const Cell &e : in) {
              float4 g, k;
              g.x = (float)e.dx;
              g.y = (float)e.dy;
              const int q = (e.qy << 16) | (e.qx & 0xffff);
              memcpy(&g.z, &q, 4);
              g.w = 0.f;
              float kv[4] = {0.f, 0.f, 0.f, 0.f};
              for (int t = 0; t < nsp; t++)
                if (e.r2 < R2[t]) {
                  kv[t] = (float)(std::exp(-e.r2 / (2.0 * sg[t] * sg[t])) - taper);  // Eq. 8, truncated and tapered
                  nq[t]++;
                }
              k = make_float4(kv[0], kv[1], kv[2], kv[3]);
              cells.push_back(g);
              cells.push_back(k);
              qxmin = std::min(qxmin, e.qx);
              qxmax = std::max(qxmax, e.qx);
              qymin = std::min(qymin, e.qy);
              qymax = std::max(qymax, e.qy);
            }
            if (in.empty()) qxmin = qxmax = qymin = qymax = 0;
            h[0].z = pack(qxmin, qxmax);
            h[0].w = pack(qymin, qymax);
            h[1] = make_int4(nq[0], nq[1], nq[2], nq[3]);
          }
        }
  }
  // one padding cell: the kernel loads the cell after each one it reads
  cells.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
  cells.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
  // content hash (FNV-1a) -> device copy
  const size_t nb = hdr.size() * sizeof(int4) + cells.size() * sizeof(float4);
  uint64_t hsh = 1469598103934665603ull;
  auto mix = [&](const void *ptr, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(ptr);
    for (size_t i = 0; i < n; i++) hsh = (hsh ^ b[i]) * 1099511628211ull;
  };
  mix(hdr.data(), hdr.size() * sizeof(int4));
  mix(cells.data(), cells.size() * sizeof(float4));
  hsh ^= (uint64_t)hdr.size() << 40;
  auto it = env.tabs->dev.find(hsh);
  if (it == env.tabs->dev.end()) {
    if (env.tabs->dev.size() >= env.tabs->max_tables) {
      // every launch made so far may use the tables: wait for the device, then free them, unless
      // plans that are not launched yet may hold them (then they wait in `retired`)
      CUDA_TRY(cudaDeviceSynchronize());
      PlanCache &tc = *env.tabs;
      size_t keep = 0;
      for (auto &t : tc.retired) {
        if (tc.hold > 0 && t.second == tc.scope) tc.retired[keep++] = t;
        else cudaFree(t.first);
      }
      tc.retired.resize(keep);
      for (auto &t : tc.dev) {
        if (tc.hold == 0) cudaFree(t.second);
        else tc.retired.push_back({t.second, tc.scope});
      }
      env.tabs->dev.clear();
      env.tabs->by_inputs.clear();
      env.tabs->epoch++;
    }
    void *d = nullptr;
    CUDA_TRY(cudaMalloc(&d, std::max<size_t>(nb, 16)));
    cudaError_t e = cudaMemcpy(d, hdr.data(), hdr.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !cells.empty())
      e = cudaMemcpy(static_cast<int4 *>(d) + hdr.size(), cells.data(), cells.size() * sizeof(float4),
                     cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d);
      return fail(HDR_E_CUDA, "uploading the weight table failed: %s", cudaGetErrorString(e));
    }
    it = env.tabs->dev.emplace(hsh, d).first;
  }
  if (env.tabs->by_inputs.size() >= 4 * env.tabs->max_tables) env.tabs->by_inputs.clear();
  env.tabs->by_inputs.emplace(std::move(inputs), it->second);
  L.tab_hdr = static_cast<const int4 *>(it->second);
  L.tab_cells = reinterpret_cast<const float4 *>(static_cast<const int4 *>(it->second) + hdr.size());
  L.tab_nsp = nsp;
  L.mode = LPA_TABULATED;
  return HDR_OK;
}

#ifndef LPA_FRAME_TILE_H
#define LPA_FRAME_TILE_H 16  // tile height of single-frame launches
#endif

// Fill the launch descriptor for one frame. raw: device pointers per sensor.
// reach: the largest window grows by this factor (the steered window of Section 5.4 reaches
// 1 / sqrt(smallest eigenvalue of C) times the isotropic radius).
// stages: 2 = the two-buffer kernel (each CTA copies its next tile while computing the current one)
// where it is built (plain sums, the searched or tabulated window), else 1.
// conv: a buffer of conv_elems(rig) float2 to convert the frames into ahead of the launch (the
// kernel then copies converted footprints and does no conversion), or nullptr.
hdr_status plan_env(const PlanEnv &env, const Rig &rig, const hdr_params *p, const uint16_t *const *raw,
                    LpaLaunch &L, int tile_h = 16, double reach = 1.0, int stages = 1, float2 *conv = nullptr) {
  memset(&L, 0, sizeof(L));
  L.n_sensors = rig.n;
  L.order = p->order;
  L.n_scales = p->n_scales;
  for (int j = 0; j < p->n_scales; j++) L.sigma[j] = (float)p->sigma[j];
  L.green_ratio = (float)p->green_ratio;
  L.trunc_k = (float)p->trunc_k;
  L.ici_gamma = (float)p->ici_gamma;
  L.min_pivot = (float)p->min_pivot;
  L.cond_fallback = (float)p->cond_fallback;
  L.taper = (float)std::exp(-0.5 * p->trunc_k * p->trunc_k);
  L.out_w = p->out_w;
  L.out_h = p->out_h;
  L.tile_h = tile_h;
  L.tile0 = 0;
  L.tiles_x = (p->out_w + LPA_TILE - 1) / LPA_TILE;
  L.tiles_y = (p->out_h + tile_h - 1) / tile_h;
  L.out_half = p->out_dtype;
  L.status = env.status;
  const double rmax = reach * p->trunc_k * p->sigma[p->n_scales - 1] * std::fmax(1.0, p->green_ratio);
  uint32_t off = 0, tx = 0;
  size_t conv_off = 0;
  L.conv = conv ? 1 : 0;
  for (int s = 0; s < rig.n; s++) {
    const hdr_sensor_desc &d = rig.s[s].d;
    LpaSensorK &K = L.s[s];
    if (!raw[s]) return fail(HDR_E_INVALID, "raw pointer of sensor %d is NULL", s);
    if (reinterpret_cast<uintptr_t>(raw[s]) % 16) return fail(HDR_E_INVALID, "raw pointer of sensor %d not 16-byte aligned", s);
    double tinv[6];
    invert_affine(d.affine, tinv);
    compose_affine(tinv, p->out_affine, K.G);
    for (int i = 0; i < 4; i++) K.Gf[i] = (float)K.G[i < 2 ? i : i + 1];
    K.A[0] = (float)d.affine[0];
    K.A[1] = (float)d.affine[1];
    K.A[2] = (float)d.affine[3];
    K.A[3] = (float)d.affine[4];
    const double hxu = std::sqrt(tinv[0] * tinv[0] + tinv[1] * tinv[1]);
    const double hyu = std::sqrt(tinv[3] * tinv[3] + tinv[4] * tinv[4]);
    K.hx_unit = (float)hxu;
    K.hy_unit = (float)hyu;
    const double gtn = d.gain * d.exposure * d.nd;
    K.inv_gtn = (float)(1.0 / gtn);
    K.gtn2 = (float)(gtn * gtn);
    K.gain = (float)d.gain;
    K.read_var = (float)d.read_var;
    K.black = (float)d.black;
    K.sat = (float)d.sat;
    K.width = d.width;
    K.height = d.height;
    K.bias = rig.s[s].bias;
    K.prnu = rig.s[s].prnu;
    K.rvar = rig.s[s].rvar;
    K.satf = rig.s[s].satf;
    // staging box: the tile's pixel points span |G_lin| * (TILE-1) in sensor space; add the
    // largest window's half extent plus margin on both sides, the floor of the origin and
    // the alignment of the origin (x to 8 elements = 16 bytes, y to 2)
    K.ext_x = (float)(rmax * hxu + LPA_MARGIN);
    K.ext_y = (float)(rmax * hyu + LPA_MARGIN);
    const double span_x = std::fabs(K.G[0]) * (LPA_TILE - 1) + std::fabs(K.G[1]) * (tile_h - 1);
    const double span_y = std::fabs(K.G[3]) * (LPA_TILE - 1) + std::fabs(K.G[4]) * (tile_h - 1);
    int bw = (int)std::ceil(span_x + 2.0 * K.ext_x) + 9;
    int bh = (int)std::ceil(span_y + 2.0 * K.ext_y) + 3;
    bw = (bw + 7) / 8 * 8;
    bh = (bh + 1) / 2 * 2;
    if (bw > 256 || bh > 256)
      return fail(HDR_E_UNSUPPORTED, "sensor %d staging box %dx%d exceeds 256 (window or output scale too large)", s, bw, bh);
    K.box_w = bw;
    K.box_h = bh;
    K.raw = raw[s];
    K.raw_pitch = d.pitch_elems;
    if (conv) {
      // the converted frame's colour-phase planes, copied straight into the staged planes
      K.conv_pitch = conv_pitch_of(d.width);
      K.conv_h = (d.height + 1) / 2;
      K.conv = conv + conv_off;
      conv_off += conv_elems_of(d.width, d.height);
      off = (off + 127) / 128 * 128;
      K.off_raw = K.off_planes = off;
      off += (uint32_t)(bw * bh * 8);
      tx += (uint32_t)(bw * bh * 8);
      const std::array<uint64_t, 4> ckey = {reinterpret_cast<uint64_t>(K.conv),
                                            ((uint64_t)K.conv_pitch << 32) | (uint32_t)K.conv_h, (1ull << 63) | 4u,
                                            ((uint64_t)bw << 32) | (uint32_t)bh};
      auto hit = env.tabs ? env.tabs->tmaps.find(ckey) : std::map<std::array<uint64_t, 4>, CUtensorMap>::iterator();
      if (env.tabs && hit != env.tabs->tmaps.end()) {
        K.tmap = hit->second;
      } else {
        cuuint64_t cdim[3] = {(cuuint64_t)K.conv_pitch, (cuuint64_t)K.conv_h, 4};
        cuuint64_t cstride[2] = {(cuuint64_t)K.conv_pitch * 8, (cuuint64_t)K.conv_pitch * K.conv_h * 8};
        cuuint32_t cbox[3] = {(cuuint32_t)(bw / 2), (cuuint32_t)(bh / 2), 4};
        cuuint32_t cestr[3] = {1, 1, 1};
        CUresult cr = env.encode(&K.tmap, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, K.conv, cdim, cstride, cbox, cestr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS)
          return fail(HDR_E_CUDA, "cuTensorMapEncodeTiled failed for the converted planes of sensor %d (code %d)", s, (int)cr);
        if (env.tabs) {
          if (env.tabs->tmaps.size() >= 4096) env.tabs->tmaps.clear();
          env.tabs->tmaps.emplace(ckey, K.tmap);
        }
      }
      continue;
    }
    off = (off + 127) / 128 * 128;
    K.off_raw = off;
    off += (uint32_t)(bw * bh * 2);
    tx += (uint32_t)(bw * bh * 2);
    off = (off + 127) / 128 * 128;
    K.off_planes = off;
    off += (uint32_t)(bw * bh * 8);
    // tensor map of the raw frame
    cuuint64_t gdim[2] = {(cuuint64_t)d.width, (cuuint64_t)d.height};
    cuuint64_t gstride[1] = {(cuuint64_t)d.pitch_elems * 2};
    cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    cuuint32_t estr[2] = {1, 1};
    const std::array<uint64_t, 4> mkey = {reinterpret_cast<uint64_t>(raw[s]),
                                          ((uint64_t)d.width << 32) | (uint32_t)d.height, (uint64_t)d.pitch_elems,
                                          ((uint64_t)bw << 32) | (uint32_t)bh};
    auto known = env.tabs ? env.tabs->tmaps.find(mkey) : std::map<std::array<uint64_t, 4>, CUtensorMap>::iterator();
    if (env.tabs && known != env.tabs->tmaps.end()) {
      K.tmap = known->second;
    } else {
      CUresult cr = env.encode(&K.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<uint16_t *>(raw[s]), gdim, gstride,
                                box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (cr != CUDA_SUCCESS) return fail(HDR_E_CUDA, "cuTensorMapEncodeTiled failed for sensor %d (code %d)", s, (int)cr);
      if (env.tabs) {
        if (env.tabs->tmaps.size() >= 4096) env.tabs->tmaps.clear();
        env.tabs->tmaps.emplace(mkey, K.tmap);
      }
    }
  }
  L.tx_bytes = tx;
  // a usable fit's equilibrated pivots lie in (min_pivot, 1]: when min_pivot * cond_fallback >= 2
  // their spread never exceeds cond_fallback and the FP64 re-solve cannot trigger
  const bool f64_possible = p->cond_fallback > 0.0 && (p->min_pivot - 1e-4) * p->cond_fallback < 2.0;
  if (p->weight_mode == 1) {  // the printed noise weight K / s: searched window, its own kernel
    L.mode = LPA_LITERAL;
  } else {
    hdr_status st = build_tables(env, rig, p, f64_possible, L);
    if (st) return st;
  }
  if (!f64_possible) L.mode = lpa_mode_to_f32(L.mode);
  if (!lpa_mode_tab(L.mode)) {  // each thread's sample cell in each sensor (tables need none)
    off = (off + 15) / 16 * 16;
    L.off_pos = off;
    off += (uint32_t)(rig.n * 16 * LPA_TILE * tile_h);
  }
  int max_smem = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, env.device));
  L.stages = 1;
  for (int s = 0; s < rig.n; s++) L.s[s].off_raw2 = L.s[s].off_raw;
  if (stages == 2 && !conv && lpa_stages2_built(L.mode, p->accum != 0)) {
    // the second buffer's raw boxes, where they fit beside the rest (else one buffer)
    uint32_t off2 = off, at[LPA_MAX_SENSORS];
    for (int s = 0; s < rig.n; s++) {
      off2 = (off2 + 127) / 128 * 128;
      at[s] = off2;
      off2 += (uint32_t)(L.s[s].box_w * L.s[s].box_h * 2);
    }
    if ((int)off2 <= max_smem - 1024) {
      for (int s = 0; s < rig.n; s++) L.s[s].off_raw2 = at[s];
      off = off2;
      L.stages = 2;
    }
  }
  L.smem_bytes = off;
  if ((int)off > max_smem - 1024)
    return fail(HDR_E_UNSUPPORTED, "staging needs %u bytes of shared memory (limit %d)", off, max_smem - 1024);
  return HDR_OK;
}

hdr_status plan(hdr_ctx *ctx, const Rig &rig, const hdr_params *p, const uint16_t *const *raw, LpaLaunch &L,
                double reach = 1.0, bool tabulate = true, int stages = 1, float2 *conv = nullptr) {
  return plan_env(PlanEnv{ctx->encode, ctx->status, ctx->device, &ctx->tabs, tabulate}, rig, p, raw, L,
                  LPA_FRAME_TILE_H, reach, stages, conv);
}

// The context's conversion buffer, at least `need` float2; growing it waits for the work that
// used it.
hdr_status conv_capacity(hdr_ctx *ctx, size_t need) {
  if (need > ctx->conv_cap) {
    if (ctx->conv_ev) CUDA_TRY(cudaEventSynchronize(ctx->conv_ev));
    cudaFree(ctx->conv_buf);
    ctx->conv_buf = nullptr;
    ctx->conv_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->conv_buf, need * sizeof(float2)));
    ctx->conv_cap = need;
  }
  if (!ctx->conv_ev) CUDA_TRY(cudaEventCreateWithFlags(&ctx->conv_ev, cudaEventDisableTiming));
  return HDR_OK;
}

// The conversion buffer of a single-frame call for this rig, or nullptr when the frame is
// converted in the kernel (lpa_conv_eligible).
hdr_status conv_buffer(hdr_ctx *ctx, const Rig &rig, const hdr_params *p, float2 **buf) {
  *buf = nullptr;
  if (!lpa_conv_eligible(p, false)) return HDR_OK;
  hdr_status st = conv_capacity(ctx, conv_elems(rig));
  if (st) return st;
  *buf = ctx->conv_buf;
  return HDR_OK;
}

// Convert rows [r0[s], r1[s]) of every sensor of L into its planes on `st`, after the last use of
// the buffer (the first call of a reconstruction passes first = true).
// Rows to convert, with the row past an odd height (its last plane row pairs with a row outside
// the frame, which converts to zeros) when the range reaches the height.
LpaRows rows_with_padding(const LpaLaunch &L, LpaRows R) {
  for (int s = 0; s < L.n_sensors; s++)
    if (R.r1[s] == L.s[s].height && (L.s[s].height & 1)) R.r1[s]++;
  return R;
}
LpaRows all_rows(const LpaLaunch &L) {
  LpaRows R{};
  for (int s = 0; s < L.n_sensors; s++) R.r1[s] = L.s[s].height;
  return rows_with_padding(L, R);
}

hdr_status convert_rows(hdr_ctx *ctx, const LpaLaunch &L, const LpaRows &rows, bool first, cudaStream_t st) {
  if (first) CUDA_TRY(cudaStreamWaitEvent(st, ctx->conv_ev, 0));
  cudaError_t e = lpa_launch_convert(L, rows_with_padding(L, rows), L.mode == LPA_LITERAL, st);
  if (e != cudaSuccess) return fail(HDR_E_CUDA, "conversion launch failed: %s", cudaGetErrorString(e));
  return HDR_OK;
}

// plan() of a single-frame call through the context's plan cache.
hdr_status cached_plan(hdr_ctx *ctx, int32_t rig_id, const hdr_params *p, const uint16_t *const *raw, LpaLaunch &L,
                       bool tabulate, int stages, float2 *conv) {
  const Rig &rig = ctx->rigs[rig_id];
  std::vector<uint8_t> key(sizeof(int32_t) + 2 * sizeof(uint64_t) + sizeof(hdr_params) + 2 + (rig.n + 1) * sizeof(void *));
  uint8_t *k = key.data();
  memcpy(k, &rig_id, sizeof(int32_t));
  k += sizeof(int32_t);
  memcpy(k, &ctx->rig_gen[rig_id], sizeof(uint64_t));
  k += sizeof(uint64_t);
  memcpy(k, &ctx->tabs.epoch, sizeof(uint64_t));  // tables the plan points at are still allocated
  k += sizeof(uint64_t);
  memcpy(k, p, sizeof(hdr_params));
  k += sizeof(hdr_params);
  *k++ = tabulate ? 1 : 0;
  *k++ = (uint8_t)stages;
  memcpy(k, &conv, sizeof(void *));
  k += sizeof(void *);
  memcpy(k, raw, rig.n * sizeof(void *));
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    L = it->second;
    return HDR_OK;
  }
  hdr_status st = plan(ctx, rig, p, raw, L, 1.0, tabulate, stages, conv);
  if (st) return st;
  if (ctx->plans.size() >= 256) ctx->plans.clear();
  ctx->plans.emplace(std::move(key), L);
  return HDR_OK;
}

hdr_status launch(const LpaLaunch &L, int accum, bool diag, cudaStream_t st) {
  if (L.tiles_x == 0 || L.tiles_y == 0) return HDR_OK;
  cudaError_t e;
  switch (L.order) {
    case 0: e = lpa_launch_order0(L, accum != 0, diag, st); break;
    case 1: e = lpa_launch_order1(L, accum != 0, diag, st); break;
    default: e = lpa_launch_order2(L, accum != 0, diag, st); break;
  }
  if (e != cudaSuccess) return fail(HDR_E_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  return HDR_OK;
}

hdr_status common_checks(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const void *raw, const void *out) {
  if (!ctx) return fail(HDR_E_INVALID, "ctx is NULL");
  if (rig_id < 0 || rig_id >= kMaxRigs || ctx->rigs[rig_id].n == 0)
    return fail(HDR_E_INVALID, "rig %d is not defined", rig_id);
  hdr_status st = check_params(params);
  if (st) return st;
  if (!raw) return fail(HDR_E_INVALID, "raw pointer array is NULL");
  if (!out && (long long)params->out_w * params->out_h > 0) return fail(HDR_E_INVALID, "output pointer is NULL");
  CUDA_TRY(cudaSetDevice(ctx->device));
  return HDR_OK;
}

hdr_status reconstruct_impl(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                            void *out_dev, uint8_t *choice_dev, float *levels_dev, void *stream) {
  hdr_status st = common_checks(ctx, rig_id, params, raw_dev, out_dev);
  if (st) return st;
  if (levels_dev && params->weight_mode != 0)
    return fail(HDR_E_UNSUPPORTED, "the level maps are computed with the inverse-variance weight (weight_mode 0)");
  LpaLaunch L;
  float2 *conv = nullptr;
  st = conv_buffer(ctx, ctx->rigs[rig_id], params, &conv);
  if (st) return st;
  // the diagnostic (level maps) kernel searches every window
  st = cached_plan(ctx, rig_id, params, raw_dev, L, levels_dev == nullptr, levels_dev ? 1 : LPA_FRAME_STAGES, conv);
  if (st) return st;
  L.out = out_dev;
  L.choice = choice_dev;
  L.levels = levels_dev;
  const cudaStream_t cs = (cudaStream_t)stream;
  if (L.conv) {  // the whole frame converted once, then the reconstruction
    st = convert_rows(ctx, L, all_rows(L), true, cs);
    if (st) return st;
  }
  st = launch(L, params->accum, levels_dev != nullptr, cs);
  if (st == HDR_OK && L.conv) CUDA_TRY(cudaEventRecord(ctx->conv_ev, cs));
  return st;
}

}  // namespace

extern "C" {

void hdr_params_default(hdr_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->order = 2;
  p->n_scales = 4;
  p->sigma[0] = 0.5;
  p->sigma[1] = 0.8;
  p->sigma[2] = 1.2;
  p->sigma[3] = 1.8;
  p->green_ratio = 1.0 / std::sqrt(2.0);
  p->trunc_k = 3.0;
  p->ici_gamma = 2.0;
  p->min_pivot = 1e-3;
  p->cond_fallback = 1e6;
  p->out_affine[0] = 1.0;
  p->out_affine[4] = 1.0;
  p->out_dtype = 0;
  p->accum = 0;
  p->tab_weights = 1;
  p->weight_mode = 0;
}

hdr_status hdr_create(int device, hdr_ctx **out) {
  if (!out) return fail(HDR_E_INVALID, "out is NULL");
  *out = nullptr;
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(HDR_E_INVALID, "device %d not present (%d devices)", device, n);
  CUDA_TRY(cudaSetDevice(device));
  hdr_ctx *c = new (std::nothrow) hdr_ctx();
  if (!c) return fail(HDR_E_NOMEM, "host allocation failed");
  c->device = device;
  cudaDriverEntryPointQueryResult q;
  void *fn = nullptr;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
    delete c;
    return fail(HDR_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
  }
  c->encode = reinterpret_cast<EncodeTiledFn>(fn);
  // HDR_LPA_MAX_TABLES (optional): fewer cached weight tables, so that tests can force evictions
  if (const char *mt = getenv("HDR_LPA_MAX_TABLES")) {
    const long v = strtol(mt, nullptr, 10);
    if (v >= 1 && v <= 4096) c->tabs.max_tables = (size_t)v;
  }
  e = cudaMalloc(&c->status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(c->status, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    cudaFree(c->status);
    delete c;
    return fail(HDR_E_NOMEM, "status word allocation failed: %s", cudaGetErrorString(e));
  }
  *out = c;
  return HDR_OK;
}

void hdr_destroy(hdr_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (int r = 0; r < kMaxRigs; r++) free_rig(ctx->rigs[r]);
  for (int s = 0; s < HDR_MAX_SENSORS; s++) cudaFree(ctx->raw_stage[s]);
  cudaFree(ctx->out_stage);
  cudaFree(ctx->choice_stage);
  cudaFree(ctx->calpa);
  for (auto &t : ctx->tabs.dev) cudaFree(t.second);
  for (auto &t : ctx->tabs.retired) cudaFree(t.first);
  if (ctx->h2d) cudaStreamDestroy(ctx->h2d);
  if (ctx->d2h) cudaStreamDestroy(ctx->d2h);
  if (ctx->band2) cudaStreamDestroy(ctx->band2);
  if (ctx->conv_ev) cudaEventDestroy(ctx->conv_ev);
  cudaFree(ctx->conv_buf);
  for (int b = 0; b < kMaxBands; b++) {
    if (ctx->ev_in[b]) cudaEventDestroy(ctx->ev_in[b]);
    if (ctx->ev_done[b]) cudaEventDestroy(ctx->ev_done[b]);
  }
  cudaFree(ctx->status);
  for (auto &g : ctx->batch.graphs) cudaGraphExecDestroy(g.second);
  for (auto &g : ctx->batch.frame_graphs) {
    cudaGraphExecDestroy(g.second.exec);
    cudaGraphDestroy(g.second.graph);
  }
  cudaFree(ctx->batch.frames_dev);
  cudaFree(ctx->batch.tiles_dev);
  cudaFree(ctx->batch.bounds_dev);
  cudaFree(ctx->batch.counters_dev);
  for (auto &S : ctx->batch.stage) {
    cudaFreeHost(S.frames);
    cudaFreeHost(S.tiles);
    cudaFreeHost(S.bounds);
    if (S.done) cudaEventDestroy(S.done);
  }
  delete ctx;
}

hdr_status hdr_set_rig(hdr_ctx *ctx, int32_t rig_id, int32_t n_sensors, const hdr_sensor_desc *sensors) {
  if (!ctx) return fail(HDR_E_INVALID, "ctx is NULL");
  if (rig_id < 0 || rig_id >= kMaxRigs) return fail(HDR_E_INVALID, "rig_id %d not in [0,%d)", rig_id, kMaxRigs);
  hdr_status vst = check_sensors(n_sensors, sensors);
  if (vst) return vst;
  CUDA_TRY(cudaSetDevice(ctx->device));
  Rig &rig = ctx->rigs[rig_id];
  if (rig.n) {
    CUDA_TRY(cudaDeviceSynchronize());
    free_rig(rig);
  }
  Rig fresh;
  fresh.n = n_sensors;
  for (int s = 0; s < n_sensors; s++) {
    RigSensor &rs = fresh.s[s];
    rs.d = sensors[s];
    const size_t npx = (size_t)rs.d.width * rs.d.height;
    auto up = [&](const void *src, size_t bytes, void **dst) -> cudaError_t {
      if (!src) return cudaSuccess;
      cudaError_t e = cudaMalloc(dst, bytes);
      if (e != cudaSuccess) return e;
      return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
    };
    cudaError_t e = up(rs.d.bias_frame, npx * 4, (void **)&rs.bias);
    if (e == cudaSuccess) e = up(rs.d.prnu_frame, npx * 4, (void **)&rs.prnu);
    if (e == cudaSuccess) e = up(rs.d.read_var_frame, npx * 4, (void **)&rs.rvar);
    if (e == cudaSuccess) e = up(rs.d.sat_frame, npx * 2, (void **)&rs.satf);
    rs.d.bias_frame = rs.d.prnu_frame = rs.d.read_var_frame = nullptr;
    rs.d.sat_frame = nullptr;
    if (e != cudaSuccess) {
      free_rig(fresh);
      return fail(e == cudaErrorMemoryAllocation ? HDR_E_NOMEM : HDR_E_CUDA, "rig upload failed: %s",
                  cudaGetErrorString(e));
    }
  }
  rig = fresh;
  for (int s = 0; s < n_sensors; s++) fresh.s[s] = RigSensor();   // ownership moved
  fresh.n = 0;
  ctx->rig_gen[rig_id]++;  // plans made for the previous rig no longer match
  return HDR_OK;
}

hdr_status hdr_reconstruct(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                           void *out_dev, uint8_t *choice_dev, void *cuda_stream) {
  return reconstruct_impl(ctx, rig_id, params, raw_dev, out_dev, choice_dev, nullptr, cuda_stream);
}

hdr_status hdr_reconstruct_levels(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                  const uint16_t *const *raw_dev, void *out_dev, uint8_t *choice_dev,
                                  float *levels_dev, void *cuda_stream) {
  if (!levels_dev && (long long)params->out_w * params->out_h > 0) return fail(HDR_E_INVALID, "levels_dev is NULL");
  return reconstruct_impl(ctx, rig_id, params, raw_dev, out_dev, choice_dev, levels_dev, cuda_stream);
}

}  // extern "C"

namespace {

// Device staging of the host-buffer entry points, grown on demand (growing waits for `stream`):
// one raw frame per sensor, the output planes and, when asked for, the level map.
hdr_status ensure_host_staging(hdr_ctx *ctx, const Rig &rig, const hdr_params *params, const uint16_t *const *raw_host,
                               bool want_choice, cudaStream_t stream, const uint16_t **raw_dev) {
  for (int s = 0; s < rig.n; s++) {
    if (!raw_host[s]) return fail(HDR_E_INVALID, "raw_host[%d] is NULL", s);
    const size_t bytes = (size_t)rig.s[s].d.pitch_elems * rig.s[s].d.height * 2;
    if (ctx->raw_cap[s] < bytes) {
      CUDA_TRY(cudaStreamSynchronize(stream));
      cudaFree(ctx->raw_stage[s]);
      ctx->raw_stage[s] = nullptr;
      ctx->raw_cap[s] = 0;
      CUDA_TRY(cudaMalloc(&ctx->raw_stage[s], bytes));
      ctx->raw_cap[s] = bytes;
    }
    raw_dev[s] = ctx->raw_stage[s];
  }
  const size_t npx = (size_t)params->out_w * params->out_h * 3;
  const size_t obytes = npx * (params->out_dtype ? 2 : 4);
  if (ctx->out_cap < obytes) {
    CUDA_TRY(cudaStreamSynchronize(stream));
    cudaFree(ctx->out_stage);
    ctx->out_stage = nullptr;
    ctx->out_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->out_stage, obytes));
    ctx->out_cap = obytes;
  }
  if (want_choice && ctx->choice_cap < npx) {
    CUDA_TRY(cudaStreamSynchronize(stream));
    cudaFree(ctx->choice_stage);
    ctx->choice_stage = nullptr;
    ctx->choice_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->choice_stage, npx));
    ctx->choice_cap = npx;
  }
  return HDR_OK;
}

}  // namespace

extern "C" {

hdr_status hdr_reconstruct_adaptive_host(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params,
                                         const hdr_calpa_params *calpa, const uint16_t *const *raw_host,
                                         void *out_host, uint8_t *choice_host, void *cuda_stream) {
  hdr_status st = common_checks(ctx, rig_id, params, raw_host, out_host);
  if (st) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const Rig &rig = ctx->rigs[rig_id];
  const uint16_t *raw_dev[HDR_MAX_SENSORS];
  st = ensure_host_staging(ctx, rig, params, raw_host, choice_host != nullptr, stream, raw_dev);
  if (st) return st;
  for (int s = 0; s < rig.n; s++)
    CUDA_TRY(cudaMemcpyAsync(ctx->raw_stage[s], raw_host[s], (size_t)rig.s[s].d.pitch_elems * rig.s[s].d.height * 2,
                             cudaMemcpyHostToDevice, stream));
  st = hdr_reconstruct_adaptive(ctx, rig_id, params, calpa, raw_dev, ctx->out_stage,
                                choice_host ? ctx->choice_stage : nullptr, cuda_stream);
  if (st) return st;
  const size_t npx = (size_t)params->out_w * params->out_h * 3;
  if (npx) {
    CUDA_TRY(cudaMemcpyAsync(out_host, ctx->out_stage, npx * (params->out_dtype ? 2 : 4), cudaMemcpyDeviceToHost,
                             stream));
    if (choice_host) CUDA_TRY(cudaMemcpyAsync(choice_host, ctx->choice_stage, npx, cudaMemcpyDeviceToHost, stream));
  }
  CUDA_TRY(cudaStreamSynchronize(stream));
  return HDR_OK;
}

hdr_status hdr_reconstruct_host(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_host,
                                void *out_host, uint8_t *choice_host, void *cuda_stream) {
  hdr_status st = common_checks(ctx, rig_id, params, raw_host, out_host);
  if (st) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const Rig &rig = ctx->rigs[rig_id];
  const uint16_t *raw_dev[HDR_MAX_SENSORS];
  st = ensure_host_staging(ctx, rig, params, raw_host, choice_host != nullptr, stream, raw_dev);
  if (st) return st;
  const size_t plane = (size_t)params->out_w * params->out_h;
  const size_t esize = params->out_dtype ? 2 : 4;
  LpaLaunch L;
  float2 *conv = nullptr;
  st = conv_buffer(ctx, rig, params, &conv);
  if (st) return st;
  st = cached_plan(ctx, rig_id, params, raw_dev, L, true, LPA_FRAME_STAGES, conv);
  if (st) return st;
  L.out = ctx->out_stage;
  L.choice = choice_host ? ctx->choice_stage : nullptr;
  L.levels = nullptr;
  if (!ctx->h2d) {
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->band2, cudaStreamNonBlocking));
    for (int b = 0; b < kMaxBands; b++) {
      CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_in[b], cudaEventDisableTiming));
      CUDA_TRY(cudaEventCreateWithFlags(&ctx->ev_done[b], cudaEventDisableTiming));
    }
  }
  // Bands of tile rows: the raw rows a band's windows can reach are copied in (on the copy
  // stream) while the previous band is reconstructed, and a finished band's output rows are
  // copied out while the next one is reconstructed. Consecutive bands run on two streams
  // (`stream` and a second one; a band waits only for its own input rows), so that a band's first
  // CTAs fill the SMs its predecessor's last wave leaves idle.
  const int rows = L.tiles_y;
  const int nb = std::max(1, std::min(LPA_HOST_BANDS, rows / 8));
  const int nstreams = LPA_HOST_BAND_STREAMS;
  size_t have[HDR_MAX_SENSORS] = {};
  CUDA_TRY(cudaEventRecord(ctx->ev_done[0], stream));  // the copies start after earlier work on `stream`
  CUDA_TRY(cudaStreamWaitEvent(ctx->h2d, ctx->ev_done[0], 0));
  if (nstreams > 1 && nb > 1) CUDA_TRY(cudaStreamWaitEvent(ctx->band2, ctx->ev_done[0], 0));
  bool converted = false;
  for (int b = 0; b < nb; b++) {
    cudaStream_t sb = (nstreams > 1 && (b & 1)) ? ctx->band2 : stream;
    const int r0 = rows * b / nb, r1 = rows * (b + 1) / nb;
    const int v0 = r0 * L.tile_h, v1 = std::min(r1 * L.tile_h, params->out_h);
    LpaRows R{};  // the rows this band copies in, converted behind their copy on the copy stream
    bool fresh = false;
    for (int s = 0; s < rig.n; s++) {
      const LpaSensorK &Sk = L.s[s];
      const int H = rig.s[s].d.height;
      size_t need = (size_t)H;
      if (b + 1 < nb) {  // the last band takes every remaining row
        double ymax = -1e300;
        for (int k = 0; k < 4; k++) {
          const double uu = (k & 1) ? params->out_w - 1 : 0, vv = (k & 2) ? v1 - 1 : v0;
          ymax = std::max(ymax, Sk.G[3] * uu + Sk.G[4] * vv + Sk.G[5]);
        }
        // every staged box row of the band's tiles lies below the lowest window row + box height
        const double lim = std::min<double>(H, std::max(0.0, std::ceil(ymax) + Sk.box_h + 2));
        need = std::max(have[s], (size_t)lim);
      }
      if (need > have[s]) {
        const size_t row_bytes = (size_t)rig.s[s].d.pitch_elems * 2;
        CUDA_TRY(cudaMemcpyAsync(ctx->raw_stage[s] + have[s] * rig.s[s].d.pitch_elems,
                                 raw_host[s] + have[s] * rig.s[s].d.pitch_elems, (need - have[s]) * row_bytes,
                                 cudaMemcpyHostToDevice, ctx->h2d));
        R.r0[s] = (int)have[s];
        R.r1[s] = (int)need;
        fresh = true;
        have[s] = need;
      }
    }
    if (L.conv && fresh) {
      st = convert_rows(ctx, L, R, !converted, ctx->h2d);
      if (st) return st;
      converted = true;
    }
    CUDA_TRY(cudaEventRecord(ctx->ev_in[b], ctx->h2d));
    CUDA_TRY(cudaStreamWaitEvent(sb, ctx->ev_in[b], 0));
    L.tile0 = r0 * L.tiles_x;
    L.tile_count = (r1 - r0) * L.tiles_x;
    if (L.tile_count > 0) {
      st = launch(L, params->accum, false, sb);
      if (st) return st;
    }
    CUDA_TRY(cudaEventRecord(ctx->ev_done[b], sb));
    CUDA_TRY(cudaStreamWaitEvent(ctx->d2h, ctx->ev_done[b], 0));
    if (v1 > v0) {
      const size_t off = (size_t)v0 * params->out_w, n = (size_t)(v1 - v0) * params->out_w;
      for (int c = 0; c < 3; c++) {
        CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(out_host) + (c * plane + off) * esize,
                                 static_cast<char *>(ctx->out_stage) + (c * plane + off) * esize, n * esize,
                                 cudaMemcpyDeviceToHost, ctx->d2h));
        if (choice_host)
          CUDA_TRY(cudaMemcpyAsync(choice_host + c * plane + off, ctx->choice_stage + c * plane + off, n,
                                   cudaMemcpyDeviceToHost, ctx->d2h));
      }
    }
  }
  // `stream` is ordered after every band and copy (the call returns when they are done)
  CUDA_TRY(cudaEventRecord(ctx->ev_in[0], ctx->d2h));
  CUDA_TRY(cudaStreamWaitEvent(stream, ctx->ev_in[0], 0));
  if (converted) CUDA_TRY(cudaEventRecord(ctx->conv_ev, stream));
  CUDA_TRY(cudaStreamSynchronize(ctx->d2h));
  CUDA_TRY(cudaStreamSynchronize(stream));
  return HDR_OK;
}

hdr_status hdr_check(hdr_ctx *ctx, void *cuda_stream) {
  if (!ctx) return fail(HDR_E_INVALID, "ctx is NULL");
  CUDA_TRY(cudaSetDevice(ctx->device));
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)cuda_stream));
  CUDA_TRY(cudaGetLastError());
  unsigned int word = 0;
  CUDA_TRY(cudaMemcpy(&word, ctx->status, sizeof(word), cudaMemcpyDeviceToHost));
  if (word) CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(word)));
  if (word & LPA_ERR_TIMEOUT) return fail(HDR_E_TIMEOUT, "a bounded device wait ran out (status 0x%x)", word);
  if (word & LPA_ERR_BOUNDS) return fail(HDR_E_INTERNAL, "a window left the staged footprint (status 0x%x)", word);
  return HDR_OK;
}

hdr_status hdr_selftest_timeout(hdr_ctx *ctx, void *cuda_stream) {
  if (!ctx) return fail(HDR_E_INVALID, "ctx is NULL");
  CUDA_TRY(cudaSetDevice(ctx->device));
  CUDA_TRY(lpa_launch_selftest_wait(ctx->status, (cudaStream_t)cuda_stream));
  return HDR_OK;
}

const char *hdr_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ------------------------------------------------------------------ batched launch

namespace {

// Relative cost of a frame's tile (for the most-expensive-first order): order weight x sensors
// x summed squared scales (the expected samples per window).
double frame_cost(const hdr_params &p, int n_sensors) {
  static const double order_w[3] = {11.0, 41.0, 92.0};
  double s2 = 0.0;
  for (int j = 0; j < p.n_scales; j++) s2 += p.sigma[j] * p.sigma[j];
  return order_w[p.order] * n_sensors * s2;
}

uint64_t batch_kind(const hdr_ctx *ctx, int n, const hdr_frame *frames) {
  uint64_t orders = 0, max_s = 0, scales = 0, px = 0, adaptive = 0;
  for (int f = 0; f < n; f++) {
    const hdr_params *p = frames[f].params;
    orders |= 1ull << p->order;
    adaptive |= frames[f].calpa ? 1 : 0;
    max_s = std::max<uint64_t>(max_s, ctx->rigs[frames[f].rig_id].n);
    scales = std::max<uint64_t>(scales, p->n_scales);
    px += (uint64_t)p->out_w * p->out_h;
  }
  uint64_t bucket = 0;
  while ((1ull << (bucket + 1)) <= px / 65536 + 1) bucket++;
  return orders | (max_s << 4) | (scales << 8) | (bucket << 12) | ((uint64_t)frames[0].params->accum << 20) |
         (adaptive << 21);
}

hdr_status check_batch(hdr_ctx *ctx, int32_t n, const hdr_frame *frames) {
  if (!ctx) return fail(HDR_E_INVALID, "ctx is NULL");
  if (n < 1 || n > 4096) return fail(HDR_E_INVALID, "n_frames %d not in [1, 4096]", n);
  if (!frames) return fail(HDR_E_INVALID, "frames is NULL");
  for (int f = 0; f < n; f++) {
    const hdr_frame &F = frames[f];
    if (F.rig_id < 0 || F.rig_id >= kMaxRigs || ctx->rigs[F.rig_id].n == 0)
      return fail(HDR_E_INVALID, "frame %d: rig %d is not defined", f, F.rig_id);
    hdr_status st = check_params(F.params);
    if (st) return st;
    if (F.params->weight_mode != 0)
      return fail(HDR_E_UNSUPPORTED, "frame %d: batches use the inverse-variance weight (weight_mode 0)", f);
    if (F.params->accum != frames[0].params->accum)
      return fail(HDR_E_INVALID, "frame %d: all frames of a batch must use the same accum", f);
    if (!F.out_dev && (long long)F.params->out_w * F.params->out_h > 0)
      return fail(HDR_E_INVALID, "frame %d: output pointer is NULL", f);
    if (F.calpa) {
      st = lpa_check_calpa(F.calpa);
      if (st) return fail(st, "frame %d: %s", f, g_err.c_str());
    }
  }
  return HDR_OK;
}

// Grow the device tables and both pinned staging buffers of the batched launch (waits for the
// launches in flight first; graphs recorded on the old tables are dropped).
hdr_status batch_reserve(hdr_ctx *ctx, size_t n_frames, size_t n_tiles) {
  BatchState &B = ctx->batch;
  if (!B.counters_dev) {
    CUDA_TRY(cudaMalloc(&B.counters_dev, 3 * sizeof(unsigned int)));
    CUDA_TRY(cudaMalloc(&B.bounds_dev, 4 * sizeof(int)));
    for (auto &S : B.stage) {
      CUDA_TRY(cudaMallocHost(&S.bounds, 4 * sizeof(int)));
      CUDA_TRY(cudaEventCreateWithFlags(&S.done, cudaEventDisableTiming));
    }
  }
  if (n_frames <= B.cap_frames && n_tiles <= B.cap_tiles) return HDR_OK;
  for (auto &S : B.stage)
    if (S.pending) {
      CUDA_TRY(cudaEventSynchronize(S.done));
      S.pending = false;
    }
  for (auto &g : B.graphs) cudaGraphExecDestroy(g.second);
  B.graphs.clear();
  if (n_frames > B.cap_frames) {
    size_t cap = std::max<size_t>(n_frames, 2 * B.cap_frames);
    cudaFree(B.frames_dev);
    B.frames_dev = nullptr;
    B.cap_frames = 0;
    for (auto &S : B.stage) {
      cudaFreeHost(S.frames);
      S.frames = nullptr;
    }
    CUDA_TRY(cudaMalloc(&B.frames_dev, cap * sizeof(LpaLaunch)));
    for (auto &S : B.stage) CUDA_TRY(cudaMallocHost(&S.frames, cap * sizeof(LpaLaunch)));
    B.cap_frames = cap;
  }
  if (n_tiles > B.cap_tiles) {
    size_t cap = std::max<size_t>(n_tiles, 2 * B.cap_tiles);
    cudaFree(B.tiles_dev);
    B.tiles_dev = nullptr;
    B.cap_tiles = 0;
    for (auto &S : B.stage) {
      cudaFreeHost(S.tiles);
      S.tiles = nullptr;
    }
    CUDA_TRY(cudaMalloc(&B.tiles_dev, cap * sizeof(int2)));
    for (auto &S : B.stage) CUDA_TRY(cudaMallocHost(&S.tiles, cap * sizeof(int2)));
    B.cap_tiles = cap;
  }
  return HDR_OK;
}

// Plan every frame into the pinned staging and write the tile list (all tiles of each frame, or
// the tiles [ranges[f].x, ranges[f].y) when ranges is given), grouped by polynomial order. Returns
// each order's tile count and the shared memory its kernel needs.
hdr_status batch_plan(hdr_ctx *ctx, int n, const hdr_frame *frames, const int2 *ranges, const hdr_batch_config &cfg,
                      uint32_t smem[3], int n_tiles[3]) {
  BatchState &B = ctx->batch;
  std::vector<LpaLaunch> plans(n);
  size_t total = 0;
  for (int o = 0; o < 3; o++) smem[o] = 0, n_tiles[o] = 0;
  for (int f = 0; f < n; f++) {
    const hdr_frame &F = frames[f];
    // no tables: the persistent kernels search every window
    hdr_status st = plan_env(PlanEnv{ctx->encode, ctx->status, ctx->device, &ctx->tabs, false}, ctx->rigs[F.rig_id],
                             F.params, F.raw_dev, plans[f], cfg.tile_h);
    if (st) return fail(st, "frame %d: %s", f, g_err.c_str());
    if (plans[f].mode != LPA_SEARCHED && plans[f].mode != LPA_SEARCHED_F32)
      return fail(HDR_E_INTERNAL, "frame %d: the persistent form searches windows", f);
    plans[f].out = F.out_dev;
    plans[f].choice = F.choice_dev;
    plans[f].levels = nullptr;
    const int nt = plans[f].tiles_x * plans[f].tiles_y;
    if (ranges && (ranges[f].x < 0 || ranges[f].y > nt || ranges[f].x > ranges[f].y))
      return fail(HDR_E_INVALID, "frame %d: tile range [%d, %d) outside [0, %d)", f, ranges[f].x, ranges[f].y, nt);
    const size_t cnt = ranges ? (size_t)(ranges[f].y - ranges[f].x) : (size_t)nt;
    total += cnt;
    if (cnt) smem[plans[f].order] = std::max(smem[plans[f].order], plans[f].smem_bytes);
  }
  if (total > (size_t)INT32_MAX) return fail(HDR_E_UNSUPPORTED, "too many tiles in one batch");
  hdr_status st = batch_reserve(ctx, n, std::max<size_t>(total, 1));
  if (st) return st;
  BatchState::Staging &S = B.stage[B.cur];
  if (S.pending) {  // the launch before the previous one may still be reading this buffer
    CUDA_TRY(cudaEventSynchronize(S.done));
    S.pending = false;
  }
  std::vector<int> order(n);
  for (int f = 0; f < n; f++) order[f] = f;
  std::vector<double> cost(n, 0.0);
  if (cfg.cost_order)
    for (int f = 0; f < n; f++) cost[f] = frame_cost(*frames[f].params, ctx->rigs[frames[f].rig_id].n);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (plans[a].order != plans[b].order) return plans[a].order < plans[b].order;
    return cost[a] > cost[b];
  });
  size_t t = 0;
  S.bounds[0] = 0;
  for (int k = 0; k < n; k++) {
    const int f = order[k];
    S.frames[f] = plans[f];
    const int t0 = ranges ? ranges[f].x : 0;
    const int t1 = ranges ? ranges[f].y : plans[f].tiles_x * plans[f].tiles_y;
    for (int i = t0; i < t1; i++) S.tiles[t++] = make_int2(f, i);
    n_tiles[plans[f].order] += t1 - t0;
  }
  S.bounds[1] = n_tiles[0];
  S.bounds[2] = n_tiles[0] + n_tiles[1];
  S.bounds[3] = (int)total;
  return HDR_OK;
}

// Form 0 of a batched launch: one grid per frame (tiles [ranges[f].x, ranges[f].y) of frame f, or
// all of them) as independent kernel nodes of one graph, recorded once per shape; a replay only
// updates the nodes' parameters.
hdr_status batch_run_frames(hdr_ctx *ctx, int n, const hdr_frame *frames, const int2 *ranges,
                            const hdr_batch_config &cfg, cudaStream_t stream, float *const *scratch,
                            float2 *const *conv_in, bool conv_done) {
  BatchState &B = ctx->batch;
  TableHold hold(ctx->tabs);  // the plans of every frame stay valid until the launch
  std::vector<LpaLaunch> plans(n);
  std::vector<int> grid(n, 0);
  // frames converted ahead (lpa_conv_eligible; not with two staging buffers) into the caller's
  // buffers, else into the context's buffer, one slice per frame
  std::vector<float2 *> cv(n, nullptr);
  bool ctx_conv = false;
  if (cfg.stages != 2) {
    if (conv_in) {
      for (int f = 0; f < n; f++) cv[f] = conv_in[f];
    } else {
      size_t total = 0;
      for (int f = 0; f < n; f++)
        if (lpa_conv_eligible(frames[f].params, frames[f].calpa != nullptr)) total += conv_elems(ctx->rigs[frames[f].rig_id]);
      if (total) {
        hdr_status st = conv_capacity(ctx, total);
        if (st) return st;
        float2 *p = ctx->conv_buf;
        for (int f = 0; f < n; f++)
          if (lpa_conv_eligible(frames[f].params, frames[f].calpa != nullptr)) {
            cv[f] = p;
            p += conv_elems(ctx->rigs[frames[f].rig_id]);
          }
        ctx_conv = true;
      }
    }
  }
  // adaptive frames: gradients and steering matrices (5 floats per output pixel) in the caller's
  // scratch, else in one context buffer shared by the batch
  std::vector<float *> aux(n, nullptr);
  if (!scratch) {
    size_t total = 0;
    for (int f = 0; f < n; f++)
      if (frames[f].calpa) total += (size_t)frames[f].params->out_w * frames[f].params->out_h * 5;
    if (total) {
      void *base = nullptr;
      hdr_status st = lpa_ctx_calpa_scratch(ctx, total * sizeof(float), &base);
      if (st) return st;
      float *p = static_cast<float *>(base);
      for (int f = 0; f < n; f++)
        if (frames[f].calpa) {
          aux[f] = p;
          p += (size_t)frames[f].params->out_w * frames[f].params->out_h * 5;
        }
    }
  } else {
    for (int f = 0; f < n; f++) aux[f] = frames[f].calpa ? scratch[f] : nullptr;
  }
  for (int f = 0; f < n; f++) {
    const hdr_frame &F = frames[f];
    const size_t npx = (size_t)F.params->out_w * F.params->out_h;
    if (F.calpa && npx > 0 && !aux[f]) return fail(HDR_E_INVALID, "frame %d: no scratch for the adaptive passes", f);
    // the adaptive passes 1 and 2 of a frame run with the launch that takes its first tile
    if (F.calpa && npx > 0 && (!ranges || ranges[f].x == 0)) {
      hdr_status st = lpa_calpa_prepare(ctx, F.rig_id, F.params, F.calpa, F.raw_dev, aux[f], stream);
      if (st) return fail(st, "frame %d: %s", f, g_err.c_str());
    }
    hdr_params sp;
    const hdr_params *pp = F.params;
    if (F.calpa) {  // the steered window is searched (offsets and weights differ per pixel)
      sp = *F.params;
      sp.tab_weights = 0;
      pp = &sp;
    }
    const int px = (cfg.px_per_thread == 2 && !F.calpa) ? 2 : 1;
    hdr_status st = plan_env(PlanEnv{ctx->encode, ctx->status, ctx->device, &ctx->tabs, !F.calpa}, ctx->rigs[F.rig_id],
                             pp, F.raw_dev, plans[f], F.calpa ? 16 : cfg.tile_h,
                             F.calpa ? lpa_calpa_reach(F.calpa) : 1.0, (F.calpa || px != 1) ? 1 : cfg.stages,
                             F.calpa ? nullptr : cv[f]);
    if (st) return fail(st, "frame %d: %s", f, g_err.c_str());
    if (F.calpa) {
      plans[f].mode = lpa_mode_f32(plans[f].mode) ? LPA_STEERED_F32 : LPA_STEERED;
      plans[f].aux = aux[f] + npx * 2;  // the steering matrices
    }
    plans[f].px = px;
    plans[f].out = F.out_dev;
    plans[f].choice = F.choice_dev;
    plans[f].levels = nullptr;
    const int nt = plans[f].tiles_x * plans[f].tiles_y;
    if (ranges && (ranges[f].x < 0 || ranges[f].y > nt || ranges[f].x > ranges[f].y))
      return fail(HDR_E_INVALID, "frame %d: tile range [%d, %d) outside [0, %d)", f, ranges[f].x, ranges[f].y, nt);
    plans[f].tile0 = ranges ? ranges[f].x : 0;
    grid[f] = ranges ? ranges[f].y - ranges[f].x : nt;
  }
  std::vector<int> order;
  for (int f = 0; f < n; f++)
    if (grid[f] > 0) order.push_back(f);
  if (cfg.cost_order) {
    std::vector<double> cost(n);
    for (int f = 0; f < n; f++)
      cost[f] = frame_cost(*frames[f].params, ctx->rigs[frames[f].rig_id].n) * grid[f] * (frames[f].calpa ? 3.0 : 1.0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  }
  if (order.empty()) return HDR_OK;
  const bool comp = frames[0].params->accum != 0;
  // graph nodes: each frame's reconstruction grid, behind its conversion where the frame is
  // converted ahead and this launch takes its first tile
  std::vector<std::array<int64_t, 5>> key;
  std::vector<cudaKernelNodeParams> kp;
  std::vector<int> dep;
  std::vector<LpaRows> rows(n);
  std::vector<std::array<void *, 2>> args;
  args.reserve(2 * order.size());
  for (size_t k = 0; k < order.size(); k++) {
    const int f = order[k];
    const LpaLaunch &L = plans[f];
    int d = -1;
    if (L.conv && !conv_done && (!ranges || ranges[f].x == 0)) {
      rows[f] = all_rows(L);
      args.push_back({&plans[f], &rows[f]});
      cudaKernelNodeParams c{};
      c.func = const_cast<void *>(lpa_convert_kernel(L.mode == LPA_LITERAL));
      c.gridDim = lpa_convert_grid(L, rows[f]);
      c.blockDim = dim3(256);
      c.sharedMemBytes = 0;
      c.kernelParams = args.back().data();
      key.push_back({-1, L.mode == LPA_LITERAL ? 1 : 0, 0, 0, 0});
      d = (int)kp.size();
      kp.push_back(c);
      dep.push_back(-1);
    }
    const void *fn = lpa_kernel(L.order, comp, false, L.mode, L.tile_h, L.px, L.stages);
    if (!fn)
      return fail(HDR_E_INTERNAL, "no kernel for order %d, mode %d, tile height %d, %d pixels per thread, %d stages",
                  L.order, L.mode, L.tile_h, L.px, L.stages);
    CUDA_TRY(lpa_opt_in(fn));
    // grid size and shared memory are set on each replay: graphs are kept per sequence of kernels
    key.push_back({L.order * 8 + L.mode, comp ? 1 : 0, L.tile_h, L.px, L.stages + 4 * (d >= 0 ? 1 : 0)});
    args.push_back({&plans[f], nullptr});
    cudaKernelNodeParams r{};
    r.func = const_cast<void *>(fn);
    r.gridDim = dim3((unsigned)lpa_grid_ctas(grid[f], L.stages));
    r.blockDim = dim3((unsigned)(LPA_TILE * L.tile_h / L.px));
    r.sharedMemBytes = L.smem_bytes;
    r.kernelParams = args.back().data();
    kp.push_back(r);
    dep.push_back(d);
  }
  auto it = B.frame_graphs.find(key);
  if (it != B.frame_graphs.end()) {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < kp.size() && e == cudaSuccess; k++)
      e = cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.nodes[k], &kp[k]);
    if (e != cudaSuccess) {  // an update the driver refuses: record the graph again
      cudaGetLastError();
      cudaGraphExecDestroy(it->second.exec);
      cudaGraphDestroy(it->second.graph);
      B.frame_graphs.erase(it);
      it = B.frame_graphs.end();
    }
  }
  if (it == B.frame_graphs.end()) {
    if (B.frame_graphs.size() >= 256) {  // kernel sequences that never repeat: start over
      for (auto &g : B.frame_graphs) {
        cudaGraphExecDestroy(g.second.exec);
        cudaGraphDestroy(g.second.graph);
      }
      B.frame_graphs.clear();
    }
    BatchState::FrameGraph fg;
    cudaError_t e = cudaGraphCreate(&fg.graph, 0);
    fg.nodes.resize(kp.size());
    for (size_t k = 0; k < kp.size() && e == cudaSuccess; k++)
      e = cudaGraphAddKernelNode(&fg.nodes[k], fg.graph, dep[k] >= 0 ? &fg.nodes[dep[k]] : nullptr, dep[k] >= 0 ? 1 : 0,
                                 &kp[k]);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&fg.exec, fg.graph, 0);
    if (e != cudaSuccess) {
      if (fg.graph) cudaGraphDestroy(fg.graph);
      return fail(HDR_E_CUDA, "recording the batch graph failed: %s", cudaGetErrorString(e));
    }
    it = B.frame_graphs.emplace(key, fg).first;
  }
  // the context's conversion buffer: after its previous users, and before its next ones
  if (ctx_conv) CUDA_TRY(cudaStreamWaitEvent(stream, ctx->conv_ev, 0));
  CUDA_TRY(cudaGraphLaunch(it->second.exec, stream));
  if (ctx_conv) CUDA_TRY(cudaEventRecord(ctx->conv_ev, stream));
  return HDR_OK;
}

}  // namespace

// One batched launch over the listed tiles of several frames (see hdr_reconstruct_batch).
hdr_status lpa_batch_run(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames, const int2 *ranges,
                         const hdr_batch_config *cfg_in, cudaStream_t stream, float *const *scratch,
                         float2 *const *conv, bool conv_done) {
  hdr_status st = check_batch(ctx, n_frames, frames);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  hdr_batch_config cfg = {16, 0, 1, 0, 1, 1};
  if (cfg_in) {
    cfg = *cfg_in;
  } else {
    auto it = ctx->batch.tuned.find(batch_kind(ctx, n_frames, frames));
    if (it != ctx->batch.tuned.end()) cfg = it->second;
  }
  if (cfg.tile_h != 8 && cfg.tile_h != 16) return fail(HDR_E_INVALID, "tile_h must be 8 or 16");
  if (cfg.ctas_per_sm < 0 || cfg.ctas_per_sm > 8) return fail(HDR_E_INVALID, "ctas_per_sm must be in [0, 8]");
  if (cfg.form != 0 && cfg.form != 1) return fail(HDR_E_INVALID, "form must be 0 or 1");
  if (cfg.px_per_thread < 0 || cfg.px_per_thread > 2) return fail(HDR_E_INVALID, "px_per_thread must be 0, 1 or 2");
  if (cfg.px_per_thread == 2 && (cfg.tile_h != 16 || cfg.form != 0))
    return fail(HDR_E_INVALID, "two pixels per thread need tile_h 16 and form 0");
  if (cfg.stages < 0 || cfg.stages > 2) return fail(HDR_E_INVALID, "stages must be 0, 1 or 2");
  if (cfg.stages == 2 && (cfg.px_per_thread == 2 || cfg.form != 0))
    return fail(HDR_E_INVALID, "two staging buffers need one pixel per thread and form 0");
  for (int f = 0; f < n_frames; f++)
    if (frames[f].calpa) cfg.form = 0;  // the persistent kernels have no steered window
  if (cfg.form == 0) return batch_run_frames(ctx, n_frames, frames, ranges, cfg, stream, scratch, conv, conv_done);
  uint32_t smem[3];
  int n_tiles[3];
  st = batch_plan(ctx, n_frames, frames, ranges, cfg, smem, n_tiles);
  if (st) return st;
  BatchState &B = ctx->batch;
  const bool comp = frames[0].params->accum != 0;
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  const int buf = B.cur;
  BatchState::Staging &S = B.stage[buf];
  BatchState::Key key{comp ? 1 : 0, cfg.tile_h, buf, {0, 0, 0}, {0, 0, 0}, B.cap_frames, B.cap_tiles};
  for (int o = 0; o < 3; o++) {
    if (n_tiles[o] == 0) continue;
    const int fit = lpa_batch_ctas_per_sm(o, comp, cfg.tile_h, smem[o]);
    if (fit < 1)
      return fail(HDR_E_UNSUPPORTED, "the order-%d batched kernel does not fit an SM with %u bytes of shared memory", o,
                  smem[o]);
    const int per_sm = cfg.ctas_per_sm > 0 ? std::min(cfg.ctas_per_sm, fit) : fit;
    // Small segments get a power-of-two grid (extra CTAs find no tile and leave), so the number
    // of recorded graphs stays small when the tile counts change from launch to launch.
    int grid = sms * per_sm;
    if (n_tiles[o] < grid) {
      int g = 1;
      while (g < n_tiles[o]) g *= 2;
      grid = std::min(grid, g);
    }
    key.grid[o] = grid;
    key.smem[o] = smem[o];
  }
  auto it = B.graphs.find(key);
  if (it == B.graphs.end()) {
    // record: tables from this buffer's pinned staging, counters to zero, then one persistent
    // kernel per order present, as parallel branches so that one order's tail overlaps the next
    cudaStream_t cap = nullptr, side[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    for (int o = 0; o < 3 && e == cudaSuccess; o++) {
      e = cudaStreamCreateWithFlags(&side[o], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[o], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    cudaGraph_t g = nullptr;
    bool capturing = false;
    if (e == cudaSuccess) {
      e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      capturing = e == cudaSuccess;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B.frames_dev, S.frames, B.cap_frames * sizeof(LpaLaunch), cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(B.tiles_dev, S.tiles, B.cap_tiles * sizeof(int2), cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B.bounds_dev, S.bounds, 4 * sizeof(int), cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(B.counters_dev, 0, 3 * sizeof(unsigned int), cap);
    if (e == cudaSuccess) e = cudaEventRecord(fork, cap);
    for (int o = 0; o < 3 && e == cudaSuccess; o++) {
      if (!key.grid[o]) continue;
      e = cudaStreamWaitEvent(side[o], fork, 0);
      LpaBatch lb{B.frames_dev, B.tiles_dev, B.bounds_dev, B.counters_dev, smem[o]};
      if (e == cudaSuccess) e = lpa_launch_batch(o, lb, comp, cfg.tile_h, key.grid[o], side[o]);
      if (e == cudaSuccess) e = cudaEventRecord(join[o], side[o]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, join[o], 0);
    }
    if (capturing) {
      cudaError_t e2 = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = e2;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    for (int o = 0; o < 3; o++) {
      if (side[o]) cudaStreamDestroy(side[o]);
      if (join[o]) cudaEventDestroy(join[o]);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(HDR_E_CUDA, "recording the batch graph failed: %s", cudaGetErrorString(e));
    it = B.graphs.emplace(key, exec).first;
  }
  // The device tables are shared by both buffers: a launch on another stream must not overwrite
  // them while the previous launch still runs.
  const BatchState::Staging &prev = B.stage[buf ^ 1];
  if (prev.pending) CUDA_TRY(cudaStreamWaitEvent(stream, prev.done, 0));
  CUDA_TRY(cudaGraphLaunch(it->second, stream));
  CUDA_TRY(cudaEventRecord(S.done, stream));
  S.pending = true;
  B.cur = buf ^ 1;
  return HDR_OK;
}

int lpa_ctx_device(const hdr_ctx *ctx) { return ctx->device; }
int lpa_ctx_rig_sensors(const hdr_ctx *ctx, int rig_id) {
  return (rig_id >= 0 && rig_id < kMaxRigs) ? ctx->rigs[rig_id].n : 0;
}
void lpa_ctx_rig_sizes(const hdr_ctx *ctx, int rig_id, int *pitch, int *height) {
  const Rig &r = ctx->rigs[rig_id];
  for (int s = 0; s < r.n; s++) {
    pitch[s] = r.s[s].d.pitch_elems;
    height[s] = r.s[s].d.height;
  }
}
hdr_status lpa_fail(hdr_status st, const char *msg) { return fail(st, "%s", msg); }
size_t lpa_conv_elems(const hdr_ctx *ctx, int rig_id) { return conv_elems(ctx->rigs[rig_id]); }
hdr_status lpa_convert_frame(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                             float2 *conv, cudaStream_t st) {
  LpaLaunch L;
  hdr_status s = plan_env(PlanEnv{ctx->encode, ctx->status, ctx->device, &ctx->tabs, true}, ctx->rigs[rig_id], params,
                          raw_dev, L, 16, 1.0, 1, conv);
  if (s) return s;
  cudaError_t e = lpa_launch_convert(L, all_rows(L), L.mode == LPA_LITERAL, st);
  if (e != cudaSuccess) return fail(HDR_E_CUDA, "conversion launch failed: %s", cudaGetErrorString(e));
  return HDR_OK;
}
hdr_status lpa_ctx_calpa_scratch(hdr_ctx *ctx, size_t bytes, void **ptr) {
  if (bytes > ctx->calpa_cap) {
    CUDA_TRY(cudaSetDevice(ctx->device));
    CUDA_TRY(cudaDeviceSynchronize());
    cudaFree(ctx->calpa);
    ctx->calpa = nullptr;
    ctx->calpa_cap = 0;
    CUDA_TRY(cudaMalloc(&ctx->calpa, bytes));
    ctx->calpa_cap = bytes;
  }
  *ptr = ctx->calpa;
  return HDR_OK;
}
hdr_status lpa_launch_mode(hdr_ctx *ctx, int32_t rig_id, const hdr_params *params, const uint16_t *const *raw_dev,
                           int mode, float *aux, double reach, void *out_dev, uint8_t *choice_dev, cudaStream_t st,
                           bool ahead) {
  hdr_status s = common_checks(ctx, rig_id, params, raw_dev, mode == LPA_GRADIENTS ? aux : out_dev);
  if (s) return s;
  if (params->weight_mode != 0)
    return fail(HDR_E_UNSUPPORTED, "the adaptive passes use the inverse-variance weight (weight_mode 0)");
  hdr_params p = *params;
  p.tab_weights = 0;  // the window is searched: offsets or weights differ per pixel
  float2 *conv = nullptr;
  if (ahead) {
    s = conv_buffer(ctx, ctx->rigs[rig_id], &p, &conv);
    if (s) return s;
  }
  LpaLaunch L;
  s = plan(ctx, ctx->rigs[rig_id], &p, raw_dev, L, reach, true, 1, conv);
  if (s) return s;
  if (L.conv) {  // the frame converted once, then the pass
    s = convert_rows(ctx, L, all_rows(L), true, st);
    if (s) return s;
  }
  // the plan picked the FP32-only variant when these parameters cannot trigger the FP64 re-solve
  L.mode = lpa_mode_f32(L.mode) ? lpa_mode_to_f32(mode) : mode;
  L.aux = aux;
  L.out = out_dev;
  L.choice = choice_dev;
  s = launch(L, p.accum, false, st);
  if (s == HDR_OK && L.conv) CUDA_TRY(cudaEventRecord(ctx->conv_ev, st));
  return s;
}
hdr_status lpa_check_params(const hdr_params *p) { return check_params(p); }
hdr_status lpa_take_status(hdr_ctx *ctx) {
  unsigned int word = 0;
  CUDA_TRY(cudaMemcpy(&word, ctx->status, sizeof(word), cudaMemcpyDeviceToHost));
  if (word) CUDA_TRY(cudaMemset(ctx->status, 0, sizeof(word)));
  if (word & LPA_ERR_TIMEOUT) return fail(HDR_E_TIMEOUT, "a bounded device wait ran out (status 0x%x)", word);
  if (word & LPA_ERR_BOUNDS) return fail(HDR_E_INTERNAL, "a window left the staged footprint (status 0x%x)", word);
  return HDR_OK;
}

extern "C" hdr_status hdr_reconstruct_batch(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames,
                                            const hdr_batch_config *cfg_in, void *cuda_stream) {
  return lpa_batch_run(ctx, n_frames, frames, nullptr, cfg_in, (cudaStream_t)cuda_stream);
}

extern "C" hdr_status hdr_tune_batch(hdr_ctx *ctx, int32_t n_frames, const hdr_frame *frames, hdr_batch_config *best,
                                     void *cuda_stream) {
  hdr_status st = check_batch(ctx, n_frames, frames);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  hdr_batch_config win = {16, 0, 1, 0, 1, 1};
  float win_ms = 1e30f;
  // form, tile height, pixels per thread, staging buffers, persistent CTAs per SM and frame order
  const hdr_batch_config cands[] = {{16, 0, 1, 0, 1, 1}, {8, 0, 1, 0, 1, 1}, {16, 0, 1, 0, 2, 1}, {16, 0, 1, 0, 1, 2},
                                    {8, 0, 1, 0, 1, 2},  {16, 0, 0, 0, 1, 1}, {16, 0, 1, 1, 1, 1}, {16, 1, 1, 1, 1, 1},
                                    {16, 2, 1, 1, 1, 1}, {8, 0, 1, 1, 1, 1},  {8, 2, 1, 1, 1, 1},  {8, 4, 1, 1, 1, 1},
                                    {16, 0, 0, 1, 1, 1}};
  for (const hdr_batch_config &c : cands) {
    st = hdr_reconstruct_batch(ctx, n_frames, frames, &c, cuda_stream);  // warm-up (and graph record)
    if (st == HDR_E_UNSUPPORTED) continue;
    if (st) break;
    float ms = 0.f;
    cudaError_t e = cudaEventRecord(e0, stream);
    for (int r = 0; r < 2 && e == cudaSuccess && st == HDR_OK; r++) st = hdr_reconstruct_batch(ctx, n_frames, frames, &c, cuda_stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = fail(HDR_E_CUDA, "timing a batch configuration failed: %s", cudaGetErrorString(e));
      break;
    }
    if (st) break;
    if (ms < win_ms) {
      win_ms = ms;
      win = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st && st != HDR_E_UNSUPPORTED) return st;
  if (win_ms >= 1e30f) return fail(HDR_E_UNSUPPORTED, "no batch configuration fits this device");
  ctx->batch.tuned[batch_kind(ctx, n_frames, frames)] = win;
  if (best) *best = win;
  return HDR_OK;
}

// ------------------------------------------------------------------ reconstruction without allocation
//
// Scratch of hdr_reconstruct_noalloc: the kernel's status word and any per-pixel calibration
// frames live in this fixed array instead of in device memory allocated by a context. Every GPU
// that loads the library holds it until the process exits. In host code its name only stands
// in for the array; the device address comes from cudaGetSymbolAddress, looked up once per
// device with that device current.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HDR_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kScratchHeader = 256;  // bytes before the first frame; the status word is at 0
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[kMaxDevices] = {};
EncodeTiledFn g_noalloc_encode = nullptr;

// One-time set-up for `device` (which must be current): the scratch address and the encoder.
hdr_status noalloc_setup(int device, unsigned char **scratch, EncodeTiledFn *encode) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_encode) {
    cudaDriverEntryPointQueryResult q;
    void *fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return fail(HDR_E_CUDA, "cuTensorMapEncodeTiled not available from the driver");
    g_noalloc_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  if (!g_noalloc_ptr[device]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return fail(HDR_E_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    g_noalloc_ptr[device] = static_cast<unsigned char *>(ptr);
  }
  *scratch = g_noalloc_ptr[device];
  *encode = g_noalloc_encode;
  return HDR_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" hdr_status hdr_reconstruct_noalloc(int device, int32_t n_sensors, const hdr_sensor_desc *sensors,
                                              const hdr_params *params, const uint16_t *const *raw_dev,
                                              void *out_dev, uint8_t *choice_dev, void *cuda_stream) {
  hdr_status st = check_sensors(n_sensors, sensors);
  if (st) return st;
  st = check_params(params);
  if (st) return st;
  if (!raw_dev) return fail(HDR_E_INVALID, "raw pointer array is NULL");
  if (!out_dev && (long long)params->out_w * params->out_h > 0) return fail(HDR_E_INVALID, "output pointer is NULL");
  if (device < 0 || device >= kMaxDevices) return fail(HDR_E_INVALID, "device %d out of range", device);
  // scratch layout: status word, then each sensor's per-pixel frames on 256-byte boundaries
  size_t need = kScratchHeader;
  for (int s = 0; s < n_sensors; s++) {
    const size_t npx = (size_t)sensors[s].width * sensors[s].height;
    if (sensors[s].bias_frame) need += align256(npx * 4);
    if (sensors[s].prnu_frame) need += align256(npx * 4);
    if (sensors[s].read_var_frame) need += align256(npx * 4);
    if (sensors[s].sat_frame) need += align256(npx * 2);
  }
  if (need > (size_t)HDR_NOALLOC_SCRATCH_BYTES)
    return fail(HDR_E_UNSUPPORTED,
                "the per-pixel calibration frames need %zu bytes of scratch; this entry point holds at most %u "
                "(use a context and hdr_set_rig for larger frames)",
                need, (unsigned)HDR_NOALLOC_SCRATCH_BYTES);
  int n_dev = 0;
  CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device >= n_dev) return fail(HDR_E_INVALID, "device %d not present (%d devices)", device, n_dev);
  CUDA_TRY(cudaSetDevice(device));
  unsigned char *scratch = nullptr;
  EncodeTiledFn encode = nullptr;
  st = noalloc_setup(device, &scratch, &encode);
  if (st) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned int *status = reinterpret_cast<unsigned int *>(scratch);
  // the array keeps the previous call's contents: clear the status word, copy this call's frames
  CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned int), stream));
  Rig rig;
  rig.n = n_sensors;
  size_t off = kScratchHeader;
  for (int s = 0; s < n_sensors; s++) {
    RigSensor &rs = rig.s[s];
    rs.d = sensors[s];
    const size_t npx = (size_t)rs.d.width * rs.d.height;
    auto place = [&](const void *src, size_t bytes, void **dst) -> cudaError_t {
      if (!src) return cudaSuccess;
      *dst = scratch + off;
      off += align256(bytes);
      return cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, stream);
    };
    CUDA_TRY(place(rs.d.bias_frame, npx * 4, (void **)&rs.bias));
    CUDA_TRY(place(rs.d.prnu_frame, npx * 4, (void **)&rs.prnu));
    CUDA_TRY(place(rs.d.read_var_frame, npx * 4, (void **)&rs.rvar));
    CUDA_TRY(place(rs.d.sat_frame, npx * 2, (void **)&rs.satf));
  }
  LpaLaunch L;
  st = plan_env(PlanEnv{encode, status, device, nullptr, false}, rig, params, raw_dev, L);
  for (int s = 0; s < n_sensors; s++) rig.s[s] = RigSensor();  // the frames belong to the scratch array
  rig.n = 0;
  if (st) return st;
  L.out = out_dev;
  L.choice = choice_dev;
  L.levels = nullptr;
  st = launch(L, params->accum, false, stream);
  if (st) return st;
  unsigned int word = 0;
  CUDA_TRY(cudaStreamSynchronize(stream));
  CUDA_TRY(cudaMemcpy(&word, status, sizeof(word), cudaMemcpyDeviceToHost));
  if (word & LPA_ERR_TIMEOUT) return fail(HDR_E_TIMEOUT, "a bounded device wait ran out (status 0x%x)", word);
  if (word & LPA_ERR_BOUNDS) return fail(HDR_E_INTERNAL, "a window left the staged footprint (status 0x%x)", word);
  return HDR_OK;
}
