// Launch descriptor shared by the host code and the reconstruction kernels.
// Internal to the CUDA library; not part of the C ABI.
#pragma once
#include <cuda.h>
#include <stdint.h>

#define LPA_MAX_SENSORS 8
#define LPA_MAX_SCALES 8
#define LPA_TILE 16         // output tile width in pixels; the height TH is 8 or 16 (one thread per pixel)
#define LPA_ANCHOR 8        // edge of the output blocks whose sensor positions are anchored in FP64
#define LPA_MARGIN 4        // staging margin in sensor px around every window box
#define LPA_STAGED_TILES 4  // tiles per CTA of the single-frame kernel with two staging buffers

// Device status word bits (read and cleared by hdr_check).
#define LPA_ERR_TIMEOUT 1u  // a bounded mbarrier wait ran out
#define LPA_ERR_BOUNDS 2u   // a window row fell outside the staged footprint

struct alignas(64) LpaSensorK {
  CUtensorMap tmap;         // 2-D tiled map of the raw frame (uint16, dims width x height)
  double G[6];              // output px -> sensor px: T_s^{-1} composed with the output mapping
  float Gf[4];              // linear part of G in FP32 (steps between neighbouring output pixels)
  float A[4];               // linear part of T_s (sensor px -> reference px), row-major
  float hx_unit, hy_unit;   // sensor-space half extent of a reference disc of radius 1
  float inv_gtn;            // 1 / (g t n)
  float gtn2;               // (g t n)^2
  float gain, read_var, black, sat;
  int width, height;
  int box_w, box_h;         // staged footprint in elements; box_w % 8 == 0, box_h even
  float ext_x, ext_y;       // half extent of the window box in sensor px incl. margin (max scale)
  uint32_t off_raw;         // byte offset of the raw box in dynamic shared memory
  uint32_t off_raw2;        // the second staging buffer's raw box (= off_raw with one buffer)
  uint32_t off_planes;      // byte offset of the four colour-phase planes (float2 each)
  int ix_shift, iy_shift;   // tabulated weights: floor of the translation of G (sensor px)
  const float *bias;        // optional per-pixel frames [height][width] (device)
  const float *prnu;
  const float *rvar;
  const uint16_t *satf;
  // Frames converted ahead of the reconstruction (LpaLaunch::conv): the raw frame (pitch in
  // elements) and its staged values in global memory, float2 [4][conv_h][conv_pitch]: colour phase
  // ox + 2 oy, row y >> 1, column x >> 1, (0, 0) outside the frame; tmap then maps these planes.
  const uint16_t *raw;
  float2 *conv;
  int raw_pitch, conv_pitch, conv_h;
};

struct LpaLaunch {
  LpaSensorK s[LPA_MAX_SENSORS];
  int n_sensors;
  int order;
  int n_scales;
  float sigma[LPA_MAX_SCALES];   // R/B scales in reference px
  float green_ratio;
  float trunc_k;
  float ici_gamma;
  float min_pivot;
  float cond_fallback;           // <= 0: never
  float taper;                   // exp(-k^2 / 2)
  int out_w, out_h;
  int tiles_x, tiles_y;
  int out_half;                  // 0 float32, 1 float16
  void *out;
  uint8_t *choice;
  float *levels;
  unsigned int *status;
  uint32_t tx_bytes;             // bytes landed by the bulk tensor copies of one tile
  uint32_t smem_bytes;
  uint32_t off_pos;              // byte offset of each thread's pixel position in each sensor
                                 // (int4 {ix, iy, fx bits, fy bits}, [n_sensors][threads])
  int tile_h;                    // tile height (rows) the plan was made for
  int px;                        // output pixels per thread (0 or 1: one; 2: two, 16-row tiles)
  int tile0;                     // single-frame grid: CTA b reconstructs tile tile0 + b
  int tile_count;                // tiles of the launch from tile0 on; 0 = every tile from tile0 on
  // Staging buffers per CTA of the single-frame kernel: 1 = one tile per CTA; 2 = each CTA takes
  // LPA_STAGED_TILES tiles (tile0 + b + k grid) and copies the next tile's raw boxes into the
  // second buffer while it reconstructs the current one.
  int stages;
  // 1: the staged values come converted from global memory (LpaSensorK::conv, one 3-D bulk copy
  // of the four colour-phase planes per sensor) and the kernel does no conversion; 0: it copies
  // the raw footprints and converts them itself.
  int conv;
  // Tabulated window weights (NULL = the window is searched and evaluated per pixel), in passes of
  // tab_nsp scales as the kernel walks them (lpa_scale_passes). Entry
  // ((((s * 2 + pu) * 2 + pv) * 4 + phase) * n_pass + pass) of tab_hdr, two int4, describes the
  // cells of sensor s, output parity (pu, pv) and colour phase (ox + 2 oy) inside the window of the
  // pass's largest scale, sorted by distance: {first cell, number of cells, qx bounds, qy bounds}
  // and {n_0 .. n_3}, the cells of slot q's scale being the first n_q (0 for the slots a short
  // first pass leaves empty). A cell is two float4: {dx, dy, bits of (qy << 16) | (qx & 0xffff),
  // 0}, the offset of the sample from the pixel's point in reference px and its lattice offset from
  // the pixel's even lattice cell, and {K_0 .. K_3}, its window weight at the scale of each slot.
  const int4 *tab_hdr;           // bounds packed as (min & 0xffff) | (max << 16)
  const float4 *tab_cells;
  int tab_nsp;                   // scales per pass the table was built for
  // Kernel mode (LPA_SEARCHED .. LPA_TABULATED_F32 below). Adaptive reconstruction (Sections 5.4-5.5):
  // LPA_STEERED reads the steering matrix of each output pixel from aux ([out_h][out_w][3]: C11,
  // C12, C22); LPA_GRADIENTS writes the gradient of the green fit to aux ([out_h][out_w][2]).
  // LPA_LITERAL: the searched window with the noise weight printed in Eq. 6 (K / s, not K / s2).
  int mode;
  float *aux;
};

// LPA_SEARCHED_F32, LPA_STEERED_F32, LPA_TABULATED_F32: the searched, steered or tabulated window
// with every fit solved in FP32 only, for parameters under which the FP64 re-solve can never
// trigger ((min_pivot - 1e-4) * cond_fallback >= 2: a usable fit's equilibrated pivots lie in
// (min_pivot, 1], so their spread stays below cond_fallback).
enum {
  LPA_SEARCHED = 0,
  LPA_TABULATED = 1,
  LPA_STEERED = 2,
  LPA_GRADIENTS = 3,
  LPA_LITERAL = 4,
  LPA_SEARCHED_F32 = 5,
  LPA_STEERED_F32 = 6,
  LPA_TABULATED_F32 = 7
};
__host__ __device__ constexpr bool lpa_mode_steered(int mode) { return mode == LPA_STEERED || mode == LPA_STEERED_F32; }
__host__ __device__ constexpr bool lpa_mode_tab(int mode) { return mode == LPA_TABULATED || mode == LPA_TABULATED_F32; }
__host__ __device__ constexpr bool lpa_mode_f32(int mode) {
  return mode == LPA_SEARCHED_F32 || mode == LPA_STEERED_F32 || mode == LPA_TABULATED_F32;
}
// the FP32-only variant of a mode, where it has one
__host__ __device__ constexpr int lpa_mode_to_f32(int mode) {
  return mode == LPA_SEARCHED    ? LPA_SEARCHED_F32
         : mode == LPA_STEERED   ? LPA_STEERED_F32
         : mode == LPA_TABULATED ? LPA_TABULATED_F32
                                 : mode;
}

// Scales per walk of the window cells: the searched, steered and tabulated windows with plain FP32
// sums feed up to four nested scales from one walk at orders 0 and 1, two at order 2 when the FP64
// re-solve is compiled out (their sums stay in registers); the other variants walk once per scale.
#ifndef LPA_MULTI_SCALE
#define LPA_MULTI_SCALE 2      // order 2
#endif
#ifndef LPA_MULTI_SCALE_LOW
#define LPA_MULTI_SCALE_LOW 4  // order 1
#endif
#ifndef LPA_MULTI_SCALE_M0
#define LPA_MULTI_SCALE_M0 4   // order 0
#endif
__host__ __device__ constexpr int lpa_scales_per_walk(int order, bool comp, int mode) {
  return comp ? 1
         : lpa_mode_f32(mode)
             ? (order == 2 ? LPA_MULTI_SCALE : order == 1 ? LPA_MULTI_SCALE_LOW : LPA_MULTI_SCALE_M0)
         : (mode == LPA_SEARCHED || mode == LPA_STEERED || mode == LPA_TABULATED)
             ? (order == 2 ? 1 : order == 1 ? LPA_MULTI_SCALE_LOW : LPA_MULTI_SCALE_M0)
             : 1;
}
// The passes over J scales in walks of nsp: the first pass takes what the later full passes leave
// (the small scales), so that the largest scales share the longest walk. Pass k covers scales
// j0 .. j0 + nj - 1 in slots lead .. nsp - 1 (lead = nsp - nj).
__host__ __device__ constexpr int lpa_n_passes(int J, int nsp) { return (J + nsp - 1) / nsp; }
__host__ __device__ constexpr int lpa_first_pass_scales(int J, int nsp) { return J - nsp * (lpa_n_passes(J, nsp) - 1); }

// Rows [r0[s], r1[s]) of sensor s to convert (lpa_convert).
struct LpaRows {
  int r0[LPA_MAX_SENSORS], r1[LPA_MAX_SENSORS];
};

// The two-buffer single-frame kernel is built for plain sums with the searched or tabulated window.
__host__ __device__ constexpr bool lpa_stages2_built(int mode, bool comp) {
  return !comp && (mode == LPA_SEARCHED || mode == LPA_SEARCHED_F32 || lpa_mode_tab(mode));
}
// CTAs of a single-frame launch over `tiles` tiles: one per tile, or one per LPA_STAGED_TILES tiles
// with two staging buffers.
__host__ __device__ constexpr int lpa_grid_ctas(int tiles, int stages) {
  return stages == 2 ? (tiles + LPA_STAGED_TILES - 1) / LPA_STAGED_TILES : tiles;
}

// Several frames in one graph launch: the tile list is grouped by polynomial order and each
// order's persistent kernel takes tiles from its own segment. The tile list, the segment bounds
// and the counters live in device memory so that a recorded graph stays valid when the frames
// change.
struct LpaBatch {
  const LpaLaunch *frames;       // [n_frames] (device)
  const int2 *tiles;             // [n_tiles] (frame index, tile index within the frame) (device)
  const int *bounds;             // [4]: the tiles of order M are [bounds[M], bounds[M+1]) (device)
  unsigned int *counters;        // [3] tile counters, zero at launch (device)
  uint32_t smem_bytes;           // max over the frames of the kernel's order
};
