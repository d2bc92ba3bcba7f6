// Fused multi-sensor HDR reconstruction kernel for sm_103a.
//
// One CTA reconstructs one 16x16 tile of output pixels, one thread per pixel.
//   1. Stage: the raw uint16 footprint of the tile in every sensor is fetched
//      by one bulk tensor copy per sensor (cp.async.bulk.tensor, completion on
//      an mbarrier with a bounded wait), then converted once per sample to
//      radiant power and inverse variance (Section 6, Eqs. 18 and 20;
//      saturated and out-of-sensor samples get inverse variance 0 = excluded)
//      into four colour-phase planes of float2 in shared memory.
//   2. Fit: per channel and window scale the thread walks the samples of its
//      window in sensor space (the bounding box of the pre-image of the
//      reference-space disc), computes the reference-frame offset d = X - P_j
//      from small sensor-space offsets (Section 4.2), and accumulates the
//      distinct moments sum w d^a d^b (a+b <= 2M), sum w f phi and
//      sum w K d^a d^b in registers (w = K / s2, K the tapered Gaussian window
//      of Eq. 8). The normal equations of Eq. 6 are then equilibrated and
//      factored (LDL^T, FP32; FP64 when the condition estimate is large),
//      giving C_0 and Var C_0.
//   3. Scale choice: intersection of confidence intervals over the scales in
//      ascending order, with a warp-wide early exit once every lane's
//      intersection is empty; order fallback at the largest scale; NaN when
//      nothing is usable.
// Warps hold pixels of one output parity class (16x8 pixels, stride 2), so on
// rigs close to a translation at 1x output every lane sees the same sample
// layout and the window loops run without divergence.
#pragma once
#include <cuda_fp16.h>
#include <stdint.h>

#include "lpa_launch.h"
#include "lpa_ptx.cuh"

namespace lpa {

#define LPA_FULL 0xffffffffu

__host__ __device__ constexpr int mono_index(int a, int b) { return (a + b) * (a + b + 1) / 2 + b; }
__host__ __device__ constexpr int n_unknowns(int order) { return order == 0 ? 1 : (order == 1 ? 3 : 6); }
__host__ __device__ constexpr int n_monos(int order) { return order == 0 ? 1 : (order == 1 ? 6 : 15); }
// exponents of the basis [1, dx, dy, dx^2, dx dy, dy^2] (Section 5.1, tril order)
__host__ __device__ constexpr int ex(int m) { return (m == 1 || m == 4) ? 1 : (m == 3 ? 2 : 0); }
__host__ __device__ constexpr int ey(int m) { return (m == 2 || m == 4) ? 1 : (m == 5 ? 2 : 0); }

// ---------------------------------------------------------------- moments

// Error-free sum of two floats (Knuth's two-sum) and product (FMA residual).
__device__ __forceinline__ void comp_add(float &hi, float &lo, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);
  float s = __fadd_rn(hi, p);
  float bb = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

template <int ORDER, bool COMP>
struct Moments {
  static constexpr int NA = n_monos(ORDER);     // sum w d^a d^b, a+b <= 2M
  static constexpr int NB = n_unknowns(ORDER);  // sum w f phi
  float a[NA], b[NB], k[NA];                    // k: sum w K d^a d^b (variance of C_0)
  float al[COMP ? NA : 1], bl[COMP ? NB : 1], kl[COMP ? NA : 1];
  float cnt;

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NA; i++) a[i] = k[i] = 0.f;
#pragma unroll
    for (int i = 0; i < NB; i++) b[i] = 0.f;
    if (COMP) {
#pragma unroll
      for (int i = 0; i < NA; i++) al[i] = kl[i] = 0.f;
#pragma unroll
      for (int i = 0; i < NB; i++) bl[i] = 0.f;
    }
    cnt = 0.f;
  }

  __device__ __forceinline__ void add2(float2 D, float2 D2, float w, float wf, float wk) { add(D.x, D.y, w, wf, wk); }
  // order 0: the three sums and the sample count (`one` is 1 for a window sample, else 0)
  __device__ __forceinline__ void add0(float w, float wf, float wk, float one) {
    if (COMP) {
      comp_add(a[0], al[0], w, 1.f);
      comp_add(k[0], kl[0], wk, 1.f);
      comp_add(b[0], bl[0], wf, 1.f);
    } else {
      a[0] += w;
      k[0] += wk;
      b[0] += wf;
    }
    cnt += one;
  }

  __device__ __forceinline__ void add(float dx, float dy, float w, float wf, float wk) {
    float m[15];
    m[0] = 1.f;
    if (NA > 1) {
      m[1] = dx;
      m[2] = dy;
      m[3] = dx * dx;
      m[4] = dx * dy;
      m[5] = dy * dy;
    }
    if (NA > 6) {
      m[6] = m[3] * dx;
      m[7] = m[3] * dy;
      m[8] = m[4] * dy;
      m[9] = m[5] * dy;
      m[10] = m[3] * m[3];
      m[11] = m[3] * m[4];
      m[12] = m[3] * m[5];
      m[13] = m[4] * m[5];
      m[14] = m[5] * m[5];
    }
    if (COMP) {
#pragma unroll
      for (int i = 0; i < NA; i++) {
        comp_add(a[i], al[i], w, m[i]);
        comp_add(k[i], kl[i], wk, m[i]);
      }
#pragma unroll
      for (int i = 0; i < NB; i++) comp_add(b[i], bl[i], wf, m[i]);
    } else {
      a[0] += w;
      k[0] += wk;
      b[0] += wf;
#pragma unroll
      for (int i = 1; i < NA; i++) {
        a[i] = fmaf(w, m[i], a[i]);
        k[i] = fmaf(wk, m[i], k[i]);
      }
#pragma unroll
      for (int i = 1; i < NB; i++) b[i] = fmaf(wf, m[i], b[i]);
    }
    cnt += 1.f;
  }

  __device__ __forceinline__ float count() const { return cnt; }
  template <typename T>
  __device__ __forceinline__ T A(int i) const { return COMP ? (T)a[i] + (T)al[i] : (T)a[i]; }
  template <typename T>
  __device__ __forceinline__ T B(int i) const { return COMP ? (T)b[i] + (T)bl[i] : (T)b[i]; }
  template <typename T>
  __device__ __forceinline__ T Kv(int i) const { return COMP ? (T)k[i] + (T)kl[i] : (T)k[i]; }
};

#ifndef LPA_PACKED_MOMENTS
#define LPA_PACKED_MOMENTS 1
#endif



// The same plain FP32 moments with the Gram and variance sums of each monomial held as one pair
// (sum w m, sum w K m): one paired FMA (fma.rn.f32x2, weights (w, w K), the monomial in both
// halves) advances both, rounding each half as the scalar FMA would. The monomials of degree 3
// and 4 are formed two at a time by paired products (x^3, y^3), (x^2 y, x y^2), ..., so they
// round in another order than Moments<ORDER, false> forms them (a few units in the last place);
// Blackwell issues two FP32 operations per paired instruction, so fewer instructions are issued.
template <int ORDER>
struct MomentsPacked {
  static constexpr int NA = n_monos(ORDER);
  static constexpr int NB = n_unknowns(ORDER);
  float2 ak[NA];  // (sum w m_i, sum w K m_i)
  // the right-hand side sum w f m_i in pairs of monomials held in register pairs:
  // (sum w f, count), (m_1, m_2) = D, (m_3, m_5) = D2; m_4 alone
  float2 b0n, b12, b35;
  float b4;

  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < NA; i++) ak[i] = make_float2(0.f, 0.f);
    b0n = b12 = b35 = make_float2(0.f, 0.f);
    b4 = 0.f;
  }
  __device__ __forceinline__ float count() const { return b0n.y; }

  // the monomials of one sample at offset D = (dx, dy) with squares D2 = (dx^2, dy^2): degree 3
  // and 4 come two at a time from paired products
  static __device__ __forceinline__ void monomials(float2 D, float2 D2, float (&s)[15]) {
    s[1] = D.x;
    s[2] = D.y;
    s[3] = D2.x;
    s[4] = D.x * D.y;
    s[5] = D2.y;
    if (NA > 6) {
      const float2 SW = make_float2(D.y, D.x);
      const float2 P3 = __fmul2_rn(D2, D);    // (x^3, y^3)
      const float2 P21 = __fmul2_rn(D2, SW);  // (x^2 y, x y^2)
      const float2 P4 = __fmul2_rn(D2, D2);   // (x^4, y^4)
      const float2 P31 = __fmul2_rn(P3, SW);  // (x^3 y, x y^3)
      s[6] = P3.x;
      s[7] = P21.x;
      s[8] = P21.y;
      s[9] = P3.y;
      s[10] = P4.x;
      s[11] = P31.x;
      s[12] = s[4] * s[4];
      s[13] = P31.y;
      s[14] = P4.y;
    }
  }
  // one sample with its monomials s, weight w = K / s2, w f and w K
  __device__ __forceinline__ void adds(const float (&s)[15], float2 D, float2 D2, float w, float wf, float wk) {
    const float2 W = make_float2(w, wk);
    ak[0] = __fadd2_rn(ak[0], W);
#pragma unroll
    for (int i = 1; i < NA; i++) ak[i] = __ffma2_rn(W, make_float2(s[i], s[i]), ak[i]);
    const float2 F = make_float2(wf, wf);
    b0n = __fadd2_rn(b0n, make_float2(wf, 1.f));
    b12 = __ffma2_rn(F, D, b12);
    if (NB > 3) {
      b35 = __ffma2_rn(F, D2, b35);
      b4 = fmaf(wf, s[4], b4);
    }
  }
  __device__ __forceinline__ void add2(float2 D, float2 D2, float w, float wf, float wk) {
    float s[15];
    monomials(D, D2, s);
    adds(s, D, D2, w, wf, wk);
  }

  template <typename T>
  __device__ __forceinline__ T A(int i) const { return (T)ak[i].x; }
  template <typename T>
  __device__ __forceinline__ T B(int i) const {
    return (T)(i == 0 ? b0n.x : i == 1 ? b12.x : i == 2 ? b12.y : i == 3 ? b35.x : i == 4 ? b4 : b35.y);
  }
  template <typename T>
  __device__ __forceinline__ T Kv(int i) const { return (T)ak[i].y; }
};

// The accumulator a kernel uses: paired for plain FP32 sums of order >= 1.
template <int ORDER, bool COMP, bool PACKED = (LPA_PACKED_MOMENTS != 0) && !COMP && ORDER >= 1>
struct MomentsSel {
  using type = Moments<ORDER, COMP>;
};
template <int ORDER>
struct MomentsSel<ORDER, false, true> {
  using type = MomentsPacked<ORDER>;
};

// ---------------------------------------------------------------- solve

struct FitOut {
  float c0, var;
  float dmin, dmax;  // extreme pivots of the equilibrated LDL^T
  bool valid;
  float c1, c2;      // first-order coefficients c = A^{-1} b (only when asked for)
};

__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.f, x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }

// packed lower-triangle index (i >= j)
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Eq. 6 for the first P basis functions: the normal matrix A = Phi^T W Phi is factored LDL^T as
// it stands. Usability and the condition estimate are judged on the pivots of the
// Jacobi-equilibrated matrix D A D (D = diag(A)^{-1/2}), which are d_j / A_jj: equilibration
// changes L but scales each pivot by 1 / A_jj. l = A^{-1} e_0, C_0 = l^T b,
// Var C_0 = l^T (Phi^T W S W Phi) l with S the sample variances.
template <typename T, int P, class MOM, bool COEF = false>
__device__ __forceinline__ FitOut solve(const MOM &m, float min_pivot) {
  FitOut r;
  T a[P * (P + 1) / 2];  // lower triangle, overwritten by L (below the diagonal) and D
#pragma unroll
  for (int i = 0; i < P; i++)
#pragma unroll
    for (int j = 0; j <= i; j++) a[tri(i, j)] = m.template A<T>(mono_index(ex(i) + ex(j), ey(i) + ey(j)));
  T rdiag[P];
  bool pos = true;
#pragma unroll
  for (int i = 0; i < P; i++) {
    pos = pos && (a[tri(i, i)] > T(0));
    rdiag[i] = a[tri(i, i)] > T(0) ? rcp_t(a[tri(i, i)]) : T(0);
  }
  // triangular loops are written with fixed trip counts and guards so that they unroll fully;
  // u holds L_iq d_q (the column before its division by the pivot), so that each update term
  // is one FMA
  T dinv[P], u[P * (P + 1) / 2];
  T dmin = T(1e30), dmax = T(0);
#pragma unroll
  for (int j = 0; j < P; j++) {
    T dj = a[tri(j, j)];
#pragma unroll
    for (int q = 0; q < P; q++)
      if (q < j) dj -= a[tri(j, q)] * u[tri(j, q)];
    a[tri(j, j)] = dj;
    const T de = dj * rdiag[j];  // pivot of the equilibrated matrix
    dmin = de < dmin ? de : dmin;
    dmax = de > dmax ? de : dmax;
    dinv[j] = dj > T(0) ? rcp_t(dj) : T(0);
#pragma unroll
    for (int i = 0; i < P; i++) {
      if (i > j) {
        T t = a[tri(i, j)];
#pragma unroll
        for (int q = 0; q < P; q++)
          if (q < j) t -= a[tri(i, q)] * u[tri(j, q)];
        u[tri(i, j)] = t;
        a[tri(i, j)] = t * dinv[j];
      }
    }
  }
  r.dmin = (float)dmin;
  r.dmax = (float)dmax;
  r.valid = pos && (m.count() >= (float)P) && (dmin > (T)min_pivot);
  // l = A^{-1} e_0: forward (unit L), diagonal, backward (L^T)
  T x[P];
#pragma unroll
  for (int i = 0; i < P; i++) {
    T t = (i == 0) ? T(1) : T(0);
#pragma unroll
    for (int q = 0; q < P; q++)
      if (q < i) t -= a[tri(i, q)] * x[q];
    x[i] = t;
  }
#pragma unroll
  for (int i = 0; i < P; i++) x[i] *= dinv[i];
#pragma unroll
  for (int ii = 0; ii < P; ii++) {
    const int i = P - 1 - ii;
    T t = x[i];
#pragma unroll
    for (int q = 0; q < P; q++)
      if (q > i) t -= a[tri(q, i)] * x[q];
    x[i] = t;
  }
  // the quadratic form over the symmetric K: diagonal terms once, the others doubled
  T c0 = T(0), var = T(0);
#pragma unroll
  for (int i = 0; i < P; i++) {
    c0 += x[i] * m.template B<T>(i);
    T row = T(0);
#pragma unroll
    for (int j = 0; j < P; j++)
      if (j > i) row += x[j] * m.template Kv<T>(mono_index(ex(i) + ex(j), ey(i) + ey(j)));
    row = T(2) * row + x[i] * m.template Kv<T>(mono_index(2 * ex(i), 2 * ey(i)));
    var += x[i] * row;
  }
  r.c0 = (float)c0;
  r.var = (float)var;
  if constexpr (COEF && P >= 3) {
    // c = A^{-1} b by the same factors: forward (unit L), diagonal, backward (L^T)
    T y[P];
#pragma unroll
    for (int i = 0; i < P; i++) {
      T t = m.template B<T>(i);
#pragma unroll
      for (int q = 0; q < P; q++)
        if (q < i) t -= a[tri(i, q)] * y[q];
      y[i] = t;
    }
#pragma unroll
    for (int i = 0; i < P; i++) y[i] *= dinv[i];
#pragma unroll
    for (int ii = 0; ii < P; ii++) {
      const int i = P - 1 - ii;
      T t = y[i];
#pragma unroll
      for (int q = 0; q < P; q++)
        if (q > i) t -= a[tri(q, i)] * y[q];
      y[i] = t;
    }
    r.c1 = (float)y[1];
    r.c2 = (float)y[2];
  }
  return r;
}

// Bound on the absolute error of an FP32 pivot of the equilibrated normal matrix
// (unit diagonal): at most 6 x 6 terms accumulated over a few hundred samples at
// 2^-24 relative rounding each stays well below this.
#define LPA_PIVOT_FP32_ERR 1e-4f

// FP32 solve; the same solve in FP64 when the FP32 pivots span more than
// cond_fallback and the fit could still pass min_pivot in exact arithmetic.
template <int P, class MOM, bool COEF = false, bool F64 = true>
__device__ __forceinline__ FitOut solve_with_fallback(const MOM &m, float min_pivot, float cond_fallback) {
  FitOut r = solve<float, P, MOM, COEF>(m, min_pivot);
  if constexpr (!F64) return r;
  bool redo = cond_fallback > 0.f && m.count() >= (float)P && !(r.dmin * cond_fallback >= r.dmax) &&
              r.dmin > min_pivot - LPA_PIVOT_FP32_ERR;
  if (redo) r = solve<double, P, MOM, COEF>(m, min_pivot);
  return r;
}

// Lower-order fits at the largest scale reuse the leading block of the moments.
template <int ORDER, int I, bool F64, class MOM>
__device__ __forceinline__ FitOut fallback_fit(const MOM &m, float min_pivot, float cond_fallback) {
  if constexpr (ORDER - 1 - I == 1) return solve_with_fallback<3, MOM, false, F64>(m, min_pivot, cond_fallback);
  else return solve_with_fallback<1, MOM, false, F64>(m, min_pivot, cond_fallback);
}

// ---------------------------------------------------------------- scale choice

struct Ici {
  float lo, hi, val;
  int choice;
  bool done;
  __device__ __forceinline__ void reset(bool active) {
    lo = -INFINITY;
    hi = INFINITY;
    val = __int_as_float(0x7fffffff);
    choice = 255;
    done = !active;
  }
  // running intersection of C_0 +- gamma sqrt(Var C_0) over usable scales in ascending order
  __device__ __forceinline__ void step(const FitOut &f, int level, float gamma) {
    if (done || !f.valid) return;
    float h = gamma * sqrtf(fmaxf(f.var, 0.f));
    float nlo = fmaxf(lo, f.c0 - h), nhi = fminf(hi, f.c0 + h);
    if (nlo > nhi) {
      done = true;
      return;
    }
    lo = nlo;
    hi = nhi;
    val = f.c0;
    choice = level;
  }
};

// ---------------------------------------------------------------- kernel

#ifndef LPA_M0_CTAS_256
#define LPA_M0_CTAS_256 4      // resident 256-thread CTAs per SM the order-0 kernel is built for
#endif
template <int ORDER, bool COMP, int MODE>
struct MultiScale {
  static constexpr int value = lpa_scales_per_walk(ORDER, COMP, MODE);
};

// sensor-space positions are clamped to +-LPA_FAR px (far outside any sensor) before integer conversion
#define LPA_FAR 1.0e7

struct Anchor {
  int ix, iy;
  float fx, fy;
};

// Staged sample layout: (f, 1/s2) (1/s for the printed weight); 1/s2 = 0 excludes the sample.
__device__ __forceinline__ float2 stage_pair(float f, float iv) { return make_float2(f, iv); }
__device__ __forceinline__ bool sample_ok(float2 fv) { return fv.y > 0.f; }
// The staged value of raw sample y at sensor pixel (X, Y), inside the frame: Eq. 18 and the inverse
// of Eq. 20 (its square root for the printed weight K / s); (0, 0) when saturated. `scalar`: the
// sensor has no per-pixel calibration frames.
template <bool LIT>
__device__ __forceinline__ float2 convert_sample(const LpaSensorK &Sk, bool scalar, int X, int Y, float y) {
  float f = 0.f, iv = 0.f;
  if (scalar) {
    if (y < Sk.sat) {
      const float e0 = y - Sk.black;
      f = e0 * Sk.inv_gtn;
      iv = __fdividef(Sk.gtn2, fmaf(Sk.gain, fmaxf(e0, 0.f), Sk.read_var));
      if (LIT) iv = sqrtf(iv);
    }
  } else {
    const long px = (long)Y * Sk.width + X;
    const float b = Sk.bias ? Sk.bias[px] : Sk.black;
    const float rv = Sk.rvar ? Sk.rvar[px] : Sk.read_var;
    const float sat = Sk.satf ? (float)Sk.satf[px] : Sk.sat;
    if (y < sat) {
      const float a = Sk.prnu ? Sk.prnu[px] : 1.f;
      const float e0 = y - b;
      f = __fdividef(e0 * Sk.inv_gtn, a);
      iv = __fdividef(Sk.gtn2 * a * a, fmaf(Sk.gain, fmaxf(e0, 0.f), rv));
      if (LIT) iv = sqrtf(iv);
    }
  }
  return stage_pair(f, iv);
}

// (w, w f) of a staged sample for window value K: w = K / s2
__device__ __forceinline__ float2 weights(float K, float2 fv) {
  const float w = K * fv.y;
  return make_float2(w, w * fv.x);
}

// One window cell: offset D from the pixel's point, disc test, Eq. 8 weight times inverse
// variance, moment update.
template <int ORDER, int MODE, class MOM>
__device__ __forceinline__ void window_cell(MOM &m, float2 D, float2 fv, float R2, float cexp, float taper,
                                            float4 Q) {
  constexpr bool STEER = lpa_mode_steered(MODE);
  // the variance sums take w^2 s2 = K w for the inverse-variance weight; with the printed weight
  // K / s (fv.y = 1 / s) it is K^2
  constexpr bool LIT = MODE == LPA_LITERAL;
  const float2 D2 = __fmul2_rn(D, D);
  // |d|^2, or d^T C d for the steered window (Section 5.4)
  const float r2 = STEER ? fmaf(Q.x, D2.x, fmaf(Q.z, D2.y, 2.f * Q.y * (D.x * D.y))) : D2.x + D2.y;
  const bool in = r2 < R2 && sample_ok(fv);
  if constexpr (ORDER == 0) {
    // four sums: cheaper to add exact zeros for cells outside the window than to branch
    const float K = ex2_approx(r2 * cexp) - taper;  // Eq. 8, truncated and tapered
    const float2 W = weights(in ? K : 0.f, fv);     // window x inverse variance, times f
    m.add0(W.x, W.y, (LIT ? (in ? K : 0.f) : W.x) * K, in ? 1.f : 0.f);
  } else if (in) {
    const float K = ex2_approx(r2 * cexp) - taper;
    const float2 W = weights(K, fv);
    m.add2(D, D2, W.x, W.y, (LIT ? K : W.x) * K);
  }
}

// Several window scales in one walk (the windows of one channel are nested discs): the cell's
// offset, its disc test against the largest scale and its monomials are computed once, then each
// scale whose disc holds the sample adds it with its own Eq. 8 weight. Slot q of the scale arrays
// belongs to the q-th scale of the pass; R2[q] < 0 marks an unused slot.

template <int ORDER, int NSP, int MODE, class MOM>
__device__ __forceinline__ void window_cell_ms(MOM (&m)[NSP], float2 D, float2 fv, const float (&R2)[NSP],
                                               const float (&cexp)[NSP], float taper, float4 Q) {
  constexpr bool STEER = lpa_mode_steered(MODE);
  constexpr bool LIT = MODE == LPA_LITERAL;
  const float2 D2 = __fmul2_rn(D, D);
  const float r2 = STEER ? fmaf(Q.x, D2.x, fmaf(Q.z, D2.y, 2.f * Q.y * (D.x * D.y))) : D2.x + D2.y;
  if (!(r2 < R2[NSP - 1] && sample_ok(fv))) return;
  float sm[15];
  if constexpr (ORDER > 0) MOM::monomials(D, D2, sm);
  // two scales per walk (order 2): both window values first, in one paired multiply and add (the
  // same roundings as one at a time), so that their ex2 latencies overlap (-1 %; with four scales
  // per walk the values of scales that miss the sample cost more than that)
  float Kq[NSP];
  if constexpr (NSP == 2) {
    const float2 A = __fmul2_rn(make_float2(r2, r2), make_float2(cexp[0], cexp[1]));
    const float2 E = __fadd2_rn(make_float2(ex2_approx(A.x), ex2_approx(A.y)), make_float2(-taper, -taper));
    Kq[0] = E.x;
    Kq[1] = E.y;
  }
  // largest scale first; the windows are nested, so the first one that misses ends the loop
  // (a loop with an exit, not a chain of tests: no reconvergence point per scale)
#pragma unroll
  for (int q = NSP - 1; q >= 0; q--) {
    if (!(r2 < R2[q])) break;
    const float K = NSP == 2 ? Kq[q] : ex2_approx(r2 * cexp[q]) - taper;
    const float2 W = weights(K, fv);
    if constexpr (ORDER == 0) m[q].add0(W.x, W.y, (LIT ? K : W.x) * K, 1.f);
    else m[q].adds(sm, D, D2, W.x, W.y, (LIT ? K : W.x) * K);
  }
}

// Walk the window cells of channel c in sensor S for one pixel (sample cell and fraction `pos`):
// the cells of the bounding box of the pre-image of the window of radius R (or of the steered
// window d^T Q d < R^2), row by row inside the staged box. body(D, fv) receives each cell's offset
// D = X - P_j in reference px and its staged (f, 1/s2). The rows run UNROLL cells at a time.
template <int MODE, int UNROLL, class Body>
__device__ __forceinline__ void walk_sensor(const LpaSensorK &S, int4 pos, int c, float R, int x0, int y0,
                                            const unsigned char *smem, bool active, unsigned *status, float4 Q,
                                            Body &&body) {
  // the pixel's point in sensor s: sample cell (ix, iy) and fraction (fx, fy) in [0, 1)
  const int ix = pos.x, iy = pos.y;
  const float fx = __int_as_float(pos.z), fy = __int_as_float(pos.w);
  const int PW = S.box_w >> 1, PH = S.box_h >> 1;
  const float2 *planes = reinterpret_cast<const float2 *>(smem + S.off_planes);
  const float a00 = S.A[0], a01 = S.A[1], a10 = S.A[2], a11 = S.A[3];
  constexpr bool STEER = lpa_mode_steered(MODE);
  float hx, hy;
  if constexpr (STEER) {
    // sensor-space bounding box of the support D^T B D < R^2, B = A^T C A (d = A D)
    const float t00 = fmaf(Q.x, a00, Q.y * a10), t01 = fmaf(Q.x, a01, Q.y * a11);
    const float t10 = fmaf(Q.y, a00, Q.z * a10), t11 = fmaf(Q.y, a01, Q.z * a11);
    const float bxx = fmaf(a00, t00, a10 * t10), bxy = fmaf(a00, t01, a10 * t11), byy = fmaf(a01, t01, a11 * t11);
    const float rdet = 1.f / fmaf(bxx, byy, -bxy * bxy);
    // at most the staged box: a matrix below the planned eigenvalue bound (or not positive
    // definite) cannot make the traversal long; cells outside the box are reported as usual
    hx = fminf(R * sqrtf(byy * rdet) + 1e-3f, (float)S.box_w);
    hy = fminf(R * sqrtf(bxx * rdet) + 1e-3f, (float)S.box_h);
  } else {
    hx = R * S.hx_unit + 1e-3f;
    hy = R * S.hy_unit + 1e-3f;
  }
  const float sx = 2.f * a00, sy = 2.f * a10;
  // colour phases of channel c: R (0,0); G (1,0) and (0,1); B (1,1)
  const int nsub = (c == 1) ? 2 : 1;
#pragma unroll 1
  for (int sub = 0; sub < nsub; sub++) {
    const int ox = (c == 0) ? 0 : (c == 2 ? 1 : 1 - sub);
    const int oy = (c == 0) ? 0 : (c == 2 ? 1 : sub);
    const int bx = ix - ox, by = iy - oy;
    const int bxe = bx - (bx & 1), bye = by - (by & 1);
    const float rx = (float)(bx - bxe) + fx;  // q_x - (ox + bxe), in [0, 2)
    const float ry = (float)(by - bye) + fy;
    const int ilo = (int)ceilf((rx - hx) * 0.5f), ihi = (int)floorf((rx + hx) * 0.5f);
    const int jlo = (int)ceilf((ry - hy) * 0.5f), jhi = (int)floorf((ry + hy) * 0.5f);
    const int ni = active ? max(ihi - ilo + 1, 0) : 0;
    const int nj = active ? max(jhi - jlo + 1, 0) : 0;
    const int NI = __reduce_max_sync(LPA_FULL, ni);
    const int NJ = __reduce_max_sync(LPA_FULL, nj);
    if (NI == 0 || NJ == 0) continue;
    const int pc0 = ((bxe - x0) >> 1) + ilo;
    const int pr0 = ((bye - y0) >> 1) + jlo;
    // isotropic windows: every lane walks the warp's longest row (the staged box leaves room for
    // it). Steered windows differ in size and shape within a warp: each lane walks its own rows.
    const int nw = STEER ? ni : NI;
    const bool colok = pc0 >= 0 && pc0 + nw <= PW;
    const float2 *pl = planes + (ox + 2 * oy) * (PH * PW);
    const float Dx0 = 2.f * (float)ilo - rx;
    // a row of the lane's own window outside the staged box is an error (the footprint is planned
    // to hold every window); only the rows inside the box are walked
    if (active && nj > 0 && !(colok && pr0 >= 0 && pr0 + nj <= PH)) atomicOr(status, LPA_ERR_BOUNDS);
    const int rbeg = colok ? max(0, -pr0) : NJ;
    const int rend = min(STEER ? nj : NJ, PH - pr0);
    const float2 *rowp = pl + (pr0 + rbeg) * PW + pc0;
    // offset of the first cell of the first row; each row adds A (0, 2), each cell A (2, 0)
    const float Dy0 = 2.f * (float)(jlo + rbeg) - ry;
    const float2 DR0 = make_float2(fmaf(a00, Dx0, a01 * Dy0), fmaf(a10, Dx0, a11 * Dy0));
    const float2 T2 = make_float2(2.f * a01, 2.f * a11), S2 = make_float2(sx, sy);
    float rf = 0.f;
#pragma unroll 1
    for (int r = rbeg; r < rend; r++, rowp += PW, rf += 1.f) {
      const float2 DR = __ffma2_rn(make_float2(rf, rf), T2, DR0);
      // cell q is at DR + q A (2, 0), by repeated addition (a few roundings of the offset, well
      // within the window-position term of the parity tolerance)
      float2 Dq = DR;
#pragma unroll UNROLL
      for (int q = 0; q < nw; q++, Dq = __fadd2_rn(Dq, S2)) body(Dq, rowp[q]);
    }
  }
}

template <int ORDER, bool COMP, int MODE = LPA_SEARCHED>
__device__ __forceinline__ void accumulate_sensor(typename MomentsSel<ORDER, COMP>::type &m, const LpaSensorK &S,
                                                  int4 pos, int c, float R, float R2,
                                                  float cexp, float taper, int x0, int y0,
                                                  const unsigned char *smem, bool active, unsigned *status,
                                                  float4 Q = make_float4(1.f, 0.f, 1.f, 0.f)) {
  // two samples in flight pay off only for the long order-2 bodies (fully unrolled rows
  // dispatched on their length were measured slower)
  constexpr int kUnroll = ORDER == 2 ? 2 : 1;
  walk_sensor<MODE, kUnroll>(S, pos, c, R, x0, y0, smem, active, status, Q, [&](float2 D, float2 fv) {
    window_cell<ORDER, MODE>(m, D, fv, R2, cexp, taper, Q);
  });
}

// The windows of one pass read from the tabulated cells (Section 8; see LpaLaunch::tab_hdr): the
// pixel's even lattice cell in each colour phase follows from integer arithmetic, and every cell
// carries its offset and its weight at each scale of the pass, so nothing is searched or evaluated
// per pixel. The cells are sorted by distance and the windows are nested: cells n_{q-1} .. n_q - 1
// lie in the windows of slots q .. NSP - 1 and are added to those sums only (no per-cell test).
#ifndef LPA_TAB_PREFETCH
#define LPA_TAB_PREFETCH 1
#endif
#ifndef LPA_TAB_UNROLL
#define LPA_TAB_UNROLL 4
#endif
constexpr int kTabUnroll = LPA_TAB_UNROLL;
template <int ORDER, int NSP, class MOM>
__device__ __forceinline__ void accumulate_table(MOM (&m)[NSP], const LpaLaunch &L, int s, int c, int pass, int npass,
                                                 int u, int v, int x0, int y0, const unsigned char *smem, bool active,
                                                 unsigned *status) {
  static_assert(NSP >= 1 && NSP <= 4, "a table cell holds four weights");
  const LpaSensorK &S = L.s[s];
  const int PW = S.box_w >> 1, PH = S.box_h >> 1;
  const float2 *planes = reinterpret_cast<const float2 *>(smem + S.off_planes);
  const int ix = u + S.ix_shift, iy = v + S.iy_shift;
  const int base = ((s * 2 + (u & 1)) * 2 + (v & 1)) * 4;
  const int nsub = (c == 1) ? 2 : 1;
#pragma unroll 1
  for (int sub = 0; sub < nsub; sub++) {
    const int ox = (c == 0) ? 0 : (c == 2 ? 1 : 1 - sub);
    const int oy = (c == 0) ? 0 : (c == 2 ? 1 : sub);
    const int ph = ox + 2 * oy;
    const int cb = (((ix - ox) & ~1) - x0) >> 1, rb = (((iy - oy) & ~1) - y0) >> 1;
    const int4 *hp = L.tab_hdr + 2 * ((base + ph) * npass + pass);
    const int4 h = __ldg(hp), nc = __ldg(hp + 1);
    const int qx0 = (int)(short)(h.z & 0xffff), qx1 = h.z >> 16, qy0 = (int)(short)(h.w & 0xffff), qy1 = h.w >> 16;
    if (!(cb + qx0 >= 0 && cb + qx1 < PW && rb + qy0 >= 0 && rb + qy1 < PH)) {
      if (active && h.y > 0) atomicOr(status, LPA_ERR_BOUNDS);
      continue;
    }
    const float2 *pl = planes + ph * (PW * PH) + rb * PW + cb;
    const float4 *cell = L.tab_cells + 2 * (size_t)h.x;
    const int n[4] = {nc.x, nc.y, nc.z, nc.w};
    int k = 0;
#if LPA_TAB_PREFETCH
    // the next cell's two records are loaded while this one is added (the table ends with one
    // padding cell, so that the load after a list's last cell stays inside it)
    float4 gn = __ldg(cell), kn = __ldg(cell + 1);
#endif
#pragma unroll
    for (int q0 = 0; q0 < NSP; q0++) {
      const int kend = min(n[q0], h.y);
#pragma unroll(kTabUnroll)
      for (; k < kend; k++) {
#if LPA_TAB_PREFETCH
        const float4 g = gn, kw = kn;
        gn = __ldg(cell + 2 * k + 2);
        kn = __ldg(cell + 2 * k + 3);
#else
        const float4 g = __ldg(cell + 2 * k);
        const float4 kw = __ldg(cell + 2 * k + 1);
#endif
        const int qc = __float_as_int(g.z);
        const float2 fv = pl[(qc >> 16) * PW + (int)(short)(qc & 0xffff)];
        if (active && sample_ok(fv)) {
          const float Kq[4] = {kw.x, kw.y, kw.z, kw.w};
          const float2 D = make_float2(g.x, g.y);
          const float2 D2 = __fmul2_rn(D, D);
          if constexpr (ORDER > 0 && NSP == 1) {  // compensated sums: one scale per pass
            const float2 W = weights(Kq[0], fv);
            m[0].add2(D, D2, W.x, W.y, W.x * Kq[0]);
          } else {
            float sm[15];
            if constexpr (ORDER > 0) MOM::monomials(D, D2, sm);
#pragma unroll
            for (int q = q0; q < NSP; q++) {
              const float2 W = weights(Kq[q], fv);  // tabulated window weight x inverse variance, times f
              if constexpr (ORDER == 0) m[q].add0(W.x, W.y, W.x * Kq[q], 1.f);
              else m[q].adds(sm, D, D2, W.x, W.y, W.x * Kq[q]);
            }
          }
        }
      }
    }
  }
}

#ifndef LPA_BATCH_REREAD
#define LPA_BATCH_REREAD 1
#endif

template <bool V, typename T>
__device__ __forceinline__ T reread(const T &x) {
  if constexpr (V) return *reinterpret_cast<const volatile T *>(&x);
  else return x;
}

// One output tile (16 x TH pixels) of frame L, by a CTA of 16*TH threads (one per pixel).
// GLOBAL_MAPS: L is a shared-memory copy of a descriptor in global memory, and `maps` is that
// global descriptor, whose tensor maps the bulk copies use (otherwise `maps` is &L).
// `phase` is the parity of the CTA's mbarrier use for this tile. Returns false when the CTA must
// stop (a bounded wait ran out here or in another CTA).
// The staged footprint of tile `tile` (TR output rows) in each sensor, by threads 0 .. S - 1: the
// sensor-space bounding box of the tile's pixel points, grown by the largest window's half extent
// and the margin; x origin on a 16-byte boundary.
template <int TR>
__device__ __forceinline__ void stage_footprint(const LpaLaunch &L, int tile, int *fp_x0, int *fp_y0) {
  const int tid = threadIdx.x;
  if (tid >= L.n_sensors) return;
  const int u0 = (tile % L.tiles_x) * LPA_TILE, v0 = (tile / L.tiles_x) * TR;
  const LpaSensorK &Sk = L.s[tid];
  double mnx = 1e300, mny = 1e300;
#pragma unroll
  for (int k = 0; k < 4; k++) {
    double uu = u0 + (k & 1) * (LPA_TILE - 1), vv = v0 + (k >> 1) * (TR - 1);
    double qx = Sk.G[0] * uu + Sk.G[1] * vv + Sk.G[2];
    double qy = Sk.G[3] * uu + Sk.G[4] * vv + Sk.G[5];
    mnx = fmin(mnx, fmin(fmax(qx, -LPA_FAR), LPA_FAR));
    mny = fmin(mny, fmin(fmax(qy, -LPA_FAR), LPA_FAR));
  }
  int x0 = (int)floor(mnx - Sk.ext_x);
  int y0 = (int)floor(mny - Sk.ext_y);
  x0 -= ((x0 % 8) + 8) % 8;
  y0 -= (y0 & 1);
  fp_x0[tid] = x0;
  fp_y0[tid] = y0;
}

// One thread issues the bulk tensor copies of every sensor's footprint into staging buffer `stage`
// and the byte count they complete on `mbar`.
template <bool GLOBAL_MAPS>
__device__ __forceinline__ void stage_issue(const LpaLaunch &L, const LpaLaunch *maps, unsigned char *smem, int stage,
                                            uint64_t *mbar, const int *fp_x0, const int *fp_y0) {
  const int S = L.n_sensors;
  // tensor maps kept in global memory are rewritten between launches at the same addresses:
  // make this launch's contents visible to the tensor-map proxy before the copies use them
  if (GLOBAL_MAPS)
    for (int s = 0; s < S; s++) tensormap_acquire(&maps->s[s].tmap);
  mbar_arrive_expect_tx(mbar, L.tx_bytes);
  for (int s = 0; s < S; s++) {
    if (L.conv)  // the four colour-phase planes of the footprint, converted: [4][box_h / 2][box_w / 2]
      tma_load_3d(smem + L.s[s].off_planes, &maps->s[s].tmap, fp_x0[s] >> 1, fp_y0[s] >> 1, 0, mbar);
    else
      tma_load_2d(smem + (stage ? L.s[s].off_raw2 : L.s[s].off_raw), &maps->s[s].tmap, fp_x0[s], fp_y0[s], mbar);
  }
}

// STAGED: the footprint (fp_x0, fp_y0) and the copies of this tile into buffer `stage` were issued
// before the call (the caller waits for copies in flight if this returns false).
template <int ORDER, bool COMP, bool DIAG, int TH, bool GLOBAL_MAPS, int MODE = LPA_SEARCHED, int PX = 1,
          bool STAGED = false>
__device__ __forceinline__ bool process_tile(const LpaLaunch &L, const LpaLaunch *maps, int tile, unsigned char *smem, uint64_t *mbar,
                                             uint32_t phase, int *fp_x0, int *fp_y0,
                                             Anchor (*anchors)[LPA_MAX_SENSORS], int stage = 0) {
  constexpr int NT = LPA_TILE * TH;  // threads
  constexpr int TR = TH * PX;        // tile rows: PX pixels per thread, TH rows apart
  const int tid = threadIdx.x;
  // descriptor fields used across the pixel loops: with a shared-memory descriptor they are read
  // again at each use rather than held in registers through the loops
#define RD(x) reread<GLOBAL_MAPS && LPA_BATCH_REREAD>(x)
  // once any CTA's bounded wait has run out, later CTAs retire at once
  if (*reinterpret_cast<volatile unsigned int *>(L.status) & LPA_ERR_TIMEOUT) return false;
  const int tu = tile % L.tiles_x, tv = tile / L.tiles_x;
  const int u0 = tu * LPA_TILE, v0 = tv * TR;
  const int S = L.n_sensors;

  if constexpr (!STAGED) stage_footprint<TR>(L, tile, fp_x0, fp_y0);
  constexpr int NA = 2 * (TR / LPA_ANCHOR);  // anchor blocks per tile
  if (tid >= 32 && tid < 32 + NA * S) {
    const int k = tid - 32, a = k % NA, s = k / NA;
    const LpaSensorK &Sk = L.s[s];
    double uu = u0 + (a & 1) * LPA_ANCHOR, vv = v0 + (a >> 1) * LPA_ANCHOR;
    double qx = fmin(fmax(Sk.G[0] * uu + Sk.G[1] * vv + Sk.G[2], -LPA_FAR), LPA_FAR);
    double qy = fmin(fmax(Sk.G[3] * uu + Sk.G[4] * vv + Sk.G[5], -LPA_FAR), LPA_FAR);
    double flx = floor(qx), fly = floor(qy);
    anchors[a][s] = Anchor{(int)flx, (int)fly, (float)(qx - flx), (float)(qy - fly)};
  }
  __syncthreads();
  if constexpr (!STAGED)
    if (tid == 0) stage_issue<GLOBAL_MAPS>(L, maps, smem, 0, mbar, fp_x0, fp_y0);
  bool landed = mbar_wait_bounded(mbar, phase, 1u << 20);
  landed = __syncthreads_and(landed);
  if (!landed) {
    if (tid == 0) {
      atomicOr(L.status, LPA_ERR_TIMEOUT);
      mbar_wait_bounded(mbar, phase, 1u << 20);  // let copies in flight land before the CTA retires
    }
    return false;
  }

  // convert the staged raw values once per sample: Eq. 18 and the inverse of Eq. 20 (its square
  // root for the printed weight K / s); frames converted ahead of the launch arrive as such
  constexpr bool LIT = MODE == LPA_LITERAL;
  const int n_conv = L.conv ? 0 : S;
  for (int s = 0; s < n_conv; s++) {
    const LpaSensorK &Sk = L.s[s];
    const uint16_t *raw = reinterpret_cast<const uint16_t *>(smem + (stage ? Sk.off_raw2 : Sk.off_raw));
    float2 *planes = reinterpret_cast<float2 *>(smem + Sk.off_planes);
    const int bw = Sk.box_w, n = bw * Sk.box_h, PW = bw >> 1, PP = (bw >> 1) * (Sk.box_h >> 1);
    const int x0 = fp_x0[s], y0 = fp_y0[s];
    const bool scalar = !Sk.bias && !Sk.rvar && !Sk.satf && !Sk.prnu;
    const int W = Sk.width, H = Sk.height;
    const int step_y = NT / bw, step_x = NT - step_y * bw;
    int lx = tid % bw, ly = tid / bw;
    for (int e = tid; e < n; e += NT) {
      const int X = x0 + lx, Y = y0 + ly;
      const float2 v = (X >= 0 && X < W && Y >= 0 && Y < H) ? convert_sample<LIT>(Sk, scalar, X, Y, (float)raw[e])
                                                          : stage_pair(0.f, 0.f);
      planes[((lx & 1) + 2 * (ly & 1)) * PP + (ly >> 1) * PW + (lx >> 1)] = v;
      lx += step_x;
      ly += step_y;
      if (lx >= bw) {
        lx -= bw;
        ly += 1;
      }
    }
  }
  __syncthreads();

  constexpr bool TAB_ = lpa_mode_tab(MODE);
  if constexpr (!TAB_) {
    if (RD(L.off_pos) == 0u) {  // a plan without the position table (offset 0 holds a raw box)
      if (tid == 0) atomicOr(L.status, LPA_ERR_BOUNDS);
      return false;
    }
  } else {
    // a table built for another number of scales per pass (its passes would not be this kernel's)
    if (RD(L.tab_nsp) != (GLOBAL_MAPS ? 1 : MultiScale<ORDER, COMP, MODE>::value) || L.tab_hdr == nullptr) {
      if (tid == 0) atomicOr(L.status, LPA_ERR_BOUNDS);
      return false;
    }
  }
  // PX output pixels per thread, one after the other: slot k takes the rows k TH .. k TH + TH - 1
#pragma unroll 1
  for (int slot = 0; slot < PX; slot++) {
    // pixel of this thread: warp = parity class x half tile, lanes 8 x 4 at stride 2
    const int warp = tid >> 5, lane = tid & 31;
    const int par = warp & 3, hf = warp >> 2;
    const int u = u0 + 2 * (lane & 7) + (par & 1);
    const int v = v0 + 2 * ((lane >> 3) + 4 * hf) + (par >> 1) + slot * TH;
    const bool pix = (u < RD(L.out_w)) && (v < RD(L.out_h));
    const int ab = ((u - u0) >> 3) + 2 * ((v - v0) >> 3);  // < NA
    const int du = (u - u0) & 7, dv = (v - v0) & 7;
    constexpr int P = n_unknowns(ORDER);
    const int J = RD(L.n_scales);
    const int NL = J + ORDER;
    const size_t plane_px = (size_t)RD(L.out_w) * RD(L.out_h);
    const size_t opix = (size_t)v * RD(L.out_w) + u;
    const float log2e = 1.4426950408889634f;

    constexpr bool TAB = lpa_mode_tab(MODE), STEER = lpa_mode_steered(MODE), GRAD = MODE == LPA_GRADIENTS;
    constexpr bool F64 = !lpa_mode_f32(MODE);  // the FP64 re-solve is compiled in
    // the pixel's point in each sensor, once: anchor (FP64 at the 8x8 block corner) + small FP32
    // step, split into sample cell and fraction; every channel and scale reads it back
    int4 *pos = reinterpret_cast<int4 *>(smem + RD(L.off_pos)) + tid;
    if constexpr (!TAB) {
  #pragma unroll 1
      for (int s = 0; s < S; s++) {
        const Anchor &an = anchors[ab][s];
        const LpaSensorK &Sk = L.s[s];
        const float px = an.fx + (float)du * Sk.Gf[0] + (float)dv * Sk.Gf[1];
        const float py = an.fy + (float)du * Sk.Gf[2] + (float)dv * Sk.Gf[3];
        const float flx = floorf(px), fly = floorf(py);
        pos[s * NT] = make_int4(an.ix + (int)flx, an.iy + (int)fly, __float_as_int(px - flx), __float_as_int(py - fly));
      }
    }
    float4 Q = make_float4(1.f, 0.f, 1.f, 0.f);  // steering matrix of this pixel (Section 5.4)
    if constexpr (STEER)
      if (pix) Q = make_float4(L.aux[opix * 3], L.aux[opix * 3 + 1], L.aux[opix * 3 + 2], 0.f);

    using MOM = typename MomentsSel<ORDER, COMP>::type;
    // the fit of one (channel, scale) from its moments: factorised unless no lane of the warp has as
    // many samples as unknowns (such a fit is not usable whatever its pivots; on near-translational
    // rigs the lanes share one sample layout, so whole warps qualify)
    auto fit_of = [&](const MOM &m) {
      FitOut f;
      if (__all_sync(LPA_FULL, m.count() < (float)P)) {
        f.valid = false;
        f.c0 = f.var = f.c1 = f.c2 = 0.f;
        f.dmin = f.dmax = 0.f;
      } else {
        f = solve_with_fallback<P, MOM, GRAD, F64>(m, RD(L.min_pivot), RD(L.cond_fallback));
      }
      return f;
    };
    auto put_level = [&](int c, int level, const FitOut &f) {
      if (DIAG && pix) {
        float *o = L.levels + (((size_t)c * NL + level) * plane_px + opix) * 2;
        o[0] = f.valid ? f.c0 : __int_as_float(0x7fffffff);
        o[1] = f.valid ? f.var : __int_as_float(0x7fffffff);
      }
    };
    // order fallback at the largest scale (m holds its moments when any lane needs it), then the store
    auto finish = [&](int c, Ici &ici, const MOM &m) {
      const bool need = ici.choice == 255 && pix;
      if (DIAG || __any_sync(LPA_FULL, need)) {
        auto take = [&](const FitOut &f, int i) {
          put_level(c, J + i, f);
          if (ici.choice == 255 && f.valid) {
            ici.choice = J + i;
            ici.val = f.c0;
          }
        };
        if constexpr (ORDER >= 1) take(fallback_fit<ORDER, 0, F64>(m, RD(L.min_pivot), RD(L.cond_fallback)), 0);
        if constexpr (ORDER >= 2) take(fallback_fit<ORDER, 1, F64>(m, RD(L.min_pivot), RD(L.cond_fallback)), 1);
      }
      if (pix) {
        if (RD(L.out_half))
          reinterpret_cast<__half *>(RD(L.out))[c * plane_px + opix] = __float2half_rn(ici.val);
        else
          reinterpret_cast<float *>(RD(L.out))[c * plane_px + opix] = ici.val;
        if (RD(L.choice)) RD(L.choice)[c * plane_px + opix] = (uint8_t)ici.choice;
      }
    };

    // the persistent many-frame kernel walks once per scale (its register budget, shared by every
    // frame it serves, has no room for the sums of several scales)
    constexpr int NSP = GLOBAL_MAPS ? 1 : MultiScale<ORDER, COMP, MODE>::value;
    if constexpr (NSP > 1 || TAB) {
      if (TAB || J >= 2) {
        // all scales of a channel from one walk per sensor (up to NSP scales per pass): slot q of
        // a pass holds scale j0 + q - lead, so that the pass's largest scale is always the last slot
  #pragma unroll 1
        for (int c = 0; c < 3; c++) {
          Ici ici;
          ici.reset(pix);
          MOM m[NSP];
          const float gsc = (c == 1) ? RD(L.green_ratio) : 1.f;
          // the first pass takes what the later full passes leave (the small scales), so that the
          // largest scales share the longest walk
          const int npass = lpa_n_passes(J, NSP);
  #pragma unroll 1
          for (int pass = 0, j0 = 0, nj = lpa_first_pass_scales(J, NSP); pass < npass; pass++, j0 += nj, nj = NSP) {
            if (!DIAG && __all_sync(LPA_FULL, ici.done)) break;
            const int lead = NSP - nj;
            float R2s[NSP], cxs[NSP];
  #pragma unroll
            for (int q = 0; q < NSP; q++) {
              const float sg = RD(L.sigma[q >= lead ? j0 + q - lead : j0]) * gsc;
              const float Rq = RD(L.trunc_k) * sg;
              R2s[q] = q >= lead ? Rq * Rq : -1.f;
              cxs[q] = -log2e / (2.f * sg * sg);
              m[q].zero();
            }
            const float R = RD(L.trunc_k) * RD(L.sigma[j0 + nj - 1]) * gsc;
            const float taper = RD(L.taper);
            const bool act = DIAG ? pix : !ici.done;
  #pragma unroll 1
            for (int s = 0; s < S; s++) {
              if constexpr (TAB)
                accumulate_table<ORDER, NSP>(m, L, s, c, pass, npass, u, v, fp_x0[s], fp_y0[s], smem, act, L.status);
              else
                walk_sensor<MODE, 1>(L.s[s], pos[s * NT], c, R, fp_x0[s], fp_y0[s], smem, act, RD(L.status), Q,
                                     [&](float2 D, float2 fv) { window_cell_ms<ORDER, NSP, MODE>(m, D, fv, R2s, cxs, taper, Q); });
            }
            // the fits in ascending scale order
  #pragma unroll
            for (int q = 0; q < NSP; q++) {
              if (q >= lead) {
                if (!DIAG && __all_sync(LPA_FULL, ici.done)) break;
                const FitOut f = fit_of(m[q]);
                put_level(c, j0 + q - lead, f);
                ici.step(f, j0 + q - lead, RD(L.ici_gamma));
              }
            }
          }
          finish(c, ici, m[NSP - 1]);
        }
        continue;  // next pixel slot
      }
    }

  #pragma unroll 1
    for (int c = GRAD ? 1 : 0; c < (GRAD ? 2 : 3); c++) {  // the gradient pass fits the green channel only
      Ici ici;
      ici.reset(pix);
      MOM m;
      const float gsc = (c == 1) ? RD(L.green_ratio) : 1.f;
  #pragma unroll 1
      for (int j = 0; j < J; j++) {
        if (!DIAG && __all_sync(LPA_FULL, ici.done)) break;
        m.zero();
        const float sg = RD(L.sigma[j]) * gsc;
        const float R = RD(L.trunc_k) * sg, R2 = R * R;
        const float cexp = -log2e / (2.f * sg * sg);
        const bool act = DIAG ? pix : !ici.done;
  #pragma unroll 1
        for (int s = 0; s < S; s++)
          accumulate_sensor<ORDER, COMP, MODE>(m, L.s[s], pos[s * NT], c, R, R2, cexp, RD(L.taper), fp_x0[s],
                                                fp_y0[s], smem, act, RD(L.status), Q);
        const FitOut f = fit_of(m);
        if constexpr (GRAD) {  // Section 5.4: the order-1 fit's linear coefficients; 0 if not usable
          if (pix) {
            L.aux[opix * 2] = f.valid ? f.c1 : 0.f;
            L.aux[opix * 2 + 1] = f.valid ? f.c2 : 0.f;
          }
          break;
        }
        put_level(c, j, f);
        ici.step(f, j, RD(L.ici_gamma));
      }
      if constexpr (!GRAD) finish(c, ici, m);
    }
  }
  return true;
#undef RD
}

// Single frame: one CTA per tile (tiles tile0 .. tile0 + gridDim.x - 1).
// Resident CTAs per SM the single-frame kernel is compiled for: the order-2 sums of four scales
// need about 200 registers a thread (one 16-row CTA or two 8-row CTAs per SM).
#ifndef LPA_M2_CTAS_256
#define LPA_M2_CTAS_256 2  // resident 256-thread CTAs per SM the multi-scale order-2 kernel is built for
#endif
template <int ORDER, bool COMP, int TH, int MODE>
struct FrameOccupancy {
  static constexpr int value = (ORDER == 2 && MultiScale<ORDER, COMP, MODE>::value > 1) ? LPA_M2_CTAS_256 * 16 / TH
                               : ORDER == 0                                              ? LPA_M0_CTAS_256 * 16 / TH
                                                                                         : 16 / TH * 2;
};

// PX pixels per thread: a CTA of 16 x TH threads reconstructs a 16 x (TH PX) tile, each thread its
// pixels one after the other (the staged footprint and its conversion serve PX times the pixels).
// STAGES 2: CTA b takes the tiles tile0 + b + k gridDim.x of the launch's range and copies each
// next tile's raw boxes into the other staging buffer before it reconstructs the current tile, so
// that the copies land while it computes.
template <int ORDER, bool COMP, bool DIAG, int TH, int MODE = LPA_SEARCHED, int PX = 1, int STAGES = 1>
__global__ void __launch_bounds__(LPA_TILE *TH, (FrameOccupancy<ORDER, COMP, TH, MODE>::value)) lpa_reconstruct(const __grid_constant__ LpaLaunch L) {
  static_assert(STAGES == 1 || STAGES == 2, "one or two staging buffers");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int fp_x0[STAGES][LPA_MAX_SENSORS], fp_y0[STAGES][LPA_MAX_SENSORS];
  __shared__ Anchor anchors[2 * TH * PX / LPA_ANCHOR][LPA_MAX_SENSORS];
  __shared__ __align__(8) uint64_t mbar[STAGES];
  if (threadIdx.x < STAGES) mbar_init(&mbar[threadIdx.x], 1);
  if constexpr (STAGES == 1) {
    process_tile<ORDER, COMP, DIAG, TH, false, MODE, PX>(L, &L, L.tile0 + blockIdx.x, smem, &mbar[0], 0u, fp_x0[0],
                                                         fp_y0[0], anchors);
  } else {
    constexpr int TR = TH * PX;
    const int end = L.tile_count > 0 ? L.tile0 + L.tile_count : L.tiles_x * L.tiles_y;
    int t = L.tile0 + (int)blockIdx.x;
    if (t >= end) return;
    stage_footprint<TR>(L, t, fp_x0[0], fp_y0[0]);
    __syncthreads();  // the footprint and the barrier initialisation before the copies
    if (threadIdx.x == 0) stage_issue<false>(L, &L, smem, 0, &mbar[0], fp_x0[0], fp_y0[0]);
    // the k-th tile of this CTA uses buffer k & 1 at mbarrier phase (k >> 1) & 1; the buffer the
    // next tile takes was last read by the previous tile, which every thread has finished
    for (int k = 0; t < end; k++, t += (int)gridDim.x) {
      const int st = k & 1, nx = t + (int)gridDim.x;
      const bool ahead = nx < end;
      if (ahead) {
        stage_footprint<TR>(L, nx, fp_x0[st ^ 1], fp_y0[st ^ 1]);
        __syncthreads();
        if (threadIdx.x == 0) stage_issue<false>(L, &L, smem, st ^ 1, &mbar[st ^ 1], fp_x0[st ^ 1], fp_y0[st ^ 1]);
      }
      const bool ok = process_tile<ORDER, COMP, DIAG, TH, false, MODE, PX, true>(
          L, &L, t, smem, &mbar[st], (uint32_t)((k >> 1) & 1), fp_x0[st], fp_y0[st], anchors, st);
      if (!__syncthreads_and(ok)) {
        // let the copies in flight land before the CTA retires (a wait on a completed phase
        // returns at once)
        if (threadIdx.x == 0) {
          mbar_wait_bounded(&mbar[st], (uint32_t)((k >> 1) & 1), 1u << 20);
          if (ahead) mbar_wait_bounded(&mbar[st ^ 1], (uint32_t)(((k + 1) >> 1) & 1), 1u << 20);
        }
        return;
      }
    }
  }
}

// Conversion ahead of the reconstruction (LpaLaunch::conv): rows [R.r0[s], R.r1[s]) of sensor s =
// blockIdx.y into its colour-phase planes (r1 may be the height + 1 of an odd height: that row is
// outside the frame and writes zeros), with the arithmetic the reconstruction kernels use when
// they convert staged footprints themselves (convert_sample), so the staged values are the same.
// Each thread takes eight samples of a row per step (one 16-byte load; the rows of the raw frame
// are 16-byte aligned and padded to a multiple of 8 samples) and writes the four of each phase
// column as two 16-byte stores, so that a warp's loads and stores are contiguous.
template <bool LIT>
__global__ void __launch_bounds__(256) lpa_convert(const __grid_constant__ LpaLaunch L, const LpaRows R) {
  const int s = blockIdx.y;
  const LpaSensorK &Sk = L.s[s];
  const int r0 = R.r0[s], r1 = R.r1[s];
  if (r1 <= r0) return;
  const int CP = Sk.conv_pitch, W = Sk.width;
  const int G = (CP + 3) >> 2;  // groups of four phase columns (eight samples) per row
  const bool scalar = !Sk.bias && !Sk.rvar && !Sk.satf && !Sk.prnu;
  const long n = (long)(r1 - r0) * G;
  const size_t plane = (size_t)Sk.conv_h * CP;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int Y = r0 + (int)(i / G), c0 = 4 * (int)(i % G);
    const int X0 = 2 * c0;
    const bool in_row = Y < Sk.height;  // the padding row of an odd height converts to zeros
    uint16_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (in_row && X0 < W) {
      const uint4 q = *reinterpret_cast<const uint4 *>(Sk.raw + (size_t)Y * Sk.raw_pitch + X0);
      const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int k = 0; k < 4; k++) {
        v[2 * k] = (uint16_t)(w4[k] & 0xffffu);
        v[2 * k + 1] = (uint16_t)(w4[k] >> 16);
      }
    }
    float2 e[4], o[4];  // columns c0 .. c0 + 3 of the even-x and the odd-x phase
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const int X = X0 + 2 * k;
      e[k] = in_row && X < W ? convert_sample<LIT>(Sk, scalar, X, Y, (float)v[2 * k]) : stage_pair(0.f, 0.f);
      o[k] = in_row && X + 1 < W ? convert_sample<LIT>(Sk, scalar, X + 1, Y, (float)v[2 * k + 1]) : stage_pair(0.f, 0.f);
    }
    float2 *de = Sk.conv + (size_t)(2 * (Y & 1)) * plane + (size_t)(Y >> 1) * CP + c0;  // colour phase (0, Y & 1)
    float2 *dodd = de + plane;                                                         // colour phase (1, Y & 1)
    if (c0 + 4 <= CP) {
      reinterpret_cast<float4 *>(de)[0] = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
      reinterpret_cast<float4 *>(de)[1] = make_float4(e[2].x, e[2].y, e[3].x, e[3].y);
      reinterpret_cast<float4 *>(dodd)[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
      reinterpret_cast<float4 *>(dodd)[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
    } else {
#pragma unroll
      for (int k = 0; k < 4; k++)
        if (c0 + k < CP) {
          de[k] = e[k];
          dodd[k] = o[k];
        }
    }
  }
}

// Resident CTAs per SM the persistent kernel is compiled for (register cap 64K / (threads x this)):
// the lower orders need fewer registers, so they can keep more warps resident to hide staging.
template <int ORDER, int TH>
struct BatchOccupancy {
  static constexpr int value = (ORDER == 0 ? 4 : ORDER == 1 ? 3 : 2) * 16 / TH;
};

// Many frames in one launch, one kernel per polynomial order: persistent CTAs take tiles from
// the order's device-wide counter over its segment of the tile list (frame index, tile index),
// most expensive frames first as ordered by the host.
template <int ORDER, bool COMP, int TH>
__global__ void __launch_bounds__(LPA_TILE *TH, (BatchOccupancy<ORDER, TH>::value)) lpa_reconstruct_batch(const __grid_constant__ LpaBatch B) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int fp_x0[LPA_MAX_SENSORS], fp_y0[LPA_MAX_SENSORS];
  __shared__ Anchor anchors[4][LPA_MAX_SENSORS];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int next;
  __shared__ LpaLaunch frame;  // the current tile's frame descriptor (kernel-parameter-like reads)
  if (threadIdx.x == 0) mbar_init(&mbar, 1);
  const int t_end = B.bounds[ORDER + 1];
  const int t_begin = B.bounds[ORDER];
  uint32_t phase = 0;
  int cur = -1;
  for (;;) {
    __syncthreads();  // every thread is done with the previous tile's staging and descriptor
    if (threadIdx.x == 0) next = t_begin + (int)atomicAdd(B.counters + ORDER, 1u);
    __syncthreads();
    const int t = next;
    if (t >= t_end) break;
    const int2 ft = B.tiles[t];
    if (ft.x != cur) {  // uniform: every thread read the same tile
      const int4 *src = reinterpret_cast<const int4 *>(B.frames + ft.x);
      int4 *dst = reinterpret_cast<int4 *>(&frame);
      for (int i = threadIdx.x; i < (int)(sizeof(LpaLaunch) / sizeof(int4)); i += LPA_TILE * TH) dst[i] = src[i];
      cur = ft.x;
      __syncthreads();
    }
    const bool ok = process_tile<ORDER, COMP, false, TH, true>(frame, B.frames + ft.x, ft.y, smem, &mbar, phase,
                                                               fp_x0, fp_y0, anchors);
    if (!__syncthreads_and(ok)) break;
    phase ^= 1u;
  }
}

// Self-test of the bounded wait: an mbarrier that expects 16 bytes no copy will deliver. The wait
// gives up after `limit` tries or `max_cycles` clock cycles, whichever comes first, and reports
// LPA_ERR_TIMEOUT in the status word exactly as a reconstruction whose copies never land would.
static __global__ void lpa_selftest_wait(unsigned int *status, uint32_t limit, long long max_cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_arrive_expect_tx(&bar, 16);
    const long long t0 = clock64();
    bool done = false;
    for (uint32_t i = 0; i < limit && !done && clock64() - t0 < max_cycles; ++i) done = mbar_try_wait_hint(&bar, 0, 1000);
    if (!done) atomicOr(status, LPA_ERR_TIMEOUT);
  }
}

}  // namespace lpa
