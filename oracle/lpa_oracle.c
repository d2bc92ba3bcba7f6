/*
 * FP64 CPU oracle for multi-sensor HDR reconstruction by noise-aware local
 * polynomial approximation (LPA), after Kronander, Gustavson, Bonnet, Ynnerman
 * and Unger, "A Unified Framework for Multi-Sensor HDR Video Reconstruction".
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg load this file's library. The product (CUDA)
 * path never calls it, and the two share no code, header, table or helper.
 *
 * Everything here is the plain definition, in double precision, one output
 * pixel at a time, with no blocking, fusion or reordering:
 *   Section 3 / 4.2   output point and sample positions X_{s,i} = T_s(x_{s,i})
 *   Section 6, Eq. 18 radiant power estimate  f = (y - b) / (g t a n)
 *   Section 6.1, Eq. 20 plug-in variance     s2 = (g^2 t a n f + Var r) / (g t a n)^2
 *   Section 6.1        saturated samples are excluded (saturation frame)
 *   Section 5.1        basis phi(d) = [1, d, tril(d d^T)] truncated to order M
 *   Section 5.2, Eq. 6 C = (Phi^T W Phi)^{-1} Phi^T W f,  output C_0
 *   Section 5.3.1, Eq. 8 Gaussian window, h_G = h_RB / sqrt(2)
 *   Section 5.3.1      a scale is usable only if Phi^T W Phi is invertible
 * plus the readings the paper leaves open (the kernel follows the same ones):
 *   - noise weight 1/s2 (the Gaussian log-likelihood of Section 5.2);
 *     weight_mode = 1 keeps the printed 1/s for the record;
 *   - window exp(-|d|^2 / (2 sigma^2)) truncated at k*sigma and lowered by
 *     exp(-k^2/2) so that it reaches zero continuously at the cut;
 *   - f used inside Eq. 20 is clamped at zero;
 *   - "invertible" = every pivot of the Jacobi-equilibrated matrix is above
 *     min_pivot, and at least as many samples as unknowns;
 *   - scale choice among several scales by intersection of confidence
 *     intervals (LPA-ICI, the rule of the LPA book the paper cites in
 *     Sections 2.3 and 5.3.1): intervals C_0 +- gamma*sqrt(Var C_0) in
 *     ascending scale order, keep the last scale whose running intersection
 *     is non-empty; no usable scale -> lower the order at the largest scale;
 *     no sample at all -> NaN.
 *   - Var C_0 = l^T (Phi^T W S W Phi) l with l = (Phi^T W Phi)^{-1} e_0 and
 *     S = diag(s2): the covariance of the estimate under independent
 *     Gaussian samples (Section 6.1 assumes independence).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_SCALES 8
#define ORC_MAX_P 6
#define ORC_MAX_LEVELS (ORC_MAX_SCALES + 2)

typedef struct {
  int32_t width, height, pitch;   /* raw layout, pitch in elements */
  const uint16_t *raw;            /* [height][pitch] digital values y, or NULL in value mode */
  const double *value_f;          /* value mode: radiant power estimate per pixel [height][width] */
  const double *value_var;        /* value mode: its variance; not finite or <= 0 => sample excluded */
  double gain, exposure, nd;      /* g_s, t_s, n_s */
  double read_var, black, sat;    /* Var r, bias b, saturation level (scalar calibration) */
  const double *bias_px;          /* optional per-pixel bias frame b_{s,i}        [height][width] */
  const double *prnu_px;          /* optional per-pixel non-uniformity a_{s,i}     [height][width] */
  const double *read_var_px;      /* optional per-pixel read-noise variance        [height][width] */
  const double *sat_px;           /* optional per-pixel saturation frame           [height][width] */
  double affine[6];               /* T_s: sensor px -> reference px, row-major 2x3 */
} orc_sensor;

typedef struct {
  int32_t order;                  /* M in {0, 1, 2} */
  int32_t n_scales;               /* J >= 1 */
  double sigma[ORC_MAX_SCALES];   /* R/B window scales in reference px, ascending */
  double green_ratio;             /* sigma_G / sigma_RB */
  double trunc_k;                 /* window radius in units of sigma */
  double ici_gamma;               /* confidence-interval half-width in standard deviations */
  double min_pivot;               /* smallest admissible equilibrated pivot */
  double out_affine[6];           /* output px -> reference px, row-major 2x3 */
  int32_t weight_mode;            /* 0: K / s2 ; 1: K / s (printed form of Eq. 6) */
} orc_params;

/* ------------------------------------------------------------------ helpers */

static int n_unknowns(int order) { return order == 0 ? 1 : (order == 1 ? 3 : 6); }

/* Section 5.1: phi(d) = [1, dx, dy, tril(d d^T)] with tril(d d^T) = [dx^2, dx*dy, dy^2]. */
static void basis(double dx, double dy, int P, double *phi) {
  double full[6] = {1.0, dx, dy, dx * dx, dx * dy, dy * dy};
  for (int m = 0; m < P; m++) phi[m] = full[m];
}

static void invert_affine(const double m[6], double inv[6]) {
  double det = m[0] * m[4] - m[1] * m[3];
  inv[0] = m[4] / det;
  inv[1] = -m[1] / det;
  inv[3] = -m[3] / det;
  inv[4] = m[0] / det;
  inv[2] = -(inv[0] * m[2] + inv[1] * m[5]);
  inv[5] = -(inv[3] * m[2] + inv[4] * m[5]);
}

/* Section 2.5: RGGB Bayer colour of sensor pixel (x, y): 0 = R, 1 = G, 2 = B. */
static int cfa_color(int x, int y) {
  if ((x & 1) == 0 && (y & 1) == 0) return 0;
  if ((x & 1) == 1 && (y & 1) == 1) return 2;
  return 1;
}

/* Section 6: Eqs. 18 and 20 for one digital value. Returns 1 if the sample is
 * excluded (saturated, Section 6.1), else 0 with f and s2 set. */
int orc_radiometry(double y, double b, double g, double t, double a, double n,
                   double read_var, double sat, double *f, double *s2) {
  if (y >= sat) return 1;
  double scale = g * t * a * n;
  double fhat = (y - b) / scale;                                   /* Eq. 18 */
  double fpos = fhat > 0.0 ? fhat : 0.0;
  *f = fhat;
  *s2 = (g * g * t * a * n * fpos + read_var) / (scale * scale);   /* Eq. 20 */
  return 0;
}

/* Eqs. 18 and 20 for every pixel of one sensor's raw frame (the sensor's scalar calibration or
 * its per-pixel frames): f and s2 [height][width]; excluded (saturated) pixels get s2 = +inf. The
 * value-mode inputs that reproduce the raw-mode fit exactly, or, rounded, the fit of rounded
 * inputs. Returns 0, or -1 for a missing raw frame. */
int orc_radiometry_frame(const orc_sensor *S, double *f, double *s2) {
  if (!S || !S->raw || !f || !s2) return -1;
  for (int y = 0; y < S->height; y++)
    for (int x = 0; x < S->width; x++) {
      long idx = (long)y * S->width + x;
      double b = S->bias_px ? S->bias_px[idx] : S->black;
      double a = S->prnu_px ? S->prnu_px[idx] : 1.0;
      double rv = S->read_var_px ? S->read_var_px[idx] : S->read_var;
      double sat = S->sat_px ? S->sat_px[idx] : S->sat;
      double yv = (double)S->raw[(long)y * S->pitch + x];
      if (orc_radiometry(yv, b, S->gain, S->exposure, a, S->nd, rv, sat, &f[idx], &s2[idx])) {
        f[idx] = 0.0;
        s2[idx] = INFINITY;
      }
    }
  return 0;
}

/* One sample as the fit sees it. */
typedef struct {
  int color;
  double dx, dy;      /* X_{s,i} - P_j in reference px */
  double f, s2;       /* radiant power estimate and its variance */
  int sensor, x, y;   /* provenance */
} orc_sample;

/* Gather every non-excluded sample of every sensor whose reference position
 * lies within radius R of P (Section 4.2, Fig. 4): positions are the forward
 * transform of the sensor pixel coordinates; the sensor-space search box is
 * the bounding box of the pre-image of the disc, grown by one pixel. */
static int gather(const orc_sensor *sens, int n_sensors, const double P[2], double R,
                  orc_sample **buf, int *cap) {
  int n = 0;
  for (int s = 0; s < n_sensors; s++) {
    const orc_sensor *S = &sens[s];
    double inv[6];
    invert_affine(S->affine, inv);
    double qx = inv[0] * P[0] + inv[1] * P[1] + inv[2];
    double qy = inv[3] * P[0] + inv[4] * P[1] + inv[5];
    double hx = R * sqrt(inv[0] * inv[0] + inv[1] * inv[1]);
    double hy = R * sqrt(inv[3] * inv[3] + inv[4] * inv[4]);
    int x0 = (int)floor(qx - hx) - 1, x1 = (int)ceil(qx + hx) + 1;
    int y0 = (int)floor(qy - hy) - 1, y1 = (int)ceil(qy + hy) + 1;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > S->width - 1) x1 = S->width - 1;
    if (y1 > S->height - 1) y1 = S->height - 1;
    for (int y = y0; y <= y1; y++) {
      for (int x = x0; x <= x1; x++) {
        double X = S->affine[0] * x + S->affine[1] * y + S->affine[2];
        double Y = S->affine[3] * x + S->affine[4] * y + S->affine[5];
        double dx = X - P[0], dy = Y - P[1];
        if (dx * dx + dy * dy >= R * R) continue;
        double f, s2;
        if (S->raw) {
          long idx = (long)y * S->width + x;
          double b = S->bias_px ? S->bias_px[idx] : S->black;
          double a = S->prnu_px ? S->prnu_px[idx] : 1.0;
          double rv = S->read_var_px ? S->read_var_px[idx] : S->read_var;
          double sat = S->sat_px ? S->sat_px[idx] : S->sat;
          double yv = (double)S->raw[(long)y * S->pitch + x];
          if (orc_radiometry(yv, b, S->gain, S->exposure, a, S->nd, rv, sat, &f, &s2)) continue;
        } else {
          long idx = (long)y * S->width + x;
          f = S->value_f[idx];
          s2 = S->value_var[idx];
          if (!(s2 > 0.0) || !isfinite(s2) || !isfinite(f)) continue;
        }
        if (n == *cap) {
          *cap = *cap ? 2 * *cap : 256;
          *buf = (orc_sample *)realloc(*buf, (size_t)*cap * sizeof(orc_sample));
        }
        orc_sample *o = &(*buf)[n++];
        o->color = cfa_color(x, y);
        o->dx = dx;
        o->dy = dy;
        o->f = f;
        o->s2 = s2;
        o->sensor = s;
        o->x = x;
        o->y = y;
      }
    }
  }
  return n;
}

/* Cyclic Jacobi eigenvalue iteration of a symmetric P x P matrix; returns the
 * 2-norm condition number max|lambda| / min|lambda|. */
static double jacobi_condition(const double *Ain, int P) {
  double A[ORC_MAX_P * ORC_MAX_P];
  memcpy(A, Ain, sizeof(double) * P * P);
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < P; i++)
      for (int j = 0; j < P; j++) {
        tot += A[i * P + j] * A[i * P + j];
        if (i != j) off += A[i * P + j] * A[i * P + j];
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < P; p++)
      for (int q = p + 1; q < P; q++) {
        double apq = A[p * P + q];
        if (apq == 0.0) continue;
        double theta = (A[q * P + q] - A[p * P + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < P; k++) { /* A <- A J */
          double akp = A[k * P + p], akq = A[k * P + q];
          A[k * P + p] = c * akp - s * akq;
          A[k * P + q] = s * akp + c * akq;
        }
        for (int k = 0; k < P; k++) { /* A <- J^T A */
          double apk = A[p * P + k], aqk = A[q * P + k];
          A[p * P + k] = c * apk - s * aqk;
          A[q * P + k] = s * apk + c * aqk;
        }
      }
  }
  double lo = INFINITY, hi = 0.0;
  for (int i = 0; i < P; i++) {
    double l = fabs(A[i * P + i]);
    if (l < lo) lo = l;
    if (l > hi) hi = l;
  }
  return lo > 0.0 ? hi / lo : INFINITY;
}

/* The same condition number for a caller-supplied symmetric P x P matrix (row-major, P <= 6), so
 * that the tests can check the eigen-iteration on matrices whose spectrum is known. */
double orc_condition(const double *A, int32_t P) {
  if (!A || P < 1 || P > ORC_MAX_P) return NAN;
  return jacobi_condition(A, P);
}

/* Result of one weighted fit (one channel, one scale, one order). */
typedef struct {
  int count;         /* samples inside the window */
  int valid;         /* Phi^T W Phi numerically invertible (reading above) */
  double c0;         /* C_0 of Eq. 6 */
  double var;        /* Var C_0 */
  double min_pivot;  /* smallest pivot of the equilibrated normal matrix */
  double kappa;      /* its 2-norm condition number */
  /* Rounding scales of C_0 (diagnostics only; they do not enter the result). With
   * L1_k = sum_m |l_m phi_m(d_k)|, F1_k = sum_m |c_m phi_m(d_k)| and c = A^{-1} b the fitted
   * coefficients, a first-order perturbation of the moment sums and of the solve moves C_0 by at
   * most (relative rounding) x err_fit, and a relative perturbation of the window at each sample
   * (its evaluation and the rounding of the sample position) by at most that x err_w. */
  double err_fit;    /* sum_k w_k L1_k (|f_k| + F1_k) */
  double err_w;      /* sum_k (G_k (1 + r_k^2 / sigma^2) / s2_k) L1_k |f_k - phi(d_k)^T c|, G the Gaussian */
  double c1, c2;     /* fitted first-order coefficients (d/dx, d/dy of the local polynomial), order >= 1 */
  /* The same two rounding scales for c1 and c2 (order >= 1), with L1_k taken from the equivalent
   * kernels A^{-1} e_1 and A^{-1} e_2 of those coefficients in place of l. */
  double err_fit_c[2], err_w_c[2];
} orc_fit;

/* Squared window distance of offset (dx, dy): |d|^2, or d^T Q d for the steered window of the
 * adaptive reconstruction (Section 5.4; Q = {Q11, Q12, Q22}). */
static double wdist2(const double *Q, double dx, double dy) {
  return Q ? Q[0] * dx * dx + 2.0 * Q[1] * dx * dy + Q[2] * dy * dy : dx * dx + dy * dy;
}

/* Section 5.2, Eq. 6 for one channel at one scale and order, with the
 * Gaussian window of Eq. 8 (Section 5.3.1), or its steered form when Q is
 * given. `ell` (optional) receives the equivalent kernel
 * l_k = w_k e_0^T A^{-1} phi_k per sample (Section 5.2). */
static orc_fit fit(const orc_sample *smp, int n, int color, double sigma_c, int order,
                   const orc_params *prm, int want_kappa, double *ell, const double *Q) {
  orc_fit r = {0, 0, NAN, NAN, 0.0, INFINITY, NAN, NAN, NAN, NAN};
  int P = n_unknowns(order);
  double k = prm->trunc_k;
  double R2 = (k * sigma_c) * (k * sigma_c);
  double floor_w = exp(-0.5 * k * k);
  double A[ORC_MAX_P * ORC_MAX_P] = {0}, B[ORC_MAX_P * ORC_MAX_P] = {0}, bvec[ORC_MAX_P] = {0};
  for (int i = 0; i < n; i++) {
    const orc_sample *o = &smp[i];
    if (o->color != color) continue;
    double r2 = wdist2(Q, o->dx, o->dy);
    if (!(r2 < R2)) continue;
    r.count++;
    double K = exp(-r2 / (2.0 * sigma_c * sigma_c)) - floor_w;     /* Eq. 8, truncated and tapered */
    double w = prm->weight_mode == 1 ? K / sqrt(o->s2) : K / o->s2;  /* diagonal of W */
    double phi[ORC_MAX_P];
    basis(o->dx, o->dy, P, phi);
    for (int a = 0; a < P; a++) {
      bvec[a] += w * o->f * phi[a];                                 /* Phi^T W f */
      for (int c = 0; c < P; c++) {
        A[a * P + c] += w * phi[a] * phi[c];                        /* Phi^T W Phi */
        B[a * P + c] += w * w * o->s2 * phi[a] * phi[c];            /* Phi^T W S W Phi */
      }
    }
  }
  if (r.count == 0) return r;
  /* Jacobi equilibration D A D with D = diag(A)^{-1/2}. */
  double D[ORC_MAX_P], At[ORC_MAX_P * ORC_MAX_P];
  for (int a = 0; a < P; a++) {
    if (!(A[a * P + a] > 0.0)) return r;
    D[a] = 1.0 / sqrt(A[a * P + a]);
  }
  for (int a = 0; a < P; a++)
    for (int c = 0; c < P; c++) At[a * P + c] = D[a] * A[a * P + c] * D[c];
  /* LDL^T of the equilibrated matrix: L unit lower (stored below the diagonal), pivots d. */
  double L[ORC_MAX_P * ORC_MAX_P] = {0}, d[ORC_MAX_P];
  double minp = INFINITY;
  for (int j = 0; j < P; j++) {
    double s = At[j * P + j];
    for (int m = 0; m < j; m++) s -= L[j * P + m] * L[j * P + m] * d[m];
    d[j] = s;
    if (s < minp) minp = s;
    for (int i = j + 1; i < P; i++) {
      double t = At[i * P + j];
      for (int m = 0; m < j; m++) t -= L[i * P + m] * L[j * P + m] * d[m];
      L[i * P + j] = (s != 0.0) ? t / s : 0.0;
    }
  }
  r.min_pivot = minp;
  if (want_kappa) r.kappa = jacobi_condition(At, P);
  r.valid = (r.count >= P) && (minp > prm->min_pivot);
  /* C_0 and its variance are also reported for factorable fits below the threshold (a
   * diagnostic for decisions taken near it); the scale choice uses only usable fits. */
  if (!(minp > 0.0)) return r;
  /* l = A^{-1} e_0 = D (D A D)^{-1} D e_0 (and c = A^{-1} b the same way):
   * solve L z = D rhs, z /= d, L^T x = z, result D x. */
  double l[ORC_MAX_P], cf[ORC_MAX_P], lg[2][ORC_MAX_P];  /* lg: A^{-1} e_1, A^{-1} e_2 */
  for (int which = 0; which < (P >= 3 ? 4 : 2); which++) {
    double z[ORC_MAX_P], x[ORC_MAX_P];
    for (int i = 0; i < P; i++) {
      double e = which == 1 ? bvec[i] : (i == (which == 0 ? 0 : which - 1) ? 1.0 : 0.0);
      double s = D[i] * e;
      for (int m = 0; m < i; m++) s -= L[i * P + m] * z[m];
      z[i] = s;
    }
    for (int i = 0; i < P; i++) z[i] /= d[i];
    for (int i = P - 1; i >= 0; i--) {
      double s = z[i];
      for (int m = i + 1; m < P; m++) s -= L[m * P + i] * x[m];
      x[i] = s;
    }
    for (int i = 0; i < P; i++) (which == 0 ? l : which == 1 ? cf : lg[which - 2])[i] = D[i] * x[i];
  }
  double c0 = 0.0, v = 0.0;
  for (int a = 0; a < P; a++) {
    c0 += l[a] * bvec[a];
    for (int c = 0; c < P; c++) v += l[a] * B[a * P + c] * l[c];
  }
  r.c0 = c0;
  r.var = v;
  if (P >= 3) {
    r.c1 = cf[1];
    r.c2 = cf[2];
  }
  r.err_fit = 0.0;
  r.err_w = 0.0;
  for (int i = 0; i < n; i++) {
    const orc_sample *o = &smp[i];
    if (o->color != color) continue;
    double r2 = wdist2(Q, o->dx, o->dy);
    if (!(r2 < R2)) continue;
    double G = exp(-r2 / (2.0 * sigma_c * sigma_c));
    double nw = prm->weight_mode == 1 ? 1.0 / sqrt(o->s2) : 1.0 / o->s2;
    double phi[ORC_MAX_P], l1 = 0.0, f1 = 0.0, fit_k = 0.0;
    basis(o->dx, o->dy, P, phi);
    for (int a = 0; a < P; a++) {
      l1 += fabs(l[a] * phi[a]);
      f1 += fabs(cf[a] * phi[a]);
      fit_k += cf[a] * phi[a];
    }
    r.err_fit += (G - floor_w) * nw * l1 * (fabs(o->f) + f1);
    r.err_w += G * (1.0 + r2 / (sigma_c * sigma_c)) * nw * l1 * fabs(o->f - fit_k);
    for (int g = 0; g < 2 && P >= 3; g++) {
      double lk = 0.0;
      for (int a = 0; a < P; a++) lk += fabs(lg[g][a] * phi[a]);
      r.err_fit_c[g] += (G - floor_w) * nw * lk * (fabs(o->f) + f1);
      r.err_w_c[g] += G * (1.0 + r2 / (sigma_c * sigma_c)) * nw * lk * fabs(o->f - fit_k);
    }
  }
  if (ell) {
    for (int i = 0; i < n; i++) {
      const orc_sample *o = &smp[i];
      ell[i] = 0.0;
      if (o->color != color) continue;
      double r2 = wdist2(Q, o->dx, o->dy);
      if (!(r2 < R2)) continue;
      double K = exp(-r2 / (2.0 * sigma_c * sigma_c)) - floor_w;
      double w = prm->weight_mode == 1 ? K / sqrt(o->s2) : K / o->s2;
      double phi[ORC_MAX_P];
      basis(o->dx, o->dy, P, phi);
      double e = 0.0;
      for (int a = 0; a < P; a++) e += l[a] * phi[a];
      ell[i] = w * e;
    }
  }
  return r;
}

/* Scale choice by intersection of confidence intervals over the usable scales
 * in ascending order (see the header). Returns the chosen index or -1 and the
 * smallest |upper - lower| of the running intersection met on the way. */
int orc_ici(int n, const double *c0, const double *var, const int *valid, double gamma,
            double *margin_out) {
  double lo = -INFINITY, hi = INFINITY, margin = INFINITY;
  int chosen = -1;
  for (int j = 0; j < n; j++) {
    if (!valid[j]) continue;
    double h = gamma * sqrt(var[j]);
    double nlo = fmax(lo, c0[j] - h), nhi = fmin(hi, c0[j] + h);
    double gap = nhi - nlo;
    if (fabs(gap) < margin) margin = fabs(gap);
    if (nlo > nhi) break;
    lo = nlo;
    hi = nhi;
    chosen = j;
  }
  if (margin_out) *margin_out = margin;
  return chosen;
}

/* Levels of one (pixel, channel): 0..J-1 = order M at each scale; then
 * J + i = order M-1-i at the largest scale (the order fallback). */
static int n_levels(const orc_params *p) { return p->n_scales + p->order; }

static int check_params(const orc_sensor *sens, int n_sensors, const orc_params *p) {
  if (n_sensors < 0 || (n_sensors > 0 && !sens) || !p) return -1;
  if (p->order < 0 || p->order > 2) return -2;
  if (p->n_scales < 1 || p->n_scales > ORC_MAX_SCALES) return -3;
  for (int j = 0; j < p->n_scales; j++) {
    if (!(p->sigma[j] > 0.0)) return -4;
    if (j > 0 && !(p->sigma[j] > p->sigma[j - 1])) return -4;
  }
  if (!(p->trunc_k > 0.0) || !(p->green_ratio > 0.0) || !(p->ici_gamma >= 0.0)) return -5;
  for (int s = 0; s < n_sensors; s++) {
    const orc_sensor *S = &sens[s];
    if (S->width < 0 || S->height < 0) return -6;
    if (S->raw && S->pitch < S->width) return -6;
    if (!S->raw && (!S->value_f || !S->value_var) && S->width * S->height > 0) return -6;
    double det = S->affine[0] * S->affine[4] - S->affine[1] * S->affine[3];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return -7;
    if (S->raw && !(S->gain > 0.0 && S->exposure > 0.0 && S->nd > 0.0)) return -8;
    if (S->raw && !S->read_var_px && !(S->read_var > 0.0)) return -8;
  }
  return 0;
}

/*
 * Reconstruct the listed output pixels. Arrays:
 *   pu, pv        [n_pix] output pixel coordinates (integers, pixel centres)
 *   out           [n_pix][3] chosen C_0 per channel R, G, B (NaN: no sample)
 *   choice        [n_pix][3] chosen level (see n_levels) or -1        (optional)
 *   margin        [n_pix][3] ICI margin |upper - lower| minimum        (optional)
 *   lv_c0, lv_var, lv_pivot, lv_kappa, lv_efit, lv_ew [n_pix][3][J+M], lv_count, lv_valid
 *                 (optional; lv_efit / lv_ew are the rounding scales err_fit / err_w of orc_fit)
 * Returns 0, or a negative code for invalid arguments.
 */
/* Smallest eigenvalue of the symmetric 2x2 matrix {Q11, Q12, Q22}. */
static double min_eig2(const double *Q) {
  double h = 0.5 * (Q[0] + Q[2]), d = 0.5 * (Q[0] - Q[2]);
  return h - sqrt(d * d + Q[1] * Q[1]);
}

/* metric (optional): per output pixel the steering matrix {Q11, Q12, Q22} of the adaptive
 * reconstruction (Section 5.4): the window becomes exp(-d^T Q d / (2 sigma^2)) on the support
 * d^T Q d < (k sigma)^2; NULL = the isotropic window. */
int orc_reconstruct(const orc_sensor *sens, int n_sensors, const orc_params *p, int64_t n_pix,
                    const int32_t *pu, const int32_t *pv, const double *metric, double *out, int32_t *choice,
                    double *margin, double *lv_c0, double *lv_var, double *lv_pivot, double *lv_kappa,
                    int32_t *lv_count, int32_t *lv_valid, double *lv_efit, double *lv_ew) {
  int rc = check_params(sens, n_sensors, p);
  if (rc) return rc;
  if (n_pix < 0 || (n_pix > 0 && (!pu || !pv || !out))) return -1;
  const int J = p->n_scales, M = p->order, NL = n_levels(p);
  double rmax = p->trunc_k * p->sigma[J - 1];   /* R/B radius at the largest scale covers G too */
  if (p->green_ratio > 1.0) rmax *= p->green_ratio;
  if (metric)  /* every steering matrix must be positive definite */
    for (int64_t j = 0; j < n_pix; j++)
      if (!(min_eig2(metric + 3 * j) > 0.0)) return -3;
#pragma omp parallel
  {
    orc_sample *buf = NULL;
    int cap = 0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_pix; j++) {
      /* Section 4.2: the output pixel's point in the reference frame. */
      double P[2];
      P[0] = p->out_affine[0] * pu[j] + p->out_affine[1] * pv[j] + p->out_affine[2];
      P[1] = p->out_affine[3] * pu[j] + p->out_affine[4] * pv[j] + p->out_affine[5];
      const double *Q = metric ? metric + 3 * j : NULL;
      /* the support d^T Q d < R^2 lies within |d| < R / sqrt(lambda_min(Q)) */
      int n = gather(sens, n_sensors, P, Q ? rmax / sqrt(min_eig2(Q)) : rmax, &buf, &cap);
      for (int c = 0; c < 3; c++) {
        orc_fit lv[ORC_MAX_LEVELS];
        double sg = (c == 1) ? p->green_ratio : 1.0;
        for (int l = 0; l < J; l++)
          lv[l] = fit(buf, n, c, p->sigma[l] * sg, M, p, lv_kappa != NULL, NULL, Q);
        for (int i = 0; i < M; i++)
          lv[J + i] = fit(buf, n, c, p->sigma[J - 1] * sg, M - 1 - i, p, lv_kappa != NULL, NULL, Q);
        double c0s[ORC_MAX_LEVELS], vars[ORC_MAX_LEVELS], mg = INFINITY;
        int val[ORC_MAX_LEVELS];
        for (int l = 0; l < NL; l++) {
          c0s[l] = lv[l].c0;
          vars[l] = lv[l].var;
          val[l] = lv[l].valid;
        }
        int ch = orc_ici(J, c0s, vars, val, p->ici_gamma, &mg);
        for (int i = 0; ch < 0 && i < M; i++)
          if (val[J + i]) ch = J + i;
        out[j * 3 + c] = ch >= 0 ? c0s[ch] : NAN;
        if (choice) choice[j * 3 + c] = ch;
        if (margin) margin[j * 3 + c] = mg;
        for (int l = 0; l < NL; l++) {
          int64_t o = (j * 3 + c) * NL + l;
          if (lv_c0) lv_c0[o] = lv[l].c0;
          if (lv_var) lv_var[o] = lv[l].var;
          if (lv_pivot) lv_pivot[o] = lv[l].min_pivot;
          if (lv_kappa) lv_kappa[o] = lv[l].kappa;
          if (lv_count) lv_count[o] = lv[l].count;
          if (lv_valid) lv_valid[o] = lv[l].valid;
          if (lv_efit) lv_efit[o] = lv[l].err_fit;
          if (lv_ew) lv_ew[o] = lv[l].err_w;
        }
      }
    }
    free(buf);
  }
  return 0;
}

/*
 * Equivalent kernel of one fit (Section 5.2: the WLS solution is a linear
 * filter): for output pixel (u, v), channel c, scale sigma (R/B units) and
 * order, writes up to `cap` samples' (sensor, x, y, dx, dy, f, l_k).
 * Returns the number of samples in the window, or -1 when the fit is not
 * usable, or another negative code for bad arguments.
 */
int orc_equivalent_kernel(const orc_sensor *sens, int n_sensors, const orc_params *p, int32_t u,
                          int32_t v, int32_t c, double sigma, int32_t order, int32_t cap,
                          int32_t *o_sensor, int32_t *o_x, int32_t *o_y, double *o_dx, double *o_dy,
                          double *o_f, double *o_ell) {
  int rc = check_params(sens, n_sensors, p);
  if (rc) return rc;
  if (c < 0 || c > 2 || order < 0 || order > 2 || !(sigma > 0.0)) return -2;
  double P[2];
  P[0] = p->out_affine[0] * u + p->out_affine[1] * v + p->out_affine[2];
  P[1] = p->out_affine[3] * u + p->out_affine[4] * v + p->out_affine[5];
  double sc = sigma * (c == 1 ? p->green_ratio : 1.0);
  orc_sample *buf = NULL;
  int capb = 0;
  int n = gather(sens, n_sensors, P, p->trunc_k * sc, &buf, &capb);
  double *ell = (double *)calloc(n > 0 ? n : 1, sizeof(double));
  orc_fit r = fit(buf, n, c, sc, order, p, 0, ell, NULL);
  int w = 0;
  if (r.valid) {
    for (int i = 0; i < n; i++) {
      const orc_sample *o = &buf[i];
      double r2 = o->dx * o->dx + o->dy * o->dy;
      if (o->color != c || !(r2 < p->trunc_k * p->trunc_k * sc * sc)) continue;
      if (w < cap) {
        o_sensor[w] = o->sensor;
        o_x[w] = o->x;
        o_y[w] = o->y;
        o_dx[w] = o->dx;
        o_dy[w] = o->dy;
        o_f[w] = o->f;
        o_ell[w] = ell[i];
      }
      w++;
    }
  }
  free(ell);
  free(buf);
  return r.valid ? w : -1;
}

/*
 * First pass of the adaptive reconstruction (Section 5.4, with the green channel as in Section
 * 5.5): gradients (d/dx, d/dy in reference px) of an isotropic order-1 fit of the G channel at
 * scale grad_sigma (R/B units; G uses grad_sigma * green_ratio) at each output pixel. A pixel
 * whose fit is not usable gets gradient 0 (reading).
 */
int orc_gradients(const orc_sensor *sens, int n_sensors, const orc_params *p, double grad_sigma, int64_t n_pix,
                  const int32_t *pu, const int32_t *pv, double *gx, double *gy, double *pivot, int32_t *count,
                  double *err_fit, double *err_w) {
  int rc = check_params(sens, n_sensors, p);
  if (rc) return rc;
  if (!(grad_sigma > 0.0) || n_pix < 0 || (n_pix > 0 && (!pu || !pv || !gx || !gy))) return -2;
  const double sc = grad_sigma * p->green_ratio;
#pragma omp parallel
  {
    orc_sample *buf = NULL;
    int cap = 0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t j = 0; j < n_pix; j++) {
      double P[2];
      P[0] = p->out_affine[0] * pu[j] + p->out_affine[1] * pv[j] + p->out_affine[2];
      P[1] = p->out_affine[3] * pu[j] + p->out_affine[4] * pv[j] + p->out_affine[5];
      int n = gather(sens, n_sensors, P, p->trunc_k * sc, &buf, &cap);
      orc_fit f = fit(buf, n, 1, sc, 1, p, 0, NULL, NULL);
      gx[j] = f.valid ? f.c1 : 0.0;
      gy[j] = f.valid ? f.c2 : 0.0;
      /* optional diagnostics: the usability test's inputs and the rounding scales of c1, c2 */
      if (pivot) pivot[j] = f.min_pivot;
      if (count) count[j] = f.count;
      if (err_fit) {
        err_fit[2 * j] = f.err_fit_c[0];
        err_fit[2 * j + 1] = f.err_fit_c[1];
      }
      if (err_w) {
        err_w[2 * j] = f.err_w_c[0];
        err_w[2 * j + 1] = f.err_w_c[1];
      }
    }
    free(buf);
  }
  return 0;
}
