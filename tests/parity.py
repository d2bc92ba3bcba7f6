"""Comparison of the CUDA path's output with the FP64 oracle (test helper).

Tolerance. For the level (scale, order) used at a pixel and
channel, the GPU value g and the oracle value o must satisfy

    |g - o| <= REL_TOL * max(|o|, TAU) + U32 * (C_FIT * efit + C_W * ew)

REL_TOL = 1e-5 is the relative tolerance for FP32 accumulation; TAU = 1e-2 is the scene's
darkest radiance. efit and ew are the oracle's first-order rounding scales of that fit (see
oracle/lpa_oracle.c): efit bounds how far C_0 moves per unit relative perturbation of every
moment sum and of the normal matrix, ew how far it moves per unit relative perturbation of the
window weight at every sample. FP32 sums of n terms are off by at most about n * U32 relative,
so C_FIT covers windows of up to C_FIT samples; window evaluation (ex2.approx) and FP32 sample
positions perturb weights by a few U32 relative, covered by C_W. For well-conditioned fits of
positive data efit is about 2|C_0|, so the second term is then ~2.5e-5 relative; where the fit
cancels (dark noisy pixels, ill-conditioned normal matrices) it grows as the arithmetic requires.
FP16 output adds 2^-11 relative.

Several results are correct where the scale choice is a near-tie or a usability test sits at
its threshold: when the GPU used a different level than the oracle, the GPU's level must be one
the rule could pick with its inputs perturbed within tolerance, and the GPU value must match the
oracle's estimate at that level. A usability test may go either way where the pivot lies within
2 % of min_pivot, or within what FP32 arithmetic can resolve: moment sums rounded by up to
PIVOT_N U32 relative move a pivot of a matrix of condition kappa by up to about PIVOT_N U32 kappa
of itself (with kappa ~1e8, near-singular fits of a few samples at the frame border, the FP32
pivot is undetermined).
"""
from __future__ import annotations

import math

import numpy as np

TAU = 1e-2          # radiance floor of the relative error (the scene's darkest level)
REL_TOL = 1e-5      # FP32 accumulation, plain
U32 = 2.0 ** -24    # unit roundoff of float32
C_FIT = 128.0       # moment sums over up to ~128 samples
C_W = 32.0          # window evaluation and sample-position rounding
HALF_TOL = 2.0 ** -11
PIVOT_N = 64.0      # moment sums of up to ~64 terms: relative rounding PIVOT_N * U32


def rel_err(g, o):
    return np.abs(g - o) / np.maximum(np.abs(o), TAU)


def pivot_band(piv, kappa):
    """How far an FP32 pivot of the equilibrated normal matrix may lie from the FP64 one: a few 1e-6
    absolute for a well-conditioned matrix, and relative to the pivot about (n U32) kappa for a
    matrix of condition kappa (entrywise relative perturbations eps of the moment sums move a pivot
    by up to about eps kappa of itself; eps is the rounding of sums of up to PIVOT_N terms)."""
    k = 0.0 if kappa is None else np.where(np.isfinite(kappa), kappa, 0.0)
    return 1e-5 + PIVOT_N * U32 * k * np.abs(piv)


def admissible_levels(c0, var, valid, pivot, count, J, M, gamma, min_pivot, delta, pivot_rel=0.02, kappa=None):
    """Set of levels the choice rule can reach when every interval end moves by up to `delta`
    and every usability test whose pivot lies within pivot_rel of min_pivot, or within the FP32
    uncertainty of the pivot given the matrix's condition number (`kappa`, optional), may go
    either way."""
    P = [1, 3, 6]
    out = set()

    def usable_options(l):
        order = M if l < J else M - 1 - (l - J)
        if count[l] < P[order]:
            return [False]
        piv = pivot[l]
        # within the band either decision is correct (the oracle reports C_0 for such fits either
        # way); an FP32 factorisation cannot place the pivot of a near-singular matrix more closely
        band = pivot_rel * max(min_pivot, 1e-12) + pivot_band(piv, None if kappa is None else kappa[l])
        if np.isfinite(piv) and abs(piv - min_pivot) <= band and np.isfinite(c0[l]):
            return [True, False]
        return [bool(valid[l])]

    def walk(j, lo, hi, chosen):
        if j == J:
            finish(chosen)
            return
        for ok in usable_options(j):
            if not ok:
                walk(j + 1, lo, hi, chosen)
                continue
            h = gamma * math.sqrt(max(var[j], 0.0))
            nlo, nhi = max(lo, c0[j] - h), min(hi, c0[j] + h)
            gap = nhi - nlo
            if gap >= -delta:          # may be non-empty
                walk(j + 1, nlo, nhi, j)
            if gap <= delta:           # may be empty
                finish(chosen)

    def finish(chosen):
        if chosen >= 0:
            out.add(chosen)
            return
        for i in range(M):
            l = J + i
            opts = usable_options(l)
            if True in opts:
                out.add(l)
            if False not in opts:
                return
        out.add(-1)

    walk(0, -math.inf, math.inf, -1)
    return out


def level_tol(o_val, efit, ew, rel_tol=REL_TOL, extra_rel=0.0):
    """Absolute tolerance of one level's C_0 (see the module docstring)."""
    return rel_tol * np.maximum(np.abs(o_val), TAU) + U32 * (C_FIT * efit + C_W * ew) + \
        extra_rel * np.maximum(np.abs(o_val), TAU)


def compare(gpu_out, gpu_choice, orc, pixels, J, M, gamma, min_pivot, rel_tol=REL_TOL, extra_rel=0.0):
    """Check GPU values [3, n] / choices [3, n] at `pixels` against oracle results with levels.

    Returns a dict of statistics; raises AssertionError with details on the first failures."""
    n = pixels.shape[0]
    ratios = []
    fails = []
    mismatched_choice = 0
    for i in range(n):
        for c in range(3):
            g = float(gpu_out[c, i])
            gch = int(gpu_choice[c, i]) if gpu_choice is not None else None
            och = int(orc["choice"][i, c])
            o = float(orc["out"][i, c])
            if gch == 255:
                gch = -1
            if gch is not None and gch != och:
                lv = orc
                kap = lv["kappa"][i, c] if "kappa" in lv else None
                # levels the GPU may use: usable ones, and those whose usability FP32 cannot decide
                piv = lv["pivot"][i, c]
                ambiguous = np.isfinite(piv) & np.isfinite(lv["c0"][i, c]) & \
                    (np.abs(piv - min_pivot) <= 0.02 * max(min_pivot, 1e-12) + pivot_band(piv, kap))
                ok = lv["valid"][i, c].astype(bool) | ambiguous
                tl = np.where(ok, level_tol(lv["c0"][i, c], lv["efit"][i, c], lv["ew"][i, c], rel_tol), 0.0)
                hs = gamma * np.sqrt(np.maximum(np.where(ok, lv["var"][i, c], 0.0), 0.0))
                delta = 4.0 * float(np.nanmax(tl)) + 1e-4 * float(hs.max())
                adm = admissible_levels(lv["c0"][i, c], lv["var"][i, c], lv["valid"][i, c], lv["pivot"][i, c],
                                        lv["count"][i, c], J, M, gamma, min_pivot, delta=delta, kappa=kap)
                if gch not in adm:
                    fails.append((i, c, "choice", gch, och, sorted(adm), g, o))
                    continue
                mismatched_choice += 1
                o = float(orc["c0"][i, c, gch]) if gch >= 0 else math.nan
                och = gch
            if math.isnan(o) or math.isnan(g):
                if not (math.isnan(o) and math.isnan(g)):
                    fails.append((i, c, "nan", gch, och, None, g, o))
                continue
            tol = float(level_tol(o, orc["efit"][i, c, och], orc["ew"][i, c, och], rel_tol, extra_rel))
            err = abs(g - o)
            ratios.append(err / tol)
            if not err <= tol:
                fails.append((i, c, "value", gch, och, (err, tol), g, o))
    ratios = np.array(ratios) if ratios else np.zeros(1)
    stats = dict(n=len(ratios), median_err_over_tol=float(np.median(ratios)), p99=float(np.quantile(ratios, 0.99)),
                 max=float(ratios.max()), mismatched_choice=mismatched_choice, fails=len(fails))
    if fails:
        lines = [f"  pixel {pixels[f[0]].tolist()} ch {f[1]} {f[2]}: gpu level {f[3]} oracle level {f[4]} "
                 f"info {f[5]} gpu {f[6]!r} oracle {f[7]!r}" for f in fails[:12]]
        raise AssertionError(f"{len(fails)} of {3 * n} pixel-channels fail parity; stats {stats}\n" + "\n".join(lines))
    return stats
