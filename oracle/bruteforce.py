"""Brute-force second route of the oracle (test infrastructure; tiny rigs only).

Written independently of `lpa_oracle.c` so that each checks the other:

* every pixel of every sensor is a candidate sample (no search box);
* positions are X = T_s(x) (Section 4.2); colour from the RGGB layout (Section 2.5);
* f and its variance from Eqs. 18 and 20 of Section 6 (variance with f clamped
  at zero), saturated samples dropped (Section 6.1);
* the weighted least-squares fit of Section 5.2 (Eq. 6) is solved as an
  ordinary least-squares problem sqrt(W) Phi C = sqrt(W) f by Householder QR
  (numpy.linalg.qr), with Var C_0 = e_0^T R^{-1} R^{-T} (Phi^T W S W Phi)
  R^{-1} R^{-T} e_0.

It reports C_0, Var C_0 and the sample count per (channel, scale, order) and
makes no scale choice.
"""
from __future__ import annotations

import math
from typing import Dict, Sequence

import numpy as np


def all_samples(sensors: Sequence) -> Dict[str, np.ndarray]:
    xs_all, ys_all, X_all, Y_all, col_all, f_all, s2_all = [], [], [], [], [], [], []
    for s in sensors:
        H, W = s.height, s.width
        y, x = np.mgrid[0:H, 0:W]
        A = np.asarray(s.affine, dtype=np.float64).reshape(2, 3)
        X = A[0, 0] * x + A[0, 1] * y + A[0, 2]
        Y = A[1, 0] * x + A[1, 1] * y + A[1, 2]
        col = np.full((H, W), 1)
        col[(x % 2 == 0) & (y % 2 == 0)] = 0
        col[(x % 2 == 1) & (y % 2 == 1)] = 2
        if getattr(s, "value_f", None) is not None:
            f = np.asarray(s.value_f, dtype=np.float64).reshape(H, W)
            s2 = np.asarray(s.value_var, dtype=np.float64).reshape(H, W)
            keep = np.isfinite(s2) & (s2 > 0) & np.isfinite(f)
        else:
            yv = np.asarray(s.raw, dtype=np.float64)[:, :W]
            b = s.bias_frame if s.bias_frame is not None else s.black
            a = s.prnu_frame if s.prnu_frame is not None else 1.0
            rv = s.read_var_frame if s.read_var_frame is not None else s.read_var
            sat = s.sat_frame if s.sat_frame is not None else s.sat
            gtan = s.gain * s.exposure * a * s.nd
            f = (yv - b) / gtan
            s2 = (s.gain ** 2 * s.exposure * a * s.nd * np.maximum(f, 0.0) + rv) / gtan ** 2
            keep = yv < sat
            f = np.broadcast_to(f, (H, W))
            s2 = np.broadcast_to(s2, (H, W))
        xs_all.append(x[keep]); ys_all.append(y[keep]); X_all.append(X[keep]); Y_all.append(Y[keep])
        col_all.append(col[keep]); f_all.append(f[keep]); s2_all.append(s2[keep])
    cat = lambda l: np.concatenate(l) if l else np.zeros(0)
    return dict(x=cat(xs_all), y=cat(ys_all), X=cat(X_all), Y=cat(Y_all), col=cat(col_all).astype(int),
                f=cat(f_all), s2=cat(s2_all))


def fit_point(samples: Dict[str, np.ndarray], P, color: int, sigma_c: float, order: int,
              trunc_k: float = 3.0, weight_mode: int = 0, h_c: float = None):
    """C_0, Var C_0 and count for one channel at one (colour-adjusted) scale; C_0 is NaN if rank deficient.

    With `h_c` the window is the printed form of Eq. 8, exp(-|d|^2 / h_c), on |d|^2 < k^2 h_c / 2
    (the same k-sigma support), and sigma_c is not used."""
    dx = samples["X"] - P[0]
    dy = samples["Y"] - P[1]
    r2 = dx * dx + dy * dy
    support = (trunc_k * sigma_c) ** 2 if h_c is None else trunc_k ** 2 * h_c / 2.0
    sel = (samples["col"] == color) & (r2 < support)
    dx, dy, r2 = dx[sel], dy[sel], r2[sel]
    f, s2 = samples["f"][sel], samples["s2"][sel]
    n = int(sel.sum())
    cols = [np.ones(n)]
    if order >= 1:
        cols += [dx, dy]
    if order >= 2:
        cols += [dx * dx, dx * dy, dy * dy]
    Phi = np.stack(cols, axis=1)
    K = (np.exp(-r2 / (2 * sigma_c ** 2)) if h_c is None else np.exp(-r2 / h_c)) - math.exp(-0.5 * trunc_k ** 2)
    w = K / np.sqrt(s2) if weight_mode == 1 else K / s2
    p = Phi.shape[1]
    if n < p:
        return math.nan, math.nan, n
    sw = np.sqrt(w)
    Q, R = np.linalg.qr(sw[:, None] * Phi)
    if np.min(np.abs(np.diag(R))) <= 1e-12 * np.max(np.abs(np.diag(R))):
        return math.nan, math.nan, n
    coef = np.linalg.solve(R, Q.T @ (sw * f))
    e0 = np.zeros(p); e0[0] = 1.0
    ell = np.linalg.solve(R, np.linalg.solve(R.T, e0))     # (Phi^T W Phi)^{-1} e_0
    Bm = (Phi * (w * w * s2)[:, None]).T @ Phi
    return float(coef[0]), float(ell @ Bm @ ell), n
