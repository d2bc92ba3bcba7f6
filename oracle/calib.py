"""FP64 definitions of the radiometric calibration estimates of Section 6.2 (test infrastructure).

Only `tests/` and `bench.py`'s CPU legs use this module; the CUDA library shares no code with it.

* `stack_stats`: per-pixel mean and unbiased variance of a stack of raw frames. From black frames
  (lens covered) they are the bias frame b_{s,i} and the read-noise variance Var r_{s,i}; from
  flat-field frames, E[y_{s,i}] and Var y_{s,i}. The sums are exact integers, so the values are
  one FP64 rounding of the exact mean and variance.
* `gain`: Eq. 21, (Var y - Var b) / (E[y] - E[b]) = g_s for Poisson shot noise, pooled over the
  usable pixels as a ratio of sums (reading: the paper states the per-pixel relation only).
* `exposure`: the exposure scaling n_s as the spatial mean of the pixel-wise ratio of the
  radiant-power estimates (Eq. 18 with n = a = 1) of sensor s to those of a reference sensor, and
  the non-uniformity a_{s,i} as each pixel's ratio over n_s (reading: the reference sensor's own
  non-uniformity cannot be separated from the flat field and is taken as 1).

Usable pixels (reading): a flat-field mean at least `min_signal` DN above the black mean and below
`max_level` DN (away from saturation), in every frame pair used.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np


def stack_stats(frames: np.ndarray, width: int) -> Tuple[np.ndarray, np.ndarray]:
    """frames: uint16 [n, height, pitch] (n >= 2). Returns (mean, var) as float32 [height, width]:
    mean = S1 / n and var = (n S2 - S1^2) / (n (n - 1)) from the exact integer sums S1 = sum y,
    S2 = sum y^2, each evaluated as one FP64 division of FP64-rounded integers."""
    n = frames.shape[0]
    y = frames[:, :, :width].astype(np.int64)
    s1 = y.sum(axis=0)
    s2 = (y * y).sum(axis=0)
    mean = s1.astype(np.float64) / np.float64(n)
    var = (np.int64(n) * s2 - s1 * s1).astype(np.float64) / np.float64(n * (n - 1))
    return mean.astype(np.float32), var.astype(np.float32)


def usable(flat_mean, black_mean, min_signal: float, max_level: float) -> np.ndarray:
    fm = flat_mean.astype(np.float64)
    return (fm - black_mean.astype(np.float64) >= min_signal) & (fm < max_level)


def gain(flat_mean, flat_var, black_mean, black_var, min_signal: float, max_level: float):
    """Eq. 21 pooled over usable pixels: sum(Var y - Var b) / sum(E[y] - E[b]); also the count."""
    m = usable(flat_mean, black_mean, min_signal, max_level)
    num = (flat_var.astype(np.float64) - black_var.astype(np.float64))[m].sum()
    den = (flat_mean.astype(np.float64) - black_mean.astype(np.float64))[m].sum()
    return (num / den if den > 0 else np.nan), int(m.sum())


def exposure(flat_mean, black_mean, gain_s: float, exposure_s: float, ref_flat_mean, ref_black_mean,
             ref_gain: float, ref_exposure: float, min_signal: float, max_level: float):
    """Returns (n_s, a_s [height, width] float32, count). rho_i = ((E y - b) / (g t))_s divided by
    the same for the reference sensor at pixel i; n_s = mean rho over pixels usable in both
    sensors; a_{s,i} = rho_i / n_s there and 1 elsewhere."""
    m = usable(flat_mean, black_mean, min_signal, max_level) & usable(ref_flat_mean, ref_black_mean, min_signal,
                                                                      max_level)
    fs = (flat_mean.astype(np.float64) - black_mean.astype(np.float64)) / (gain_s * exposure_s)
    fr = (ref_flat_mean.astype(np.float64) - ref_black_mean.astype(np.float64)) / (ref_gain * ref_exposure)
    rho = np.where(m, fs / np.where(m, fr, 1.0), 0.0)
    cnt = int(m.sum())
    n_s = rho[m].sum() / cnt if cnt else np.nan
    a = np.where(m, rho / n_s, 1.0).astype(np.float32)
    return n_s, a, cnt
