"""Pins of the calibration oracle (Section 6.2): closed forms and recovery of known camera
parameters from synthetic black and flat-field stacks (Eqs. 16-17, 21)."""
import numpy as np

from oracle import calib
from paper_1308_4908_gb300 import synth


def test_stack_stats_closed_form():
    """Frames base + k, k = 0..n-1: mean base + (n-1)/2, unbiased variance n (n+1) / 12, exactly."""
    n, h, w = 37, 5, 9
    base = np.arange(h * w, dtype=np.int64).reshape(h, w) * 7 + 100
    frames = np.zeros((n, h, 16), np.uint16)
    for k in range(n):
        frames[k, :, :w] = base + k
    mean, var = calib.stack_stats(frames, w)
    np.testing.assert_array_equal(mean, (base + (n - 1) / 2).astype(np.float32))
    np.testing.assert_array_equal(var, np.full((h, w), n * (n + 1) / 12, np.float32))


def test_stack_stats_constant_and_two_frames():
    frames = np.full((4, 3, 8), 4095, np.uint16)
    mean, var = calib.stack_stats(frames, 8)
    assert (mean == 4095).all() and (var == 0).all()
    frames = np.zeros((2, 1, 8), np.uint16)
    frames[1] = 10
    mean, var = calib.stack_stats(frames, 8)
    assert (mean == 5).all() and (var == 50).all()      # (0 - 5)^2 + (10 - 5)^2 over n - 1 = 1


def test_bias_read_noise_and_gain_are_recovered():
    """Black and flat stacks of a camera with g = 2 DN/e-, Var r = 9 DN^2, bias 64 DN."""
    g, rv, bias = 2.0, 9.0, 64.0
    black = synth.flat_stack(11, 32, 64, 64, 0.0, g, rv, bias)
    flat = synth.flat_stack(12, 32, 64, 64, 600.0, g, rv, bias)
    bm, bv = calib.stack_stats(black, 64)
    fm, fv = calib.stack_stats(flat, 64)
    assert abs(bm.mean() - bias) < 0.05
    assert abs(bv.mean() - (rv + 1 / 12)) < 0.2             # rounding to integers adds 1/12 DN^2
    est, used = calib.gain(fm, fv, bm, bv, 20.0, 3800.0)
    assert used == 64 * 64
    assert abs(est - g) / g < 0.02


def test_gain_excludes_dark_and_saturated_pixels():
    fm = np.array([[100.0, 4090.0, 70.0]], np.float32)
    bm = np.full((1, 3), 64.0, np.float32)
    fv = np.array([[81.0, 0.0, 20.0]], np.float32)
    bv = np.full((1, 3), 9.0, np.float32)
    est, used = calib.gain(fm, fv, bm, bv, 20.0, 4000.0)
    assert used == 1 and est == (81.0 - 9.0) / (100.0 - 64.0)


def test_exposure_scaling_and_nonuniformity_are_recovered():
    """A sensor behind ND 1/8 with a known 2 % non-uniformity, exposed 1 time unit, against an ND 1
    reference exposed 1/8 (Section 6.2: exposure times chosen so both are well exposed) on a
    flat field of 12000 e- per time unit: n_s = mean(a) / 8."""
    r = np.random.default_rng(5)
    prnu = (1.0 + 0.02 * r.standard_normal((64, 64))).clip(0.9, 1.1)
    g, f = 2.0, 12000.0
    ref = synth.flat_stack(21, 32, 64, 64, f / 8, g, 9.0, 64.0, nd=1.0)
    sen = synth.flat_stack(22, 32, 64, 64, f, g, 9.0, 64.0, nd=1 / 8, prnu=prnu)
    black = synth.flat_stack(23, 32, 64, 64, 0.0, g, 9.0, 64.0)
    bm, _ = calib.stack_stats(black, 64)
    rm, _ = calib.stack_stats(ref, 64)
    sm, _ = calib.stack_stats(sen, 64)
    n_s, a, cnt = calib.exposure(sm, bm, g, 1.0, rm, bm, g, 1 / 8, 20.0, 3800.0)
    assert cnt == 64 * 64
    assert abs(n_s - np.mean(prnu) / 8) < 0.001
    assert abs(a.astype(np.float64).mean() - 1.0) < 1e-6    # a = rho / mean(rho)
    assert np.corrcoef(a.ravel(), prnu.ravel())[0, 1] > 0.9
    # forgetting the reference's shorter exposure would make n_s eight times too large
    wrong, _, _ = calib.exposure(sm, bm, g, 1.0, rm, bm, g, 1.0, 20.0, 3800.0)
    assert abs(wrong - 8 * n_s) < 1e-12 * wrong
