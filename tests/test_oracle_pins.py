"""Pins of the FP64 oracle against what the paper and the mathematics fix.

The paper prints no numeric results, so the oracle is pinned by hand-worked
values (golden fixtures), closed forms, invariants and an independent
brute-force route. Each test names the passage it pins.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

import oracle
from oracle import bruteforce
from paper_1308_4908_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@dataclasses.dataclass
class ValueSensor:
    """Sensor in value mode: the radiant power estimate and its variance are given per pixel."""
    width: int
    height: int
    affine: np.ndarray
    value_f: np.ndarray
    value_var: np.ndarray
    gain: float = 1.0
    exposure: float = 1.0
    nd: float = 1.0
    read_var: float = 1.0
    black: float = 0.0
    sat: float = 1e300
    bias_frame = None
    prnu_frame = None
    read_var_frame = None
    sat_frame = None


def value_rig(fn, n_sensors=3, size=24, seed=7, rot=3.0, trans=1.5, var_fn=None):
    """Value-mode rig whose sample values are fn(c, X, Y) at the transformed positions."""
    r = np.random.default_rng(seed)
    sensors = []
    for s in range(n_sensors):
        A = synth.affine_about_center(size, size, *r.uniform(-trans, trans, 2), r.uniform(-rot, rot),
                                      1.0 + r.uniform(-0.05, 0.05))
        y, x = np.mgrid[0:size, 0:size]
        X, Y = synth.apply_affine(A, x.astype(float), y.astype(float))
        col = synth.cfa_color(x, y)
        f = np.zeros((size, size))
        for c in range(3):
            f[col == c] = fn(c, X[col == c], Y[col == c])
        var = var_fn(s, f) if var_fn else r.uniform(0.5, 2.0, (size, size))
        sensors.append(ValueSensor(size, size, A, f, var))
    return sensors


# ------------------------------------------------------------------ Section 6: radiometry

def test_radiometry_golden():
    """Eqs. 18 and 20 and the saturation rule of Section 6.1, against hand-worked values."""
    rows = [l.split("#")[0].split() for l in open(os.path.join(GOLDEN, "radiometry.txt"))]
    rows = [r for r in rows if r]
    assert len(rows) >= 6
    for r in rows:
        y, b, g, t, a, n, rv, sat = map(float, r[:8])
        excl, f, s2 = int(r[8]), float(r[9]), float(r[10])
        e, fo, so = oracle.radiometry(y, b, g, t, a, n, rv, sat)
        assert e == bool(excl), r
        if not excl:
            assert fo == pytest.approx(f, rel=1e-14), r
            assert so == pytest.approx(s2, rel=1e-14), r


def test_generator_photon_transfer():
    """The generator obeys Section 6.2's gain identity (Var y - Var b)/(E y - E b) = g on a flat field."""
    W = H = 512
    sen = synth.Sensor(W, H, 1.0, synth.affine_about_center(W, H))
    for f0 in (150.0, 600.0):
        raw = synth.simulate_raw(synth.constant_scene(f0), sen, seed=99, index=int(f0))[:, :W].astype(float)
        dark = synth.simulate_raw(synth.constant_scene(1e-12), sen, seed=98, index=int(f0))[:, :W].astype(float)
        g_est = (raw.var() - dark.var()) / (raw.mean() - dark.mean())
        assert g_est == pytest.approx(synth.GAIN_DN_PER_E, rel=0.01)


def test_generator_saturates_and_is_seeded():
    a = synth.paper_scale(size=256)
    b = synth.paper_scale(size=256)
    for sa, sb in zip(a.sensors, b.sensors):
        assert np.array_equal(sa.raw, sb.raw)
        assert np.array_equal(sa.affine, sb.affine)
    assert (a.sensors[0].raw[:, :256] >= synth.CLIP_DN).mean() > 0.005   # the bright sensor clips somewhere
    assert (a.sensors[2].raw[:, :256] >= synth.CLIP_DN).mean() == 0.0


# ------------------------------------------------------------------ Section 5.3: M = 0 closed form

@pytest.mark.parametrize("sigma", [0.7, 1.3])
def test_order0_is_weighted_average(sigma):
    """Eq. 7: for M = 0 the estimate is the window-and-noise weighted average of the samples."""
    fr = synth.tiny()
    p = synth.Params(order=0, sigmas=(sigma,), out_w=64, out_h=64)
    pix = np.array([[5, 7], [31, 32], [0, 0], [63, 40], [17, 2]])
    res = oracle.reconstruct(fr.sensors, p, pix)
    smp = bruteforce.all_samples(fr.sensors)
    for i, (u, v) in enumerate(pix):
        for c in range(3):
            sc = sigma * (p.green_ratio if c == 1 else 1.0)
            d2 = (smp["X"] - u) ** 2 + (smp["Y"] - v) ** 2
            sel = (smp["col"] == c) & (d2 < (3 * sc) ** 2)
            K = np.exp(-d2[sel] / (2 * sc * sc)) - math.exp(-4.5)
            want = np.average(smp["f"][sel], weights=K / smp["s2"][sel])
            assert res["out"][i, c] == pytest.approx(want, rel=1e-12, abs=1e-12)


# ------------------------------------------------------------------ Sections 5.1-5.2: polynomial reproduction

def _poly(deg, seed):
    r = np.random.default_rng(seed)
    coef = r.uniform(-1, 1, (3, 6)) * np.array([50, 3, 3, 0.4, 0.4, 0.4])
    coef[:, 0] += 200.0
    if deg < 2:
        coef[:, 3:] = 0
    if deg < 1:
        coef[:, 1:3] = 0

    def fn(c, X, Y, ox=11.3, oy=12.1):
        dx, dy = X - ox, Y - oy
        return coef[c, 0] + coef[c, 1] * dx + coef[c, 2] * dy + coef[c, 3] * dx * dx + coef[c, 4] * dx * dy + \
            coef[c, 5] * dy * dy
    return fn


@pytest.mark.parametrize("order", [0, 1, 2])
def test_polynomial_reproduction(order):
    """A scene that is a polynomial of degree <= M is reproduced exactly (Sections 5.1-5.2) for any
    rig and any positive weights; one degree higher it is not (so the test can fail)."""
    fn = _poly(order, 3 + order)
    sensors = value_rig(fn)
    p = synth.Params(order=order, sigmas=(0.9, 1.4, 2.2), out_w=24, out_h=24, min_pivot=1e-12)
    pix = np.array([[u, v] for u in range(6, 18, 3) for v in range(6, 18, 4)])
    res = oracle.reconstruct(sensors, p, pix, levels=True)
    for i, (u, v) in enumerate(pix):
        for c in range(3):
            want = fn(c, float(u), float(v))
            for l in range(3):
                assert res["valid"][i, c, l]
                assert res["c0"][i, c, l] == pytest.approx(want, rel=1e-10)
    if order < 2:
        fn2 = _poly(order + 1, 3 + order)
        res2 = oracle.reconstruct(value_rig(fn2), p, pix)
        err = max(abs(res2["out"][i, c] - fn2(c, float(u), float(v))) for i, (u, v) in enumerate(pix) for c in range(3))
        assert err > 1e-6


def test_output_mapping_and_transform_direction():
    """Section 4.2: T_s maps sensor px to reference px and the output grid is a set of points P_j in the
    reference frame. A sensor shifted by (+2, +4) seen through a 2x output grid: output (2u', 2v') sits on
    reference point (u', v'), which is sensor pixel (u' - 2, v' - 4); sigma = 0.1 isolates that sample."""
    W = H = 16
    A = np.array([[1.0, 0, 2.0], [0, 1.0, 4.0]])
    vals = np.arange(W * H, dtype=float).reshape(H, W) + 100.0
    s = ValueSensor(W, H, A, vals, np.ones((H, W)))
    p = synth.Params(order=0, sigmas=(0.1,), out_w=40, out_h=40, out_affine=np.array([[0.5, 0, 0], [0, 0.5, 0]]))
    res = oracle.reconstruct([s], p)
    out = res["out"]
    for yo in range(H):
        for xo in range(W):
            u, v = 2 * (xo + 2), 2 * (yo + 4)
            if u >= 40 or v >= 40:
                continue
            c = synth.cfa_color(xo, yo)
            assert out[c, v, u] == pytest.approx(vals[yo, xo], rel=1e-14)
            for c2 in range(3):
                if c2 != c:
                    assert np.isnan(out[c2, v, u])
    # a 90-degree rotation about the centre permutes the sensor onto the reference grid
    A = synth.affine_about_center(W, H, rot_deg=90.0)
    s = ValueSensor(W, H, A, vals, np.ones((H, W)))
    res = oracle.reconstruct([s], synth.Params(order=0, sigmas=(0.1,), out_w=W, out_h=H))
    for yo in range(H):
        for xo in range(W):
            X, Y = synth.apply_affine(A, np.float64(xo), np.float64(yo))
            u, v = int(round(float(X))), int(round(float(Y)))
            assert res["out"][synth.cfa_color(xo, yo), v, u] == pytest.approx(vals[yo, xo], rel=1e-14)


def test_one_aligned_sensor_matches_input():
    """One aligned sensor, no noise, order 0, sigma 0.1: every output pixel's own colour equals that
    pixel's radiant power estimate (Eq. 18); the other two colours have no sample (NaN)."""
    fr = synth.tiny()
    s = fr.sensors[0]
    s2 = dataclasses.replace(s, affine=np.array([[1.0, 0, 0], [0, 1.0, 0]]))
    s2.raw = synth.simulate_raw(fr.scene, s2, 5, 0, noise=False)
    p = synth.Params(order=0, sigmas=(0.1,), out_w=64, out_h=64)
    out = oracle.reconstruct([s2], p)["out"]
    y = s2.raw[:, :64].astype(float)
    f = (y - s2.black) / (s2.gain * s2.exposure * s2.nd)
    sat = y >= s2.sat
    yy, xx = np.mgrid[0:64, 0:64]
    col = synth.cfa_color(xx, yy)
    for c in range(3):
        m = (col == c) & ~sat
        np.testing.assert_allclose(out[c][m], f[m], rtol=1e-12)
        assert np.isnan(out[c][col != c]).all()
        assert np.isnan(out[c][(col == c) & sat]).all()


def test_symmetric_layout_order1_equals_order0():
    """Symmetric samples and values around P make every odd moment vanish, so M = 1 and M = 0 agree
    (pins the basis of Section 5.1 and its sign conventions)."""
    W = H = 21
    P = (10.0, 10.0)                  # an R site of an aligned sensor: (10, 10) is (even, even)

    def fn(c, X, Y):
        return 100.0 + 7.0 * np.hypot(X - P[0], Y - P[1]) ** 1.5 + 10.0 * c
    y, x = np.mgrid[0:H, 0:W]
    col = synth.cfa_color(x, y)
    f = np.zeros((H, W))
    for c in range(3):
        f[col == c] = fn(c, x[col == c].astype(float), y[col == c].astype(float))
    var = 1.0 + 0.1 * np.hypot(x - P[0], y - P[1])
    s = ValueSensor(W, H, np.array([[1.0, 0, 0], [0, 1.0, 0]]), f, var)
    pix = np.array([[10, 10]])
    r0 = oracle.reconstruct([s], synth.Params(order=0, sigmas=(1.5,), out_w=W, out_h=H), pix)["out"]
    r1 = oracle.reconstruct([s], synth.Params(order=1, sigmas=(1.5,), out_w=W, out_h=H), pix)["out"]
    np.testing.assert_allclose(r1, r0, rtol=1e-12)
    # off-centre the symmetry is gone and the two orders differ
    pix = np.array([[11, 10]])
    r0 = oracle.reconstruct([s], synth.Params(order=0, sigmas=(1.5,), out_w=W, out_h=H), pix)["out"]
    r1 = oracle.reconstruct([s], synth.Params(order=1, sigmas=(1.5,), out_w=W, out_h=H), pix)["out"]
    assert abs(r1[0, 0] - r0[0, 0]) > 1e-6


# ------------------------------------------------------------------ invariants

def test_sensor_order_independence():
    """The fit sums over all samples (Section 5.2), so permuting the sensors changes nothing but the
    rounding order: the difference stays within a few units of double rounding times the condition
    number of the chosen fit."""
    fr = synth.paper_scale(size=96)
    pix = np.random.default_rng(1).integers(0, 96, (300, 2))
    a = oracle.reconstruct(fr.sensors, fr.params, pix, levels=True, kappa=True)
    kap = np.take_along_axis(a["kappa"], np.maximum(a["choice"], 0)[:, :, None], axis=2)[:, :, 0]
    tol = 1e-13 + 20 * np.finfo(float).eps * kap
    for perm in ([2, 1, 0], [1, 2, 0]):
        b = oracle.reconstruct([fr.sensors[i] for i in perm], fr.params, pix, levels=True)
        np.testing.assert_array_equal(b["choice"], a["choice"])
        rel = np.abs(b["out"] - a["out"]) / np.maximum(np.abs(a["out"]), 1e-2)
        assert np.all(rel <= tol)


def test_equivalent_kernel_moments():
    """Section 5.2: the solution is a linear filter. Its weights reproduce constants, cancel the
    monomials up to degree M, and applied to the samples give C_0; Var C_0 = sum l_k^2 s2_k."""
    fr = synth.paper_scale(size=64)
    for order in (0, 1, 2):
        p = dataclasses.replace(fr.params, order=order, sigmas=(1.2,))
        ek = oracle.equivalent_kernel(fr.sensors, p, 30, 33, 1, 1.2, order)
        assert ek is not None and len(ek["ell"]) > 6
        l, dx, dy = ek["ell"], ek["dx"], ek["dy"]
        assert l.sum() == pytest.approx(1.0, abs=1e-12)
        mon = [dx, dy] if order >= 1 else []
        mon += [dx * dx, dx * dy, dy * dy] if order >= 2 else []
        for m in mon:
            assert abs((l * m).sum()) < 1e-11
        res = oracle.reconstruct(fr.sensors, p, np.array([[30, 33]]), levels=True)
        assert res["c0"][0, 1, 0] == pytest.approx((l * ek["f"]).sum(), rel=1e-12)
        s2 = np.array([_sample_var(fr.sensors[s], x, y) for s, x, y in zip(ek["sensor"], ek["x"], ek["y"])])
        assert res["var"][0, 1, 0] == pytest.approx((l * l * s2).sum(), rel=1e-11)


def _sample_var(sen, x, y):
    _, _, s2 = oracle.radiometry(sen.raw[y, x], sen.black, sen.gain, sen.exposure, 1.0, sen.nd, sen.read_var,
                                 sen.sat)
    return s2


def test_variance_monte_carlo():
    """Var C_0 is the variance of the estimate when the samples carry independent Gaussian noise of
    the stated variances (Section 6.1): checked against 3000 noise draws."""
    fn = _poly(1, 11)
    base = value_rig(fn, n_sensors=2, size=20, seed=4)
    p = synth.Params(order=2, sigmas=(1.1,), out_w=20, out_h=20, min_pivot=1e-12)
    pix = np.array([[9, 10], [12, 8]])
    ref = oracle.reconstruct(base, p, pix, levels=True)
    r = np.random.default_rng(0)
    draws = []
    for _ in range(3000):
        noisy = [dataclasses.replace(s, value_f=s.value_f + r.standard_normal(s.value_f.shape) * np.sqrt(s.value_var))
                 for s in base]
        draws.append(oracle.reconstruct(noisy, p, pix)["out"])
    draws = np.array(draws)
    emp = draws.var(axis=0, ddof=1)
    want = ref["var"][:, :, 0]
    # sampling error of a variance from n draws: sqrt(2/(n-1)) ~ 2.6 %; allow 4 sigma
    np.testing.assert_allclose(emp, want, rtol=0.105)
    np.testing.assert_allclose(draws.mean(axis=0), ref["c0"][:, :, 0], atol=float(4 * np.sqrt(want.max() / 3000)))


def test_constant_scene_mean_and_scale_choice():
    """A constant scene with noise: the estimate is unbiased when the sample variances are known, and
    the widest window (smallest variance) is chosen almost everywhere at gamma = 2."""
    f0 = 300.0

    def fn(c, X, Y):
        return np.full(np.shape(X), f0)
    sensors = value_rig(fn, n_sensors=3, size=160, seed=2, rot=0.2, var_fn=lambda s, f: np.full(f.shape, f0 * (1 + s)))
    r = np.random.default_rng(5)
    for s in sensors:
        s.value_f = s.value_f + r.standard_normal(s.value_f.shape) * np.sqrt(s.value_var)
    p = synth.Params(order=2, sigmas=synth.PAPER_SCALES, out_w=160, out_h=160)
    pix = np.array([[u, v] for u in range(12, 150, 12) for v in range(12, 150, 12)])   # windows do not overlap
    res = oracle.reconstruct(sensors, p, pix, levels=True)
    out = res["out"]
    v_chosen = np.take_along_axis(res["var"], res["choice"][:, :, None], axis=2)[:, :, 0]
    z = (out.mean(axis=0) - f0) / np.sqrt(v_chosen.mean(axis=0) / len(pix))
    assert np.all(np.abs(z) < 4.5), z
    assert (res["choice"] == len(p.sigmas) - 1).mean() >= 0.90


# ------------------------------------------------------------------ scale choice and fallbacks

def test_ici_golden():
    """The scale-choice rule on hand-built interval lists."""
    n = 0
    for line in open(os.path.join(GOLDEN, "ici_cases.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        g, c0, var, valid, want = [x.split() for x in line.split("|")]
        ch, _ = oracle.ici([float(x) for x in c0], [float(x) for x in var], [int(x) for x in valid], float(g[0]))
        assert ch == int(want[0]), line
        n += 1
    assert n == 7


def test_order_fallback_and_empty():
    """No usable order-2 scale -> the order is lowered at the largest scale; no sample at all -> NaN."""
    fr = synth.tiny()
    p = synth.Params(order=2, sigmas=(0.3, 0.45), out_w=64, out_h=64)
    res = oracle.reconstruct(fr.sensors[:1], p, np.array([[20, 20], [21, 20], [5000, 5000]]), levels=True)
    J = 2
    ch = res["choice"]
    assert (ch[:2] >= J).all()                   # fallback levels
    for i in range(2):
        for c in range(3):
            l = ch[i, c]
            assert res["valid"][i, c, l] and not res["valid"][i, c, :J].any()
            assert res["out"][i, c] == res["c0"][i, c, l]
    assert (ch[2] == -1).all() and np.isnan(res["out"][2]).all()


def test_saturated_sample_is_dropped():
    """Section 6.1: a saturated sample contributes nothing; the result equals the fit without it."""
    fr = synth.tiny()
    s = fr.sensors[0]
    raw = s.raw.copy()
    raw[30, 31] = synth.CLIP_DN                       # a G site next to output pixel (31, 30)
    s_sat = dataclasses.replace(s, raw=raw)
    p = synth.Params(order=1, sigmas=(1.0,), out_w=64, out_h=64)
    pix = np.array([[31, 30], [32, 30]])
    a = oracle.reconstruct([s_sat, fr.sensors[1]], p, pix)["out"]
    # the same sample removed through a per-pixel saturation frame on the original data
    sat = np.full((64, 64), float(synth.CLIP_DN))
    sat[30, 31] = 0.0
    b = oracle.reconstruct([dataclasses.replace(s, sat_frame=sat), fr.sensors[1]], p, pix)["out"]
    np.testing.assert_array_equal(a, b)
    c = oracle.reconstruct(fr.sensors, p, pix)["out"]
    assert abs(a[0, 1] - c[0, 1]) > 0


def test_per_pixel_calibration_frames_match_scalars():
    """Per-pixel bias, non-uniformity, read variance and saturation frames (Sections 4.1, 6) equal to the
    scalar values give the same result; varying frames agree with the brute-force route."""
    fr = synth.paper_scale(size=32)
    p = dataclasses.replace(fr.params, sigmas=(0.8, 1.8))
    pix = np.array([[7, 9], [16, 16], [30, 2]])
    a = oracle.reconstruct(fr.sensors, p, pix)["out"]
    fs = [dataclasses.replace(s, bias_frame=np.full((32, 32), s.black), prnu_frame=np.ones((32, 32)),
                              read_var_frame=np.full((32, 32), s.read_var),
                              sat_frame=np.full((32, 32), float(s.sat))) for s in fr.sensors]
    b = oracle.reconstruct(fs, p, pix)["out"]
    np.testing.assert_array_equal(a, b)
    r = np.random.default_rng(3)
    fv = [dataclasses.replace(s, bias_frame=s.black + r.uniform(-3, 3, (32, 32)),
                              prnu_frame=r.uniform(0.9, 1.1, (32, 32)),
                              read_var_frame=r.uniform(5, 15, (32, 32)),
                              sat_frame=np.full((32, 32), 4000.0)) for s in fr.sensors]
    res = oracle.reconstruct(fv, p, pix, levels=True)
    smp = bruteforce.all_samples(fv)
    for i, (u, v) in enumerate(pix):
        for c in range(3):
            sc = 1.8 * (p.green_ratio if c == 1 else 1.0)
            c0, var, n = bruteforce.fit_point(smp, (u, v), c, sc, 2)
            assert res["count"][i, c, 1] == n
            if res["valid"][i, c, 1]:
                assert res["c0"][i, c, 1] == pytest.approx(c0, rel=1e-9)
                assert res["var"][i, c, 1] == pytest.approx(var, rel=1e-9)


# ------------------------------------------------------------------ independent route

@pytest.mark.parametrize("weight_mode", [0, 1])
@pytest.mark.parametrize("order", [0, 1, 2])
def test_against_bruteforce_qr(order, weight_mode):
    """The C route (search box, normal equations, LDL^T) against brute-force enumeration + Householder
    QR on a 16x16 rotated three-sensor rig, at every level, in raw mode (Eqs. 6, 18, 20), with the
    inverse-variance weight and with the printed weight K / s."""
    fr = synth.paper_scale(size=16, seed=77)
    for s, rot in zip(fr.sensors, (0.0, 6.0, -4.0)):
        s.affine = synth.affine_about_center(16, 16, 0.3, -0.2, rot, 1.01)
        s.raw = synth.simulate_raw(fr.scene, s, 77, rot != 0)
    p = dataclasses.replace(fr.params, order=order, min_pivot=1e-9, weight_mode=weight_mode)
    pix = np.array([[u, v] for u in range(0, 16, 3) for v in range(1, 16, 3)])
    res = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    smp = bruteforce.all_samples(fr.sensors)
    checked = 0
    for i, (u, v) in enumerate(pix):
        for c in range(3):
            for l, sg in enumerate(p.sigmas):
                sc = sg * (p.green_ratio if c == 1 else 1.0)
                c0, var, n = bruteforce.fit_point(smp, (float(u), float(v)), c, sc, order, weight_mode=weight_mode)
                assert res["count"][i, c, l] == n
                if res["valid"][i, c, l]:
                    # both routes carry rounding of order (double epsilon) x (condition number)
                    tol = 1e-12 + 50 * np.finfo(float).eps * res["kappa"][i, c, l]
                    assert res["c0"][i, c, l] == pytest.approx(c0, rel=tol, abs=tol)
                    assert res["var"][i, c, l] == pytest.approx(var, rel=10 * tol)
                    checked += 1
    assert checked > 100


def test_printed_window_form_is_sigma_sqrt_h_over_2():
    """The printed window exp(-|d|^2 / h) with h_G = h_RB / sqrt 2 (Section 5.3.1) is the kernel's
    exp(-|d|^2 / (2 sigma^2)) at sigma = sqrt(h / 2) with green_ratio = 2^(-1/4): the oracle run with
    those parameters against the brute-force route evaluating the printed form directly."""
    fr = synth.paper_scale(size=16, seed=78)
    hs = (0.6, 1.4, 3.0)
    p = dataclasses.replace(fr.params, order=1, sigmas=tuple(math.sqrt(h / 2) for h in hs),
                            green_ratio=2 ** -0.25, min_pivot=1e-9)
    pix = np.array([[u, v] for u in range(1, 16, 4) for v in range(0, 16, 4)])
    res = oracle.reconstruct(fr.sensors, p, pix, levels=True, kappa=True)
    smp = bruteforce.all_samples(fr.sensors)
    checked = 0
    for i, (u, v) in enumerate(pix):
        for c in range(3):
            for l, h in enumerate(hs):
                hc = h / math.sqrt(2.0) if c == 1 else h
                c0, var, n = bruteforce.fit_point(smp, (float(u), float(v)), c, 0.0, 1, h_c=hc)
                assert res["count"][i, c, l] == n
                if res["valid"][i, c, l]:
                    tol = 1e-12 + 50 * np.finfo(float).eps * res["kappa"][i, c, l]
                    assert res["c0"][i, c, l] == pytest.approx(c0, rel=tol, abs=tol)
                    checked += 1
    assert checked > 60
